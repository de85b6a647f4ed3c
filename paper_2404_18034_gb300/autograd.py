"""torch.autograd.Function over the batched solve's converged outputs.

    fuel, touch = pdg_outputs(x0, solver, n_nodes)

returns, per instance, the fuel m_1 - m_N and the touchdown error of the
converged trajectory; backward calls the hand-written adjoint kernels
(pdg_mc_grad_batch) with the upstream cotangents and returns d/d x0 (the
gradient of the solve's last SCP iteration, see include/pdg_mc.h).
"""
from __future__ import annotations

import torch


class PDGOutputs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, solver, n_nodes=None):
        x0c = x0.detach().contiguous()
        zero = torch.zeros(x0c.shape[0], dtype=torch.float64, device=x0c.device)
        o = solver.grad(x0c, n_nodes, zero, zero)
        ctx.solver = solver
        ctx.n_nodes = n_nodes
        ctx.save_for_backward(x0c)
        return o["fuel"], o["touch"]

    @staticmethod
    def backward(ctx, g_fuel, g_touch):
        (x0c,) = ctx.saved_tensors
        B = x0c.shape[0]
        z = torch.zeros(B, dtype=torch.float64, device=x0c.device)
        gf = z if g_fuel is None else g_fuel.contiguous().to(torch.float64)
        gt = z if g_touch is None else g_touch.contiguous().to(torch.float64)
        o = ctx.solver.grad(x0c, ctx.n_nodes, gf, gt)
        return o["grad"], None, None


def pdg_outputs(x0, solver, n_nodes=None):
    return PDGOutputs.apply(x0, solver, n_nodes)
