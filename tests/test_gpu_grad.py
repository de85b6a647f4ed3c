"""Adjoint gradients (pdg_mc_grad_batch) against central finite differences
(h = 1e-6) of the oracle's last SCP iteration as a function of x0, replayed at
the GPU's recorded counts and step size, and against the oracle's independent
implicit-function gradient of that iteration (oracle/pdg_grad.py)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18034_gb300 import build
    build.build()
    return torch


def _fd(oracle, p, x0, X, U, ws, sig, n, h=1e-6):
    d = len(x0)
    g = np.zeros((d, 2))
    for j in range(d):
        e = np.zeros(d); e[j] = h
        fp = np.array(oracle.final_iteration_outputs(p, x0 + e, X, U, ws, sig, n))
        fm = np.array(oracle.final_iteration_outputs(p, x0 - e, X, U, ws, sig, n))
        g[j] = (fp - fm) / (2 * h)
    return g


@pytest.mark.parametrize("nu,N,B,ov", [(4, 15, 6, {}), (4, 10, 3, {}), (7, 12, 2, {}),
                                        (4, 12, 3, {"glide_slope": 1, "dt_min": 0.3, "dt_max": 0.55}),
                                        (4, 15, 4, {"model": "3dof"}),
                                        (4, 11, 3, {"model": "3dof", "glide_slope": 1}),
                                        (4, 10, 3, {"pipg_form": 2}), (4, 10, 3, {"pipg_form": 3})])
def test_gradient_matches_oracle_finite_differences(torch_cuda, oracle, inputs, nu, N, B, ov):
    """Both models: the 6-DoF one of Sec. 4 and the 3-DoF instance of the
    template (gradient d L / d (m_wet, r, v) there).  With the shared-memory
    PIPG form the solve records the last PIPG loop's checkpoints for the
    adjoint; with the register forms (pipg_form 2 and 3) the adjoint reruns
    that loop itself: both paths are checked."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import Solver
    ov = dict(ov)
    form = ov.pop("pipg_form", 0)
    p = inputs.load_params(nu=nu, model=ov.pop("model", None), **ov)
    S = Solver(p, N)
    if form:
        S.set_pipg_form(form)
    x0 = inputs.dispersion(p, B, inputs.config_seed(3), "bj")
    d = torch.from_numpy(x0).cuda()
    sol = S.solve(d, mode=1, trace=True)
    ones = torch.ones(B, dtype=torch.float64, device="cuda")
    zeros = torch.zeros_like(ones)
    gfu = S.grad(d, None, ones, zeros)
    gtd = S.grad(d, None, zeros, ones)
    torch.cuda.synchronize()
    tr = sol["trace"].cpu().numpy()
    sc = sol["scp_iters"].cpu().numpy()
    st = sol["status"].cpu().numpy()
    np.testing.assert_array_equal(gfu["status"].cpu().numpy(), st)
    np.testing.assert_allclose(gfu["fuel"].cpu().numpy(), sol["fuel"].cpu().numpy(), rtol=1e-12, atol=1e-12)
    compared = 0
    for b in range(B):
        if st[b] not in (0, 1):
            continue
        compared += 1
        X, U, ws, sig, n = oracle.final_iteration_state(p, N, x0[b], tr[b], int(sc[b]))
        fd = _fd(oracle, p, x0[b], X, U, ws, sig, n)
        g1 = gfu["grad"][b].cpu().numpy()
        g2 = gtd["grad"][b].cpu().numpy()
        assert np.all(np.abs(g1 - fd[:, 0]) <= 1e-6 + 1e-5 * np.abs(fd[:, 0])), (b, g1, fd[:, 0])
        assert np.all(np.abs(g2 - fd[:, 1]) <= 1e-9 + 1e-4 * np.abs(fd[:, 1])), (b, g2, fd[:, 1])
        f0, t0 = oracle.final_iteration_outputs(p, x0[b], X, U, ws, sig, n)
        assert abs(gtd["touch"][b].item() - t0) <= 1e-9 + 1e-6 * abs(t0)
    assert compared >= 1
    S.close()


def _grads(torch, S, x0):
    """Solve, then the gradients of fuel and of the touchdown error (one
    adjoint call each, unit cotangents); numpy outputs."""
    d = torch.from_numpy(x0).cuda()
    sol = S.solve(d, mode=1, trace=True)
    ones = torch.ones(x0.shape[0], dtype=torch.float64, device="cuda")
    zeros = torch.zeros_like(ones)
    gfu = S.grad(d, None, ones, zeros)
    gtd = S.grad(d, None, zeros, ones)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in sol.items()}
    out["g_fuel"] = gfu["grad"].cpu().numpy()
    out["g_touch"] = gtd["grad"].cpu().numpy()
    return out


def test_gradient_workload_64_sampled_instances(torch_cuda, oracle, inputs):
    """The gradient workload: B = 4096, N = 15, FP64.  64 instances drawn by a
    seeded generator from those that end converged or at the SCP cap are
    checked against central differences (h = 1e-6) of the oracle's last SCP
    iteration at the GPU's counts, to 1e-6 + 1e-5 relative for fuel and
    1e-9 + 1e-4 relative for the touchdown error.  The implicit-function
    gradient of the same iteration with its subproblem solved exactly is
    computed beside it and its distance from the adjoint's is printed: the
    solver's last PIPG loop (2000 iterations from its warm start) is a
    truncated solve, so the two differ by its truncation."""
    torch = torch_cuda
    from oracle import pdg_grad as G
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params()
    N, B = 15, 4096
    S = Solver(p, N)
    x0 = inputs.dispersion(p, B, inputs.config_seed(3), "bj")
    o = _grads(torch, S, x0)
    ok = np.nonzero(np.isin(o["status"], (0, 1)))[0]
    assert len(ok) >= 0.95 * B
    sample = np.sort(np.random.default_rng(4).choice(ok, 64, replace=False))

    def check(b):
        X, U, ws, sig, n = oracle.final_iteration_state(p, N, x0[b], o["trace"][b], int(o["scp_iters"][b]))
        fd = _fd(oracle, p, x0[b], X, U, ws, sig, n)
        guess = ws.copy()
        _, qp = G._qp_at(p, x0[b], X, U)
        oracle.pipgc(p, qp, sig, guess, force_iters=20000)
        gi, e = G.grad_ift(p, x0[b], X, U, guess)
        return b, fd, gi, e["kkt"]

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(check, sample))
    gap = []
    for b, fd, gi, kkt in res:
        g1, g2 = o["g_fuel"][b], o["g_touch"][b]
        assert np.all(np.abs(g1 - fd[:, 0]) <= 1e-6 + 1e-5 * np.abs(fd[:, 0])), (b, g1, fd[:, 0])
        assert np.all(np.abs(g2 - fd[:, 1]) <= 1e-9 + 1e-4 * np.abs(fd[:, 1])), (b, g2, fd[:, 1])
        if kkt <= 1e-10:
            gap.append(np.abs(g1 - gi[:, 0]).max() / np.abs(gi[:, 0]).max())
    assert len(res) == 64
    print(f"64 sampled gradients match the oracle's differences; adjoint vs implicit gradient of the exact "
          f"subproblem ({len(gap)} instances): fuel relative gap median {np.median(gap):.2e}, max {np.max(gap):.2e}")
    S.close()


def test_gradient_tends_to_the_implicit_gradient(torch_cuda, oracle, inputs):
    """With the last PIPG loop run long (pipg_jmax = 20000, stop tolerance
    1e-12), the adjoint of the unrolled loop must approach the oracle's
    implicit-function gradient of the exactly solved subproblem: fuel to
    1e-5 of its largest component, touchdown error to 1e-11 + 1e-3 relative.
    The two share nothing: the adjoint runs the loop backwards on the GPU,
    the oracle solves the KKT system of the subproblem's active set."""
    torch = torch_cuda
    from oracle import pdg_grad as G
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params(pipg_jmax=20000, pipg_eps_rel=1e-12, pipg_eps_abs=1e-15)
    N, B = 10, 6
    S = Solver(p, N)
    x0 = inputs.dispersion(p, B, inputs.config_seed(3), "bj")
    o = _grads(torch, S, x0)
    compared = 0
    for b in range(B):
        if o["status"][b] not in (0, 1):
            continue
        J = int(o["scp_iters"][b])
        assert o["trace"][b, J - 1, 1] >= 5000
        X, U, ws, sig, n = oracle.final_iteration_state(p, N, x0[b], o["trace"][b], J)
        guess = ws.copy()
        _, qp = G._qp_at(p, x0[b], X, U)
        oracle.pipgc(p, qp, sig, guess, force_iters=40000)
        gi, e = G.grad_ift(p, x0[b], X, U, guess)
        assert e["kkt"] <= 1e-10
        g1, g2 = o["g_fuel"][b], o["g_touch"][b]
        assert np.abs(g1 - gi[:, 0]).max() <= 1e-5 * np.abs(gi[:, 0]).max(), (b, g1, gi[:, 0])
        assert np.all(np.abs(g2 - gi[:, 1]) <= 1e-11 + 1e-3 * np.abs(gi[:, 1])), (b, g2, gi[:, 1])
        compared += 1
    assert compared >= B - 1
    S.close()


def test_autograd_function(torch_cuda, inputs):
    torch = torch_cuda
    from paper_2404_18034_gb300.autograd import pdg_outputs
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params()
    S = Solver(p, 10)
    x0 = torch.from_numpy(inputs.dispersion(p, 4, 17, "bj")).cuda().requires_grad_(True)
    fuel, touch = pdg_outputs(x0, S)
    (fuel.sum() + 3.0 * touch.sum()).backward()
    ref = S.grad(x0.detach(), None, torch.ones(4, dtype=torch.float64, device="cuda"),
                 3.0 * torch.ones(4, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    np.testing.assert_allclose(x0.grad.cpu().numpy(), ref["grad"].cpu().numpy(), rtol=1e-12, atol=1e-15)
    S.close()
