"""A model supplied by the caller: tests/models/pdg_model_3dof_drag.cuh (the
3-DoF model with quadratic drag, c_D in pdg_params.model_params[0]) compiled
into the solver through PDG_MODEL_HEADER by build.build_model.

The oracle has no drag model, so the reference here is the 3-DoF oracle's
augmented dynamics f plus the drag term, integrated by an RK4 with FOH
controls written in this file, and central differences of that flow for the
state-transition blocks.  With c_D = 0 the model must reproduce the built-in
3-DoF library."""
import os

import numpy as np
import pytest

from gpu_helpers import assert_scaled_close

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "models", "pdg_model_3dof_drag.cuh")


@pytest.fixture(scope="module")
def drag_lib(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18034_gb300 import build
    build.build()
    return build.build_model(HEADER, str(tmp_path_factory.mktemp("user") / "libpdg_mc_drag.so"))


def _params(inputs, cd, **ov):
    p = inputs.load_params(model="3dof", **ov)
    p["model"] = "custom"
    p["model_params"] = [cd]
    return p


def _f_drag(oracle, p3, cd, x, u):
    """s (F, sum |g|_+^2) of the drag model: the 3-DoF oracle's f plus the drag term."""
    f = oracle.f(p3, x, u).copy()
    v = x[4:7]
    f[4:7] -= u[-1] * cd / x[0] * np.linalg.norm(v) * v
    return f


def _flow(oracle, p3, cd, xk, uk, uk1, nsub):
    """RK4 over a unit tau interval with FOH controls (the caller divides s by N - 1)."""
    x = np.array(xk, np.float64)
    h = 1.0 / nsub
    for n in range(nsub):
        u = lambda lp: (1.0 - lp) * uk + lp * uk1
        l0, l1, l2 = n / nsub, (n + 0.5) / nsub, (n + 1) / nsub
        k1 = _f_drag(oracle, p3, cd, x, u(l0))
        k2 = _f_drag(oracle, p3, cd, x + 0.5 * h * k1, u(l1))
        k3 = _f_drag(oracle, p3, cd, x + 0.5 * h * k2, u(l1))
        k4 = _f_drag(oracle, p3, cd, x + h * k3, u(l2))
        x = x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return x


def _fk(oracle, p3, cd, N, xk, uk, uk1, nsub):
    uk = np.array(uk, np.float64); uk1 = np.array(uk1, np.float64)
    uk[-1] /= (N - 1); uk1[-1] /= (N - 1)
    return _flow(oracle, p3, cd, xk, uk, uk1, nsub)


def test_zero_drag_reproduces_the_builtin_3dof_library(drag_lib, oracle, inputs):
    """Three chained SCP steps with forced counts, then whole solves: the user
    library at c_D = 0 against libpdg_mc_3dof.so."""
    import torch
    from paper_2404_18034_gb300.pdg_mc import Solver
    p3 = inputs.load_params(model="3dof")
    SU = Solver(_params(inputs, 0.0), 15, library=drag_lib)
    SB = Solver(p3, 15)
    assert SU.nx == 8 and SU.model == "custom"
    B = 6
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x0 = inputs.dispersion(p3, B, 7, "bj")
    Ns = np.array([15, 10, 4, 15, 2, 12], np.int32)
    X = np.zeros((B, 15, 8)); U = np.zeros((B, 15, 4))
    for b in range(B):
        Xg, Ug = oracle.init_guess(p3, int(Ns[b]), x0[b])
        X[b, :Ns[b]] = Xg; U[b, :Ns[b]] = Ug
    shapes = {"xh": (15, 8), "uh": (15, 4), "mup": (14, 8), "mum": (14, 8), "phi": (14, 8), "th": (14,)}
    state = []
    for S in (SU, SB):
        ws = {k: torch.zeros(B, *s, dtype=torch.float64, device="cuda") for k, s in shapes.items()}
        gX, gU = d(X), d(U)
        for fp, fj in [(7, 45), (5, 120), (9, 33)]:
            S.scp_step(d(x0), gX, gU, ws, d(Ns), d(np.array([[fp, fj]] * B, np.int32)))
        torch.cuda.synchronize()
        state.append((gX.cpu().numpy(), gU.cpu().numpy(), {k: v.cpu().numpy() for k, v in ws.items()}))
    assert_scaled_close(state[0][0], state[1][0], p3["P_x"], what="X")
    assert_scaled_close(state[0][1], state[1][1], p3["P_u"][:4], what="U")
    for k in shapes:
        assert_scaled_close(state[0][2][k], state[1][2][k], 1.0, what=k)
    x0 = d(inputs.dispersion(p3, 64, 8, "bj"))
    a, b = SU.solve(x0, mode=1), SB.solve(x0, mode=1)
    torch.cuda.synchronize()
    same = (a["scp_iters"] == b["scp_iters"]) & (a["pipg_iters"] == b["pipg_iters"]) & (a["status"] == 0)
    assert same.float().mean().item() >= 0.9
    assert_scaled_close(a["X"][same].cpu().numpy(), b["X"][same].cpu().numpy(), p3["P_x"], what="solve X")
    SU.close(); SB.close()


def test_drag_blocks_match_the_reference_flow(drag_lib, oracle, inputs):
    """Discretization of the drag model (c_D = 0.3): x_prop and the blocks
    A_k, B^-_k, B^+_k from the library's STM integration against the RK4
    reference flow of this file and its central differences."""
    import torch
    from paper_2404_18034_gb300.pdg_mc import Solver
    cd, N = 0.3, 6
    p = _params(inputs, cd)
    p3 = inputs.load_params(model="3dof")
    S = Solver(p, N, library=drag_lib)
    x0 = inputs.dispersion(p3, 1, 12, "bj")
    rng = np.random.default_rng(12)
    X, U = oracle.init_guess(p3, N, x0[0])
    X[1:] += rng.normal(size=X[1:].shape) * 0.2 * p3["P_x"]
    U += rng.normal(size=U.shape) * 0.2 * p3["P_u"][:4]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    o = S.subproblem(d(x0), d(X[None]), d(U[None]))
    torch.cuda.synchronize()
    Px, Pu = p3["P_x"], p3["P_u"][:4]
    Am = o["Am"][0].cpu().numpy() * Px[None, :, None] / Px[None, None, :]   # A = P_x hat A P_x^-1
    Bm = o["Bm"][0].cpu().numpy() * Px[None, :, None] / Pu[None, None, :]
    Bp = o["Bp"][0].cpu().numpy() * Px[None, :, None] / Pu[None, None, :]
    w = o["w"][0].cpu().numpy() * Px[None, :]
    nsub, h = p3["rk4_substeps"], 1e-6
    for k in range(N - 1):
        xp = _fk(oracle, p3, cd, N, X[k], U[k], U[k + 1], nsub)
        np.testing.assert_allclose(w[k], xp - X[k + 1], rtol=1e-9, atol=1e-11)
        for j in range(8):
            e = np.zeros(8); e[j] = h
            fd = (_fk(oracle, p3, cd, N, X[k] + e, U[k], U[k + 1], nsub)
                  - _fk(oracle, p3, cd, N, X[k] - e, U[k], U[k + 1], nsub)) / (2 * h)
            np.testing.assert_allclose(Am[k][:, j], fd, atol=2e-7 * (1 + np.abs(fd).max()))
        for j in range(4):
            e = np.zeros(4); e[j] = h
            fdm = (_fk(oracle, p3, cd, N, X[k], U[k] + e, U[k + 1], nsub)
                   - _fk(oracle, p3, cd, N, X[k], U[k] - e, U[k + 1], nsub)) / (2 * h)
            fdp = (_fk(oracle, p3, cd, N, X[k], U[k], U[k + 1] + e, nsub)
                   - _fk(oracle, p3, cd, N, X[k], U[k], U[k + 1] - e, nsub)) / (2 * h)
            np.testing.assert_allclose(Bm[k][:, j], fdm, atol=2e-7 * (1 + np.abs(fdm).max()))
            np.testing.assert_allclose(Bp[k][:, j], fdp, atol=2e-7 * (1 + np.abs(fdp).max()))
    S.close()


def test_drag_solves_are_feasible(drag_lib, oracle, inputs):
    """Whole solves of the drag model: converged trajectories meet the
    boundary conditions and the drag dynamics on re-propagation by the
    reference flow, and their propellant differs from the drag-free
    landings of the same initial states."""
    import torch
    from paper_2404_18034_gb300.pdg_mc import Solver
    # drag slows the prox-linear creep (at c_D = 0.3, 3 of 16 instances
    # converged within 15 SCP iterations): a lighter drag and 30 iterations
    cd, N, B = 0.1, 15, 16
    p3 = inputs.load_params(model="3dof", scp_jmax=30)
    S = Solver(_params(inputs, cd, scp_jmax=30), N, library=drag_lib)
    S0 = Solver(p3, N)
    x0 = inputs.dispersion(p3, B, 5, "bj")
    out = S.solve(torch.from_numpy(x0).cuda(), mode=1)
    ref = S0.solve(torch.from_numpy(x0).cuda(), mode=1)
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    assert np.sum(st == 0) >= 4
    X, U = out["X"].cpu().numpy(), out["U"].cpu().numpy()
    fx = p3["fix_f"].astype(bool)
    for b in np.flatnonzero(st == 0)[:4]:
        np.testing.assert_allclose(X[b, 0, :7], x0[b], atol=1e-12)
        np.testing.assert_allclose(X[b, -1][fx], p3["z_f"][fx], atol=1e-9)
        for k in range(N - 1):
            xp = _fk(oracle, p3, cd, N, X[b, k], U[b, k], U[b, k + 1], 40)
            assert np.max(np.abs(xp - X[b, k + 1])[:7] / p3["P_x"][:7]) < 2e-3
    # c_D reaches the dynamics: the landings differ from the drag-free ones
    both = (st == 0) & (ref["status"].cpu().numpy() == 0)
    dfuel = np.abs(out["fuel"].cpu().numpy()[both] - ref["fuel"].cpu().numpy()[both])
    assert both.any() and dfuel.min() > 1e-4
    S.close(); S0.close()
