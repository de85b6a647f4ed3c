"""Parity of the 3-DoF instance of the problem template (libpdg_mc_3dof.so,
through the C ABI) with the FP64 oracle built for the same model.

Same protocol as the 6-DoF tests: element-wise at |a - b| <= 1e-6 max(|b|,
P scale) in FP64, iterative decisions replayed at the GPU's recorded counts."""
import numpy as np
import pytest

from gpu_helpers import (FP32_TOL, RTOL, assert_scaled_close, check_stop_decisions, fp32_errors,
                         replay_instance)

pytestmark = pytest.mark.gpu
NX3 = 8


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18034_gb300 import build
    build.build()
    return torch


def _solver(inputs, n_max=15, precision=0, form=0, **ov):
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params(model="3dof", **ov)
    S = Solver(p, n_max, precision)
    if form:
        S.set_pipg_form(form)
    return p, S


def _d(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_library_is_the_3dof_model(torch_cuda, inputs):
    p, S = _solver(inputs)
    assert S.lib.pdg_mc_model_nx() == NX3 and S.nx == NX3
    out = S.alloc_outputs(2)
    assert tuple(out["X"].shape) == (2, 15, NX3)
    S.close()


@pytest.mark.parametrize("gs", [0, 1])
def test_subproblem_blocks(torch_cuda, oracle, inputs, gs):
    """Discretization + prescaling of the 3-DoF model on uneven N (several
    discretization waves, a ragged last wave, N = 2), perturbed references
    so that every Jacobian slot is exercised."""
    torch = torch_cuda
    Ns = np.array([2, 3, 10, 15, 17, 30, 32, 9], np.int32)
    p, S = _solver(inputs, 32, glide_slope=gs)
    B, n_max = len(Ns), 32
    x0 = inputs.dispersion(p, B, 11, "bj")
    rng = np.random.default_rng(11)
    X = np.zeros((B, n_max, NX3)); U = np.zeros((B, n_max, 4))
    for b in range(B):
        Xg, Ug = oracle.init_guess(p, int(Ns[b]), x0[b])
        Xg[1:] += rng.normal(size=Xg[1:].shape) * 0.3 * p["P_x"]
        Ug += rng.normal(size=Ug.shape) * 0.3 * p["P_u"][:4]
        X[b, :Ns[b]] = Xg; U[b, :Ns[b]] = Ug
    o = S.subproblem(_d(torch, x0), _d(torch, X), _d(torch, U), _d(torch, Ns))
    torch.cuda.synchronize()
    for b, N in enumerate(Ns):
        A, Bm, Bp, xp = oracle.discretize(p, X[b, :N], U[b, :N])
        qp = oracle.scale(p, x0[b], X[b, :N], U[b, :N], A, Bm, Bp, xp)
        assert_scaled_close(o["Am"][b, :N - 1].cpu().numpy(), qp.Am, np.abs(qp.Am).max() * 1e-3, what=f"Am N={N}")
        assert_scaled_close(o["Bm"][b, :N - 1].cpu().numpy(), qp.Bm, np.abs(qp.Bm).max() * 1e-3, what=f"Bm N={N}")
        assert_scaled_close(o["Bp"][b, :N - 1].cpu().numpy(), qp.Bp, np.abs(qp.Bp).max() * 1e-3, what=f"Bp N={N}")
        assert_scaled_close(o["w"][b, :N - 1].cpu().numpy(), qp.w, 1e-3, what=f"w N={N}")
        assert np.all(o["Am"][b, N - 1:].cpu().numpy() == 0)
    S.close()


@pytest.mark.parametrize("form,soc", [(1, 0), (2, 0), (1, 1), (2, 1), (3, 0), (3, 1)])
def test_scp_step_forced_counts(torch_cuda, oracle, inputs, form, soc):
    """Three chained SCP iterations with the oracle's counts forced, PIPG in
    shared memory (form 1), in registers (form 2) and in register tiles over
    lane groups (form 3: four lanes per 8 x 8 block here), with and without
    the thrust-sector projection."""
    torch = torch_cuda
    Ns = np.array([15, 10, 4, 15, 2], np.int32)
    p, S = _solver(inputs, 15, form=form, soc_thrust=soc)
    B, n_max = len(Ns), 15
    x0 = inputs.dispersion(p, B, 5, "bj")
    X = np.zeros((B, n_max, NX3)); U = np.zeros((B, n_max, 4))
    ows = []
    for b in range(B):
        Xg, Ug = oracle.init_guess(p, int(Ns[b]), x0[b])
        X[b, :Ns[b]] = Xg; U[b, :Ns[b]] = Ug
        ows.append(oracle.PDState(int(Ns[b]), 4, "3dof"))
    oX = [X[b, :Ns[b]].copy() for b in range(B)]
    oU = [U[b, :Ns[b]].copy() for b in range(B)]
    gX, gU = _d(torch, X), _d(torch, U)
    shapes = {"xh": (n_max, NX3), "uh": (n_max, 4), "mup": (n_max - 1, NX3), "mum": (n_max - 1, NX3),
              "phi": (n_max - 1, NX3), "th": (n_max - 1,)}
    ws = {k: torch.zeros(B, *s, dtype=torch.float64, device="cuda") for k, s in shapes.items()}
    for it, (fp, fj) in enumerate([(7, 45), (5, 120), (9, 33)]):
        force = _d(torch, np.array([[fp, fj]] * B, np.int32))
        o = S.scp_step(_d(torch, x0), gX, gU, ws, _d(torch, Ns), force)
        torch.cuda.synchronize()
        for b in range(B):
            N = int(Ns[b])
            r = oracle.scp_iterate(p, x0[b], oX[b], oU[b], ows[b], force_pow=fp, force_pipg=fj)
            assert tuple(o["iters"][b].tolist()) == (fp, fj)
            assert abs(o["sigma"][b].item() - r["sigma"]) <= RTOL * r["sigma"]
            assert_scaled_close(gX[b, :N].cpu().numpy(), oX[b], p["P_x"], what=f"X it{it} b{b}")
            assert_scaled_close(gU[b, :N].cpu().numpy(), oU[b], p["P_u"][:4], what=f"U it{it} b{b}")
            for k in shapes:
                ref = getattr(ows[b], k)
                assert_scaled_close(ws[k][b].cpu().numpy()[:ref.shape[0]], ref, 1.0, what=f"{k} it{it} b{b}")
            assert abs(o["defect"][b].item() - r["defect"]) <= RTOL * max(r["defect"], 1.0)
            assert abs(o["step"][b].item() - r["step"]) <= RTOL * max(r["step"], 1.0)
    assert S.launch_info()["pipg_form"] == form
    S.close()


def _solve_and_replay(torch, oracle, p, S, x0, Ns, mode, sample, converged_only=False):
    out = S.solve(_d(torch, x0), _d(torch, Ns) if Ns is not None else None, mode=mode, trace=True)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    for b in sample:
        N = int(Ns[b]) if Ns is not None else S.n_max
        r = replay_instance(oracle, p, x0[b], N, o["trace"][b], int(o["scp_iters"][b]))
        assert o["status"][b] == r["status"], (b, o["status"][b], r["status"])
        if r["status"] == 2 or (converged_only and r["status"] != 0):
            continue
        if r["status"] == 0:
            check_stop_decisions(p, r, o["trace"][b], o["scp_iters"][b], o["status"][b], what=f"b{b}")
        assert_scaled_close(o["X"][b, :N], r["X"], p["P_x"], what=f"X b{b}")
        assert_scaled_close(o["U"][b, :N], r["U"], p["P_u"][:4], what=f"U b{b}")
        assert abs(o["tf"][b] - r["tf"]) <= RTOL * abs(r["tf"])
        assert abs(o["fuel"][b] - r["fuel"]) <= RTOL * max(abs(r["fuel"]), p["P_x"][0])
        assert np.all(o["X"][b, N:] == 0) and np.all(o["U"][b, N:] == 0)
    return o


@pytest.mark.parametrize("mode,form", [(1, 0), (0, 0), (2, 0), (1, 2), (0, 2), (1, 3), (0, 3), (2, 3)])
def test_full_solve_matches_oracle_replay(torch_cuda, oracle, inputs, mode, form):
    """Whole SCP solves on an uneven-N batch in every execution form and both
    PIPG layouts."""
    torch = torch_cuda
    p, S = _solver(inputs, 30, form=form)
    B = 12
    x0 = inputs.dispersion(p, B, inputs.config_seed(2), "bj")
    Ns = inputs.node_counts(B, inputs.config_seed(2))
    o = _solve_and_replay(torch, oracle, p, S, x0, Ns, mode, range(B))
    assert np.mean(o["status"] == 0) >= 0.75
    S.close()


@pytest.mark.parametrize("ov", [{"soc_thrust": 1}, {"glide_slope": 1, "dt_min": 0.3, "dt_max": 0.6}])
def test_variants_match_oracle_replay(torch_cuda, oracle, inputs, ov):
    """The thrust-sector projection and the glide-slope row with the time
    bounds on the 3-DoF model, whole solves against the replay."""
    torch = torch_cuda
    p, S = _solver(inputs, 15, **ov)
    B = 8
    x0 = inputs.dispersion(p, B, 31, "bj")
    Ns = np.full(B, 15, np.int32)
    o = _solve_and_replay(torch, oracle, p, S, x0, Ns, 1, range(B), converged_only=True)
    assert np.mean(o["status"] == 0) >= 0.75
    S.close()


def test_paper_distribution_sampled(torch_cuda, oracle, inputs):
    """The paper's r(0) distribution (Sec. 6) on the 3-DoF model: 256
    instances, statuses of all within the oracle's convergence share, values
    of a sample against the replay."""
    torch = torch_cuda
    p, S = _solver(inputs, 15)
    B = 256
    x0 = inputs.dispersion(p, B, inputs.config_seed(0), "paper256")
    o = _solve_and_replay(torch, oracle, p, S, x0, None, 1, range(0, B, 32), converged_only=True)
    assert np.mean(o["status"] == 0) >= 0.9
    S.close()


@pytest.mark.parametrize("form", [0, 3])
def test_fp32_tracks_fp64_oracle(torch_cuda, oracle, inputs, form):
    """FP32 (form 0: the automatic PIPG form) against the FP64 oracle's free
    runs: on the instances converged on both sides with equal SCP counts (at
    least 64 of 96), X, U, t_f and fuel within the FP32 tolerance."""
    torch = torch_cuda
    p, S32 = _solver(inputs, 15, precision=1, form=form)
    B = 96
    x0 = inputs.dispersion(p, B, 9, "bj")
    o = {k: v.cpu().numpy() for k, v in S32.solve(_d(torch, x0), mode=1).items()}
    ref = oracle.solve_batch(p, x0, np.full(B, 15, np.int32))
    both = np.nonzero((o["status"] == 0) & (ref["status"] == 0) & (o["scp_iters"] == ref["scp_iters"]))[0]
    e = fp32_errors(p, o, ref, both)
    print(f"3-DoF FP32: {len(both)} of {B} comparable; errors {e}")
    assert len(both) >= 64
    for k, v in e.items():
        assert v <= FP32_TOL, (k, v)
    S32.close()


def test_edge_cases_and_host_api(torch_cuda, inputs):
    """Empty batch; out-of-range node counts and non-finite x0 give
    PDG_BAD_INPUT with zero outputs; N = 2 runs; the host-buffer entry point
    returns what the device one does."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import PDG_BAD_INPUT
    p, S = _solver(inputs, 12)
    x0 = inputs.dispersion(p, 5, 1, "bj")
    x0[3, 2] = np.nan
    Ns = np.array([2, 1, 13, 12, 5], np.int32)
    assert S.solve(_d(torch, x0[:0]), mode=1)["X"].shape[0] == 0
    for mode in (0, 1, 2):
        out = S.solve(_d(torch, x0), _d(torch, Ns), mode=mode)
        torch.cuda.synchronize()
        st = out["status"].cpu().numpy()
        assert list(st[[1, 2, 3]]) == [PDG_BAD_INPUT] * 3
        assert st[0] in (0, 1) and st[4] in (0, 1)
        for b in (1, 2, 3):
            assert out["X"][b].abs().max().item() == 0.0 and out["tf"][b].item() == 0.0
    ok = inputs.dispersion(p, 6, 9, "bj")
    dev = S.solve(_d(torch, ok), mode=1)
    torch.cuda.synchronize()
    host = S.solve_host(ok, mode=1)
    for k in ("X", "U", "tf", "fuel", "status", "scp_iters", "pipg_iters"):
        np.testing.assert_array_equal(dev[k].cpu().numpy(), host[k])
    S.close()


def test_full_size_sampled(torch_cuda, oracle, inputs):
    """The 3-DoF benchmark workload (B = 16384, N = 15, FP64, persistent at the
    tuned launch shape): sampled instances by oracle replay, invariants on all."""
    torch = torch_cuda
    from paper_2404_18034_gb300.autotune import DEFAULT_CACHE
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params(model="3dof")
    S = Solver(p, 15, 0, tune_cache=DEFAULT_CACHE, mode=1)
    B = 16384
    x0 = inputs.dispersion(p, B, inputs.config_seed(2), "bj")
    out = S.solve(_d(torch, x0), mode=1, trace=True)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    hist = np.bincount(o["status"], minlength=5)
    assert hist[3:].sum() == 0 and hist[0] > 0.99 * B, hist
    ok = o["status"] != 2
    np.testing.assert_allclose(o["X"][ok, 0, :7], x0[ok], atol=1e-12)
    assert np.all(o["trace"][:, :, 1].sum(1) == o["pipg_iters"])
    rng = np.random.default_rng(1)
    conv = np.nonzero(o["status"] == 0)[0]
    for b in list(rng.choice(conv, 8, replace=False)) + [conv[0], conv[-1]]:
        r = replay_instance(oracle, p, x0[b], 15, o["trace"][b], int(o["scp_iters"][b]))
        assert o["status"][b] == r["status"], (b, o["status"][b], r["status"])
        check_stop_decisions(p, r, o["trace"][b], o["scp_iters"][b], o["status"][b], what=f"b{b}")
        assert_scaled_close(o["X"][b], r["X"], p["P_x"], what=f"X b{b}")
        assert abs(o["fuel"][b] - r["fuel"]) <= RTOL * max(abs(r["fuel"]), 0.5)
    S.close()

