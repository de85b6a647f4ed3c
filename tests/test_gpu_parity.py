"""Parity of the CUDA solver (through the C ABI) with the FP64 CPU oracle.

Element-wise comparisons at the tolerance |a - b| <= 1e-6 max(|b|, P scale)
(FP64).  Iterative decisions (power-iteration, PIPG and SCP stop tests) are
replayed: the oracle runs the iteration counts the GPU recorded, so the two
compute the same algorithm step for step and differ only by rounding.  The
recorded counts are themselves checked: on the replayed iterates the oracle
evaluates its own stop tests wherever the GPU evaluated one, and each
decision must agree with the GPU's (check_stop_decisions)."""
import numpy as np
import pytest

from gpu_helpers import (FP32_TOL, RTOL, assert_scaled_close, check_stop_decisions, fp32_errors,
                         replay_instance)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18034_gb300 import build
    build.build()
    return torch


def _solver(inputs, nu=4, n_max=15, precision=0, form=0, **ov):
    """form: PIPG layout (0 automatic, 1 shared memory, 2 registers, 3 register
    tiles over lane groups)."""
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params(nu=nu, **ov)
    S = Solver(p, n_max, precision)
    if form:
        S.set_pipg_form(form)
    return p, S


def _refs(O, inputs, p, B, Ns, seed, perturb=0.03):
    """Reference trajectories: the initial guess perturbed (so that every
    Jacobian term is exercised), padded to n_max rows."""
    n_max = int(max(Ns))
    nu = p["nu"]
    x0 = inputs.dispersion(p, B, seed, "bj")
    rng = np.random.default_rng(seed)
    X = np.zeros((B, n_max, 15)); U = np.zeros((B, n_max, nu))
    for b in range(B):
        Xg, Ug = O.init_guess(p, int(Ns[b]), x0[b])
        Xg[1:] += rng.normal(size=Xg[1:].shape) * perturb * p["P_x"]
        Ug += rng.normal(size=Ug.shape) * perturb * p["P_u"][:nu]
        X[b, :Ns[b]] = Xg; U[b, :Ns[b]] = Ug
    return x0, X, U


@pytest.mark.parametrize("nu,prec", [(4, 0), (7, 0)])
def test_subproblem_blocks(torch_cuda, oracle, inputs, nu, prec):
    """Discretization + prescaling: hat A^-, hat B^-, hat B^+, hat w per
    interval, for a batch of uneven node counts (several waves of intervals
    and a ragged last wave)."""
    torch = torch_cuda
    Ns = np.array([2, 3, 10, 15, 17, 30, 32, 9], np.int32)
    p, S = _solver(inputs, nu, 32, prec)
    x0, X, U = _refs(oracle, inputs, p, len(Ns), Ns, 11)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    o = S.subproblem(d(x0), d(X), d(U), d(Ns))
    torch.cuda.synchronize()
    for b, N in enumerate(Ns):
        A, Bm, Bp, xp = oracle.discretize(p, X[b, :N], U[b, :N])
        qp = oracle.scale(p, x0[b], X[b, :N], U[b, :N], A, Bm, Bp, xp)
        sc_a = np.abs(qp.Am).max() * 1e-3
        assert_scaled_close(o["Am"][b, :N - 1].cpu().numpy(), qp.Am, sc_a, what=f"Am N={N}")
        assert_scaled_close(o["Bm"][b, :N - 1].cpu().numpy(), qp.Bm, np.abs(qp.Bm).max() * 1e-3, what=f"Bm N={N}")
        assert_scaled_close(o["Bp"][b, :N - 1].cpu().numpy(), qp.Bp, np.abs(qp.Bp).max() * 1e-3, what=f"Bp N={N}")
        assert_scaled_close(o["w"][b, :N - 1].cpu().numpy(), qp.w, 1e-3, what=f"w N={N}")
        assert np.all(o["Am"][b, N - 1:].cpu().numpy() == 0)


@pytest.mark.parametrize("nu,form", [(4, 1), (7, 1), (4, 2), (7, 2), (4, 3), (7, 3)])
def test_scp_step_forced_counts(torch_cuda, oracle, inputs, nu, form):
    """Three chained SCP iterations (discretize, scale, power iteration, PIPG
    with the oracle's counts forced, update) match the oracle's iterations,
    with the PIPG loop in shared memory (form 1), in registers (form 2) and in
    register tiles over lane groups (form 3)."""
    torch = torch_cuda
    Ns = np.array([15, 10, 4, 15], np.int32)
    p, S = _solver(inputs, nu, 15, form=form)
    B, n_max = len(Ns), 15
    x0 = inputs.dispersion(p, B, 5, "bj")
    X = np.zeros((B, n_max, 15)); U = np.zeros((B, n_max, nu))
    ows = []
    for b in range(B):
        Xg, Ug = oracle.init_guess(p, int(Ns[b]), x0[b])
        X[b, :Ns[b]] = Xg; U[b, :Ns[b]] = Ug
        ows.append(oracle.PDState(int(Ns[b]), nu))
    oX = [X[b, :Ns[b]].copy() for b in range(B)]
    oU = [U[b, :Ns[b]].copy() for b in range(B)]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gX, gU = d(X), d(U)
    ws = {k: torch.zeros(B, n_max if k in ("xh", "uh") else n_max - 1, *( (15,) if k in ("xh", "mup", "mum", "phi") else ((nu,) if k == "uh" else ())), dtype=torch.float64, device="cuda")
          for k in ("xh", "uh", "mup", "mum", "phi", "th")}
    for it, (fp, fj) in enumerate([(7, 45), (5, 120), (9, 33)]):
        force = d(np.array([[fp, fj]] * B, np.int32))
        o = S.scp_step(d(x0), gX, gU, ws, d(Ns), force)
        torch.cuda.synchronize()
        for b in range(B):
            N = int(Ns[b])
            r = oracle.scp_iterate(p, x0[b], oX[b], oU[b], ows[b], force_pow=fp, force_pipg=fj)
            assert tuple(o["iters"][b].tolist()) == (fp, fj)
            assert abs(o["sigma"][b].item() - r["sigma"]) <= RTOL * r["sigma"]
            assert_scaled_close(gX[b, :N].cpu().numpy(), oX[b], p["P_x"], what=f"X it{it} b{b}")
            assert_scaled_close(gU[b, :N].cpu().numpy(), oU[b], p["P_u"][:nu], what=f"U it{it} b{b}")
            for k in ("xh", "uh", "mup", "mum", "phi", "th"):
                g = ws[k][b].cpu().numpy()
                ref = getattr(ows[b], k)
                g = g[:ref.shape[0]]
                assert_scaled_close(g, ref, 1.0, what=f"{k} it{it} b{b}")
            assert abs(o["defect"][b].item() - r["defect"]) <= RTOL * max(r["defect"], 1.0)
            assert abs(o["step"][b].item() - r["step"]) <= RTOL * max(r["step"], 1.0)
    assert S.launch_info()["pipg_form"] == form


def _solve_and_replay(torch, oracle, inputs, p, S, x0, Ns, mode, sample, converged_only=False):
    """Solve on the GPU, replay each sampled instance in the oracle at the
    recorded counts and compare.  converged_only: compare values only where the
    solve converged (a run that does not converge is chaotic, so only its
    status and counts carry information)."""
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = S.solve(d(x0), d(Ns) if Ns is not None else None, mode=mode, trace=True)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    nu = p["nu"]
    decisions = [0, 0]
    for b in sample:
        N = int(Ns[b]) if Ns is not None else S.n_max
        r = replay_instance(oracle, p, x0[b], N, o["trace"][b], int(o["scp_iters"][b]))
        assert o["status"][b] == r["status"], (b, o["status"][b], r["status"])
        if r["status"] == 2 or (converged_only and r["status"] != 0):
            continue  # no values to compare: non-finite, or a chaotic non-converged run
        if r["status"] == 0:
            n, nb = check_stop_decisions(p, r, o["trace"][b], o["scp_iters"][b], o["status"][b], what=f"b{b}")
            decisions[0] += n; decisions[1] += nb
        assert_scaled_close(o["X"][b, :N], r["X"], p["P_x"], what=f"X b{b}")
        assert_scaled_close(o["U"][b, :N], r["U"], p["P_u"][:nu], what=f"U b{b}")
        assert abs(o["tf"][b] - r["tf"]) <= RTOL * abs(r["tf"])
        assert abs(o["fuel"][b] - r["fuel"]) <= RTOL * max(abs(r["fuel"]), p["P_x"][0])
        assert np.all(o["X"][b, N:] == 0) and np.all(o["U"][b, N:] == 0)
    print(f"stop decisions checked {decisions[0]}, borderline {decisions[1]}")
    assert decisions[1] <= 0.01 * max(decisions[0], 1)
    return o


@pytest.mark.parametrize("mode", [1, 0, 2])
def test_full_solve_matches_oracle_replay(torch_cuda, oracle, inputs, mode):
    """Whole SCP solves (persistent and plain form) on an uneven-N batch."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 30)
    B = 12
    x0 = inputs.dispersion(p, B, inputs.config_seed(2), "bj")
    Ns = inputs.node_counts(B, inputs.config_seed(2))
    o = _solve_and_replay(torch, oracle, inputs, p, S, x0, Ns, mode, range(B))
    assert np.mean(o["status"] == 0) >= 0.75  # the replayed sample above converges on both sides


@pytest.mark.parametrize("mode,form", [(1, 2), (0, 2), (2, 2), (1, 3), (0, 3), (2, 3)])
def test_register_form_matches_oracle_replay(torch_cuda, oracle, inputs, mode, form):
    """The register-resident PIPG forms in FP64, whole solves on an uneven
    batch (N in {10, 15, 20}; ragged rows and control lanes; form 3 also a
    half-used last warp at N = 15), every form of execution, against the
    oracle replay at the FP64 tolerance."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 20, form=form)
    B = 9
    x0 = inputs.dispersion(p, B, 21, "bj")
    Ns = np.array([10, 15, 20] * 3, np.int32)
    o = _solve_and_replay(torch, oracle, inputs, p, S, x0, Ns, mode, range(B))
    assert np.mean(o["status"] == 0) >= 0.75
    assert S.launch_info()["pipg_form"] == form


def test_pipg_form_selection(torch_cuda, inputs):
    """Automatic choice (register tiles for FP32, shared memory for FP64), the
    thread-count rules of the register forms, and rejected settings."""
    torch = torch_cuda
    p = inputs.load_params()
    from paper_2404_18034_gb300.pdg_mc import Solver
    x0 = torch.from_numpy(inputs.dispersion(p, 2, 3, "bj")).cuda()
    S64, S32 = Solver(p, 15, 0), Solver(p, 15, 1)
    S64.solve(x0, mode=1); S32.solve(x0, mode=1)
    torch.cuda.synchronize()
    assert S64.launch_info()["pipg_form"] == 1 and S32.launch_info()["pipg_form"] == 3
    assert S32.launch_info()["threads"] == 128  # 8 lanes per node: 120 -> 128 threads at N = 15
    S32.set_threads(96)             # below form 3's need: automatic falls back to form 1
    S32.solve(x0, mode=1)
    torch.cuda.synchronize()
    assert S32.launch_info()["pipg_form"] == 1
    S32.set_pipg_form(3)            # ... and an explicit request is refused
    with pytest.raises(RuntimeError, match="EINVAL"):
        S32.solve(x0, mode=1)
    S32.set_pipg_form(2)            # form 2 needs 224 + 64 threads
    S32.set_threads(256)
    with pytest.raises(RuntimeError, match="EINVAL"):
        S32.solve(x0, mode=1)
    S32.set_threads(0)
    S32.solve(x0, mode=1)
    torch.cuda.synchronize()
    assert S32.launch_info()["pipg_form"] == 2 and S32.launch_info()["threads"] == 288
    with pytest.raises(RuntimeError, match="EINVAL"):
        S64.set_pipg_form(4)
    S64.set_pipg_form(2)
    S64b = Solver(p, 30, 0)
    S64b.set_pipg_form(2)           # FP64 register form: at most 512 threads (N = 30 needs 576)
    with pytest.raises(RuntimeError, match="EINVAL"):
        S64b.solve(torch.from_numpy(inputs.dispersion(p, 1, 3, "bj")).cuda(), mode=1)
    S64b.set_pipg_form(3)           # form 3 at N = 30: 256 threads
    S64b.solve(torch.from_numpy(inputs.dispersion(p, 1, 3, "bj")).cuda(), mode=1)
    torch.cuda.synchronize()
    assert S64b.launch_info()["pipg_form"] == 3 and S64b.launch_info()["threads"] == 256


def test_fp32_register_form_tracks_shared_form(torch_cuda, oracle, inputs):
    """FP32: the register form against the shared-memory form and against
    FP64.  Both FP32 forms run the same iteration with different rounding, so
    they are compared at the FP32 level on instances converged in both."""
    torch = torch_cuda
    p, S2 = _solver(inputs, 4, 15, precision=1, form=2)
    _, S1 = _solver(inputs, 4, 15, precision=1, form=1)
    _, S64 = _solver(inputs, 4, 15)
    B = 32
    x0 = torch.from_numpy(inputs.dispersion(p, B, 17, "bj")).cuda()
    a, b, c = S2.solve(x0, mode=1), S1.solve(x0, mode=1), S64.solve(x0, mode=1)
    torch.cuda.synchronize()
    sa, sb, sc = (o["status"].cpu().numpy() for o in (a, b, c))
    assert np.mean(sa == 0) >= 0.8 and np.mean(sb == 0) >= 0.8
    both = np.nonzero((sa == 0) & (sb == 0) & (sc == 0))[0]
    assert len(both) >= B // 2
    for i in both:
        for o, what in ((b, "fp32 shared"), (c, "fp64")):
            assert_scaled_close(a["X"][i].cpu().numpy(), o["X"][i].cpu().numpy(), p["P_x"], rtol=2e-2,
                                what=f"fp32 registers vs {what} X {i}")
            assert abs(a["fuel"][i].item() - o["fuel"][i].item()) <= 2e-2 * p["P_x"][0]


def test_nu7_solve_matches_oracle_replay(torch_cuda, oracle, inputs):
    torch = torch_cuda
    p, S = _solver(inputs, 7, 15)
    x0 = inputs.dispersion(p, 4, 3, "bj")
    _solve_and_replay(torch, oracle, inputs, p, S, x0, None, 1, range(4))


@pytest.mark.parametrize("mode,form", [(1, 1), (0, 1), (1, 2), (2, 1), (1, 3), (0, 3)])
def test_pipg_stop_decisions_match_oracle(torch_cuda, oracle, inputs, mode, form):
    """PIPG tolerance 1e-4 at N = 10: most subproblems stop on Alg. stopping
    before the iteration cap (at the default 1e-6 nearly all run to the cap),
    so the PIPG stop decisions are exercised.  Whole solves in every
    execution form and every PIPG layout; every power, PIPG and SCP decision
    of the converged instances agrees with the oracle's own test on the
    replayed iterates, and at least 40 PIPG loops stopped on their test."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 10, form=form, pipg_eps_rel=1e-4, pipg_eps_abs=1e-8)
    B = 16
    x0 = inputs.dispersion(p, B, inputs.config_seed(1), "bj")
    o = _solve_and_replay(torch, oracle, inputs, p, S, x0, None, mode, range(B))
    conv = o["status"] == 0
    assert conv.mean() >= 0.9
    early = sum(int(np.sum(o["trace"][b, :o["scp_iters"][b], 1] < p["pipg_jmax"])) for b in np.nonzero(conv)[0])
    assert early >= 40, early


@pytest.mark.parametrize("eps_rel,form", [(1e-6, 0), (1e-4, 0), (1e-4, 3)])
def test_free_run_agrees_with_oracle(torch_cuda, oracle, inputs, eps_rel, form):
    """Without replay both sides take their own stop decisions.  With every
    decision equal (the stop-decision check above), the free runs must match
    count for count: every instance's status, SCP count and per-iteration
    power and PIPG counts, and the trajectories at the parity tolerance on the
    converged ones.  A decision may differ only where the oracle's own margin
    is borderline; such instances are counted and must be rare."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 10, form=form, pipg_eps_rel=eps_rel)
    B = 48
    x0 = inputs.dispersion(p, B, inputs.config_seed(1), "bj")
    out = S.solve(torch.from_numpy(x0).cuda(), mode=1, trace=True)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    differ = []
    for b in range(B):
        r = oracle.solve(p, 10, x0[b])
        J = int(o["scp_iters"][b])
        same = (o["status"][b] == r["status"] and J == r["scp_iters"]
                and np.array_equal(o["trace"][b, :J], r["trace"]))
        if not same:
            differ.append(b)
            continue
        assert r["pipg_iters"] == o["pipg_iters"][b]
        if r["status"] == 0:
            assert_scaled_close(o["X"][b], r["X"], p["P_x"], what=f"X b{b}")
            assert_scaled_close(o["U"][b], r["U"], p["P_u"][:4], what=f"U b{b}")
    # an instance whose counts differ must owe it to a borderline decision
    # (or to a run that never converges and wanders chaotically)
    for b in differ:
        r = replay_instance(oracle, p, x0[b], 10, o["trace"][b], int(o["scp_iters"][b]))
        if o["status"][b] == 0 and r["status"] == 0:
            n, nb = check_stop_decisions(p, r, o["trace"][b], o["scp_iters"][b], 0, what=f"free b{b}")
            assert nb >= 1, f"b{b}: counts differ although every decision agreed"
    print(f"free runs identical in every count: {B - len(differ)} of {B}")
    assert len(differ) <= B // 16


def test_single_instance_config(torch_cuda, oracle, inputs):
    """B = 1, N = 10, FP64, plain form: the single-instance workload."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 10)
    x0 = p["x0_nominal"][None, :].copy()
    _solve_and_replay(torch, oracle, inputs, p, S, x0, None, 0, [0])


def test_edge_cases(torch_cuda, inputs):
    """Empty batch; out-of-range node counts and non-finite x0 give
    PDG_BAD_INPUT with zero outputs; N = 2 runs."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import PDG_BAD_INPUT
    p, S = _solver(inputs, 4, 12)
    x0 = inputs.dispersion(p, 5, 1, "bj")
    x0[3, 2] = np.nan
    Ns = np.array([2, 1, 13, 12, 5], np.int32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    empty = S.solve(d(x0[:0]), mode=1)
    assert empty["X"].shape[0] == 0
    for mode in (0, 1):
        out = S.solve(d(x0), d(Ns), mode=mode)
        torch.cuda.synchronize()
        st = out["status"].cpu().numpy()
        assert list(st[[1, 2, 3]]) == [PDG_BAD_INPUT] * 3
        assert st[0] in (0, 1) and st[4] in (0, 1)
        for b in (1, 2, 3):
            assert out["X"][b].abs().max().item() == 0.0 and out["tf"][b].item() == 0.0


def test_host_api_equals_device_api(torch_cuda, inputs):
    """The host-buffer entry point returns what the device one does.  The
    handle's workspaces grow in turn (shape-class streams, host staging,
    gradient workspace) and each growth must leave the others intact: the
    solves and the gradient afterwards still agree and close() succeeds."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 15)
    x0 = inputs.dispersion(p, 6, 9, "bj")
    d0 = torch.from_numpy(x0).cuda()
    classed = S.solve(d0, mode=2)
    dev = S.solve(d0, mode=1)
    torch.cuda.synchronize()
    host = S.solve_host(x0, mode=1)
    for k in ("X", "U", "tf", "fuel", "status", "scp_iters", "pipg_iters"):
        np.testing.assert_array_equal(dev[k].cpu().numpy(), host[k])
    g = S.grad(d0)
    again = S.solve(d0, mode=2)
    host2 = S.solve_host(x0, mode=0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(again["status"].cpu().numpy(), classed["status"].cpu().numpy())
    np.testing.assert_array_equal(host2["status"], host["status"])
    assert np.all(np.isfinite(g["grad"].cpu().numpy()[g["status"].cpu().numpy() <= 1]))
    S.close()


def test_plain_and_persistent_agree(torch_cuda, inputs):
    """Plain, persistent and shape-class forms on the same uneven batch."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 20)
    x0 = inputs.dispersion(p, 8, 4, "bj")
    Ns = np.array([20, 15, 10, 20, 15, 10, 20, 2], np.int32)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a = S.solve(d(x0), d(Ns), mode=0)
    b = S.solve(d(x0), d(Ns), mode=1)
    torch.cuda.synchronize()
    # the two forms run the same phase code compiled into different kernels,
    # so the compiler may order a few floating-point operations differently:
    # same statuses, values within the parity tolerance
    np.testing.assert_array_equal(a["status"].cpu().numpy(), b["status"].cpu().numpy())
    for i in np.nonzero(b["status"].cpu().numpy() == 0)[0]:
        assert_scaled_close(a["X"][i].cpu().numpy(), b["X"][i].cpu().numpy(), p["P_x"], what=f"plain X {i}")
        assert_scaled_close(a["U"][i].cpu().numpy(), b["U"][i].cpu().numpy(), p["P_u"][:4], what=f"plain U {i}")
    # shape classes run each node count with its own CTA size, so block sums
    # may round differently: same status, values within the parity tolerance
    c = S.solve(d(x0), d(Ns), mode=2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(c["status"].cpu().numpy(), b["status"].cpu().numpy())
    for i in np.nonzero(b["status"].cpu().numpy() == 0)[0]:
        assert_scaled_close(c["X"][i].cpu().numpy(), b["X"][i].cpu().numpy(), p["P_x"], what=f"classed X {i}")
        assert_scaled_close(c["U"][i].cpu().numpy(), b["U"][i].cpu().numpy(), p["P_u"][:4], what=f"classed U {i}")


@pytest.mark.parametrize("N,prec,form", [(15, 1, 0), (30, 1, 0), (15, 1, 3), (30, 1, 3)])
def test_fp32_build_tracks_fp64_oracle(torch_cuda, oracle, inputs, N, prec, form):
    """The FP32 build against the FP64 oracle's free runs: on the instances
    that converge on both sides in the same number of SCP iterations (at
    least 64 of 96), the scaled X and U errors and the relative t_f and fuel
    errors are within the FP32 tolerance.  Form 0 is the automatic choice."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, N, precision=prec, form=form)
    B = 96
    x0 = inputs.dispersion(p, B, inputs.config_seed(3 if N == 15 else 5), "bj")
    out = S.solve(torch.from_numpy(x0).cuda(), mode=1)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.solve_batch(p, x0, np.full(B, N, np.int32))
    both = np.nonzero((o["status"] == 0) & (ref["status"] == 0) & (o["scp_iters"] == ref["scp_iters"]))[0]
    e = fp32_errors(p, o, ref, both)
    print(f"FP32 N={N} form {form}: {len(both)} of {B} comparable; errors {e}; converged FP32 {np.mean(o['status'] == 0):.3f}")
    assert len(both) >= 64
    for k, v in e.items():
        assert v <= FP32_TOL, (k, v)


def test_full_size_sampled(torch_cuda, oracle, inputs):
    """The benchmark workload (B = 16384, N = 15, FP64, persistent) checked
    on sampled instances by oracle replay, plus invariants on all."""
    torch = torch_cuda
    p, S = _solver(inputs, 4, 15)
    B = 16384
    x0 = inputs.dispersion(p, B, inputs.config_seed(2), "bj")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = S.solve(d(x0), mode=1, trace=True)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    hist = np.bincount(o["status"], minlength=5)
    assert hist[3:].sum() == 0, hist
    assert hist[0] > 0.9 * B and hist[2] < 0.01 * B, hist
    ok = o["status"] != 2
    np.testing.assert_allclose(o["X"][ok, 0, :14], x0[ok], atol=1e-12)
    assert np.all(o["trace"][:, :, 1].sum(1) == o["pipg_iters"])
    # Values are compared on converged instances: a run that does not converge
    # wanders chaotically (the oracle itself maps a 1e-13 relative change of x0
    # to O(1) changes of X there), so only its status is meaningful.
    rng = np.random.default_rng(0)
    conv = np.nonzero(o["status"] == 0)[0]
    sample = list(rng.choice(conv, 8, replace=False)) + [conv[0], conv[-1]]
    for b in sample:
        r = replay_instance(oracle, p, x0[b], 15, o["trace"][b], int(o["scp_iters"][b]))
        assert o["status"][b] == r["status"], (b, o["status"][b], r["status"])
        check_stop_decisions(p, r, o["trace"][b], o["scp_iters"][b], o["status"][b], what=f"b{b}")
        assert_scaled_close(o["X"][b], r["X"], p["P_x"], what=f"X b{b}")
        assert abs(o["fuel"][b] - r["fuel"]) <= RTOL * max(abs(r["fuel"]), 0.5)


def test_fp32_error_report_n30(torch_cuda, oracle, inputs):
    """N = 30 in FP32 against FP64 on the GPU: the same FP32 tolerance as
    against the oracle, on instances converged in both with equal SCP counts."""
    torch = torch_cuda
    p = inputs.load_params()
    from paper_2404_18034_gb300.pdg_mc import Solver
    S64, S32 = Solver(p, 30, 0), Solver(p, 30, 1)
    B = 64
    x0 = inputs.dispersion(p, B, inputs.config_seed(5), "bj")
    d = torch.from_numpy(x0).cuda()
    a = {k: v.cpu().numpy() for k, v in S64.solve(d, mode=1).items()}
    b = {k: v.cpu().numpy() for k, v in S32.solve(d, mode=1).items()}
    both = np.nonzero((a["status"] == 0) & (b["status"] == 0) & (a["scp_iters"] == b["scp_iters"]))[0]
    e = fp32_errors(p, b, a, both)
    print(f"FP32 vs FP64 (GPU), N = 30: {len(both)} of {B} comparable; errors {e}")
    assert len(both) >= B // 2
    for k, v in e.items():
        assert v <= FP32_TOL, (k, v)


def test_paper_model_paper256_distribution(torch_cuda, oracle, inputs):
    """The paper's model (nu = 7, RCS torque) on the Monte Carlo of Sec. 6
    (tests/golden/paper_sec6_monte_carlo.json: 256 runs, SCP <= 25, PIPG
    2500, all converge in the paper): the runs converge and sampled ones
    match the oracle replay."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_sec6_monte_carlo.json")) as fh:
        mc = json.load(fh)
    torch = torch_cuda
    p = inputs.load_params(nu=7, scp_jmax=mc["scp_iteration_limit"], pipg_jmax=mc["pipg_iterations_per_subproblem"])
    from paper_2404_18034_gb300.pdg_mc import Solver
    S = Solver(p, 15)
    n = mc["runs"]
    x0 = inputs.dispersion(p, n, inputs.config_seed(99), "paper256")
    o = _solve_and_replay(torch, oracle, inputs, p, S, x0, None, 2, range(0, n, 32), converged_only=True)
    assert np.mean(o["status"] == 0) >= 0.95
    assert o["scp_iters"].max() <= mc["scp_iteration_limit"]


def test_budget_status(torch_cuda, inputs):
    """A device-side wall-clock budget of ~0 stops every instance with
    PDG_BUDGET instead of running on (the persistent kernel checks the
    global timer before each SCP iteration)."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import PDG_BUDGET, Solver
    p = inputs.load_params()
    S = Solver(p, 10, 0, budget_seconds=1e-9)
    out = S.solve(torch.from_numpy(inputs.dispersion(p, 4, 1, "bj")).cuda(), mode=1)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == PDG_BUDGET)


@pytest.mark.parametrize("nu,form", [(4, 1), (7, 1), (4, 2), (4, 3), (7, 3)])
def test_soc_variant_matches_oracle(torch_cuda, oracle, inputs, nu, form):
    """soc_thrust = 1 (thrust sector by projection inside PIPG): chained SCP
    steps with forced counts and full solves match the oracle replay."""
    torch = torch_cuda
    p, S = _solver(inputs, nu, 15, form=form, soc_thrust=1)
    B, n_max = 3, 15
    x0 = inputs.dispersion(p, B, 12, "bj")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X = np.zeros((B, n_max, 15)); U = np.zeros((B, n_max, nu))
    ows, oX, oU = [], [], []
    for b in range(B):
        Xg, Ug = oracle.init_guess(p, n_max, x0[b])
        X[b] = Xg; U[b] = Ug
        ows.append(oracle.PDState(n_max, nu)); oX.append(Xg.copy()); oU.append(Ug.copy())
    gX, gU = d(X), d(U)
    shapes = {"xh": (n_max, 15), "uh": (n_max, nu), "mup": (n_max - 1, 15), "mum": (n_max - 1, 15),
              "phi": (n_max - 1, 15), "th": (n_max - 1,)}
    ws = {k: torch.zeros(B, *s, dtype=torch.float64, device="cuda") for k, s in shapes.items()}
    for fp, fj in [(6, 300), (4, 150)]:
        S.scp_step(d(x0), gX, gU, ws, None, d(np.array([[fp, fj]] * B, np.int32)))
        torch.cuda.synchronize()
        for b in range(B):
            oracle.scp_iterate(p, x0[b], oX[b], oU[b], ows[b], force_pow=fp, force_pipg=fj)
            assert_scaled_close(gX[b].cpu().numpy(), oX[b], p["P_x"], what=f"soc X b{b}")
            assert_scaled_close(gU[b].cpu().numpy(), oU[b], p["P_u"][:nu], what=f"soc U b{b}")
    x0 = inputs.dispersion(p, 6, 13, "bj")
    o = _solve_and_replay(torch, oracle, inputs, p, S, x0, None, 1, range(6))
    assert np.mean(o["status"] == 0) >= 0.8
    a = np.tan(p["delta_max"])
    for b in np.nonzero(o["status"] == 0)[0]:
        T = o["U"][b, :, :3]
        assert np.all(np.linalg.norm(T, axis=1) <= p["T_max"] + 1e-6)
        assert np.all(np.hypot(T[:, 1], T[:, 2]) <= a * T[:, 0] + 1e-6)


@pytest.mark.parametrize("nu", [4, 7])
def test_subproblem_blocks_with_glide_slope(torch_cuda, oracle, inputs, nu):
    """Discretization with the glide-slope row active on most nodes (the
    reference flown low, outside the cone): scaled blocks against the oracle."""
    torch = torch_cuda
    Ns = np.array([12, 15, 3], np.int32)
    p, S = _solver(inputs, nu, 15, glide_slope=1)
    x0, X, U = _refs(oracle, inputs, p, len(Ns), Ns, 41)
    X[:, 1:, 1] *= 0.25
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    o = S.subproblem(d(x0), d(X), d(U), d(Ns))
    torch.cuda.synchronize()
    active = 0
    for b, N in enumerate(Ns):
        active += sum(oracle.g(p, X[b, k], U[b, k])[-1] > 0 for k in range(N))
        A, Bm, Bp, xp = oracle.discretize(p, X[b, :N], U[b, :N])
        qp = oracle.scale(p, x0[b], X[b, :N], U[b, :N], A, Bm, Bp, xp)
        assert_scaled_close(o["Am"][b, :N - 1].cpu().numpy(), qp.Am, np.abs(qp.Am).max() * 1e-3, what=f"Am N={N}")
        assert_scaled_close(o["Bm"][b, :N - 1].cpu().numpy(), qp.Bm, np.abs(qp.Bm).max() * 1e-3, what=f"Bm N={N}")
        assert_scaled_close(o["Bp"][b, :N - 1].cpu().numpy(), qp.Bp, np.abs(qp.Bp).max() * 1e-3, what=f"Bp N={N}")
        assert_scaled_close(o["w"][b, :N - 1].cpu().numpy(), qp.w, 1e-3, what=f"w N={N}")
    assert active >= 10


@pytest.mark.parametrize("form", [1, 2, 3])
def test_glide_slope_and_time_bounds_match_oracle(torch_cuda, oracle, inputs, form):
    """Glide-slope row and the time-bound box: chained SCP steps with forced
    counts, then full solves against the oracle replay, in every PIPG form."""
    torch = torch_cuda
    ov = dict(glide_slope=1, dt_min=0.3, dt_max=0.5, tf_max=6.6)
    p, S = _solver(inputs, 4, 15, form=form, **ov)
    B, n_max, nu = 3, 15, 4
    x0 = inputs.dispersion(p, B, 12, "bj")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    X = np.zeros((B, n_max, 15)); U = np.zeros((B, n_max, nu))
    ows, oX, oU = [], [], []
    for b in range(B):
        Xg, Ug = oracle.init_guess(p, n_max, x0[b])
        X[b] = Xg; U[b] = Ug
        ows.append(oracle.PDState(n_max, nu)); oX.append(Xg.copy()); oU.append(Ug.copy())
    gX, gU = d(X), d(U)
    shapes = {"xh": (n_max, 15), "uh": (n_max, nu), "mup": (n_max - 1, 15), "mum": (n_max - 1, 15),
              "phi": (n_max - 1, 15), "th": (n_max - 1,)}
    ws = {k: torch.zeros(B, *s, dtype=torch.float64, device="cuda") for k, s in shapes.items()}
    for fp, fj in [(6, 300), (4, 150)]:
        S.scp_step(d(x0), gX, gU, ws, None, d(np.array([[fp, fj]] * B, np.int32)))
        torch.cuda.synchronize()
        for b in range(B):
            oracle.scp_iterate(p, x0[b], oX[b], oU[b], ows[b], force_pow=fp, force_pipg=fj)
            assert_scaled_close(gX[b].cpu().numpy(), oX[b], p["P_x"], what=f"X b{b}")
            assert_scaled_close(gU[b].cpu().numpy(), oU[b], p["P_u"][:nu], what=f"U b{b}")
    x0 = inputs.dispersion(p, 8, 31, "bj")
    o = _solve_and_replay(torch, oracle, inputs, p, S, x0, None, 1, range(8), converged_only=True)
    ok = np.nonzero(o["status"] == 0)[0]
    assert len(ok) >= 3
    for b in ok:
        s = o["U"][b, :, -1]
        dt = (s[:-1] + s[1:]) / (2 * (n_max - 1))
        assert dt.min() >= 0.3 - 1e-9 and dt.max() <= 0.5 + 1e-9 and o["tf"][b] <= 6.6 + 1e-9


@pytest.mark.parametrize("model", ["6dof", "3dof"])
def test_maximum_node_count_matches_oracle_replay(torch_cuda, oracle, inputs, model):
    """N = 32, the largest node count the kernels are built for (the 6-DoF
    image then takes one CTA per SM), whole solves against the replay."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params(model=model)
    S = Solver(p, 32)
    x0 = inputs.dispersion(p, 4, 77, "bj")
    o = _solve_and_replay(torch, oracle, inputs, p, S, x0, np.full(4, 32, np.int32), 1, range(4), converged_only=True)
    assert np.all(o["status"] <= 1)
    S.close()

