"""Pins of the oracle's full SCP solve (Sec. 2.3, Sec. 6): a converged
trajectory satisfies the nonlinear dynamics on re-propagation, the CTCS
budget and the path constraints between nodes; replaying recorded counts
reproduces a solve; the paper's Monte Carlo distribution converges."""
import numpy as np
import pytest


def _fine_defects(O, p, X, U, nsub=200):
    N = X.shape[0]
    out = []
    for k in range(N - 1):
        uk, uk1 = U[k].copy(), U[k + 1].copy()
        uk[-1] /= (N - 1); uk1[-1] /= (N - 1)
        out.append(np.abs(O.flow(p, X[k], uk, uk1, nsub) - X[k + 1]) / p["P_x"])
    return np.array(out)


def _dense_g(O, p, X, U, nsamp=40, integral=False):
    """g at nsamp + 1 points of every interval along the flow from each node
    (FOH controls).  integral=True also returns, per interval, the flow's
    change of the CTCS state y and the trapezoid sum of its integrand
    s sum_i max(0, g_i)^2 over the same points."""
    N, nu = U.shape
    gs, ys = [], []
    for k in range(N - 1):
        x = X[k].copy()
        uk, uk1 = U[k].copy(), U[k + 1].copy()
        vals = []
        for i in range(nsamp + 1):
            lp = i / nsamp
            u = (1 - lp) * U[k] + lp * U[k + 1]
            gi = O.g(p, x, u)
            if i < nsamp:
                gs.append(gi)
            vals.append(u[-1] * np.sum(np.maximum(gi, 0.0) ** 2))
            if i == nsamp:
                break
            a = uk * (1 - lp) + uk1 * lp
            b = uk * (1 - lp - 1 / nsamp) + uk1 * (lp + 1 / nsamp)
            a[-1] /= (N - 1) * nsamp; b[-1] /= (N - 1) * nsamp
            x = O.flow(p, x, a, b, 20)
        h = 1.0 / ((N - 1) * nsamp)
        ys.append((x[-1] - X[k, -1], h * (np.sum(vals) - 0.5 * (vals[0] + vals[-1]))))
    return (np.array(gs), np.array(ys)) if integral else np.array(gs)


@pytest.mark.parametrize("nu,seed", [(4, 21), (4, 23), (7, 21)])
def test_converged_solution_is_feasible(oracle, inputs, nu, seed):
    """At convergence (reading R8) the trajectory meets, in continuous time:
    - the dynamics: the scaled defect against a 200-substep flow is within the
      solver's own defect tolerance scp_eps_defect (the 10-substep RK4 the
      solver uses differs from the fine flow by far less);
    - the unit quaternion: the flow preserves ||q|| (Omega(w) is skew, Sec. 4),
      so ||q_k|| - 1 can only come from the defects of the nodes before k;
    - the CTCS budget: y_N - y_1 <= (N - 1) eps, and the flow's y agrees with
      a trapezoid sum of s sum_i max(0, g_i)^2 at 41 points per interval (so
      the integrator state integrates the path constraints, Eq.
      sys-dyn-dil-aug); the solve's own y_N - y_1 is that integral to 10 %;
    - non-increasing mass, the boundary conditions and the dilation box."""
    p = inputs.load_params(nu=nu)
    N = 15
    x0 = inputs.dispersion(p, 1, seed, "bj")[0]
    r = oracle.solve(p, N, x0)
    assert r["status"] == 0, r
    X, U = r["X"], r["U"]
    assert r["defect"] <= p["scp_eps_defect"] and r["step"] <= p["scp_eps_step"]
    np.testing.assert_allclose(X[0, :14], x0, atol=1e-12)
    assert X[0, 14] == 0.0
    fx = p["fix_f"].astype(bool)
    np.testing.assert_allclose(X[-1][fx], p["z_f"][fx], atol=1e-9)
    d = _fine_defects(oracle, p, X, U)
    assert d[:, :14].max() <= p["scp_eps_defect"], d.max()
    dq = np.concatenate([[0.0], np.cumsum(np.linalg.norm(d[:, 7:11] * p["P_x"][7:11], axis=1))])
    assert np.all(np.abs(np.linalg.norm(X[:, 7:11], axis=1) - 1.0) <= dq + 1e-12)
    assert np.all(np.diff(X[:, 0]) <= 0.0)
    g, ys = _dense_g(oracle, p, X, U, integral=True)
    budget = (N - 1) * p["eps_ctcs"]
    assert X[-1, 14] - X[0, 14] <= budget + 1e-12
    flow_dy, quad = ys[:, 0].sum(), ys[:, 1].sum()
    assert abs(flow_dy - quad) <= 0.1 * quad + 1e-10, (flow_dy, quad)
    assert abs((X[-1, 14] - X[0, 14]) - flow_dy) <= 0.1 * flow_dy + 1e-10
    assert np.maximum(g, 0).max() < 0.05
    assert np.all(U[:, -1] >= p["s_min"] - 1e-9) and np.all(U[:, -1] <= p["s_max"] + 1e-9)
    tf = np.sum(0.5 * (U[:-1, -1] + U[1:, -1])) / (N - 1)
    assert abs(tf - r["tf"]) < 1e-12
    assert abs((X[0, 0] - X[-1, 0]) - r["fuel"]) < 1e-12


def test_replay_reproduces_free_run(oracle, params):
    x0 = params["x0_nominal"]
    r = oracle.solve(params, 10, x0)
    rr = oracle.solve(params, 10, x0, trace=r["trace"], replay_scp=r["scp_iters"])
    np.testing.assert_array_equal(r["X"], rr["X"])
    np.testing.assert_array_equal(r["U"], rr["U"])
    assert r["status"] == rr["status"]


def test_batch_matches_single(oracle, inputs, params):
    x0 = inputs.dispersion(params, 6, 31, "bj")
    Ns = np.array([10, 15, 10, 20, 15, 10], np.int32)
    b = oracle.solve_batch(params, x0, Ns, nthreads=3)
    for i in range(6):
        r = oracle.solve(params, int(Ns[i]), x0[i])
        np.testing.assert_array_equal(b["X"][i, :Ns[i]], r["X"])
        assert b["status"][i] == r["status"] and b["scp_iters"][i] == r["scp_iters"]
        assert b["pipg_iters"][i] == r["pipg_iters"]


def _paper_mc():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_sec6_monte_carlo.json")) as fh:
        return json.load(fh)


def test_paper_monte_carlo_distribution_converges(oracle, inputs):
    """Sec. 6 (tests/golden/paper_sec6_monte_carlo.json): r(0) ~ (U(6,9),
    U(3,6), U(1,2)), SCP <= 25, 2500 PIPG iterations: 256 of 256 runs
    converge (on this project's parameter set)."""
    mc = _paper_mc()
    p = inputs.load_params(scp_jmax=mc["scp_iteration_limit"], pipg_jmax=mc["pipg_iterations_per_subproblem"])
    n = mc["runs"]
    x0 = inputs.dispersion(p, n, inputs.config_seed(99), "paper256")
    for c, (lo, hi) in enumerate(mc["initial_position_bounds"]):
        assert np.all((x0[:, 1 + c] >= lo) & (x0[:, 1 + c] <= hi))
    b = oracle.solve_batch(p, x0, np.full(n, 15, np.int32))
    assert int(np.sum(b["status"] == 0)) == mc["runs_converged"], np.bincount(b["status"])
    assert b["scp_iters"].max() <= mc["scp_iteration_limit"]


def _pack(X, U, ws):
    return np.concatenate([X[1:].ravel(), U.ravel(), ws.xh.ravel(), ws.uh.ravel(), ws.mup.ravel(), ws.mum.ravel(),
                           ws.phi.ravel(), ws.th.ravel()])


def _scp_map(O, p, x0, z, X, U, ws, sig, n):
    """One SCP iteration (sigma and the PIPG count held) as a map of the
    reference and the warm start, packed as a vector."""
    X, U, w = X.copy(), U.copy(), ws.copy()
    o = 0
    for arr in (X[1:], U, w.xh, w.uh, w.mup, w.mum, w.phi, w.th):
        arr[...] = z[o:o + arr.size].reshape(arr.shape)
        o += arr.size
    O.scp_iterate(p, x0, X, U, w, force_pow=1, force_pipg=n, force_sigma=sig)
    return _pack(X, U, w)


@pytest.mark.parametrize("model,N", [("3dof", 10), ("6dof", 8)])
def test_scp_map_is_not_contractive_at_convergence(oracle, inputs, model, N):
    """The total derivative of the converged outputs through the SCP fixed
    point, lambda = dl/dZ + J_Z^T lambda by sweeps, needs the spectral radius
    of the SCP map's Jacobian J_Z below one.  At the last iterate of converged
    solves it is not: central differences of the map (reference and warm
    start, sigma and the PIPG count held) give rho(J_Z) >= 1, so the sweeps
    diverge and the exported gradient is that of the last SCP iteration."""
    p = inputs.load_params(model=model)
    x0 = inputs.dispersion(p, 1, 3, "bj")[0]
    r = oracle.solve(p, N, x0)
    assert r["status"] == 0
    X, U, ws, sig, n = oracle.final_iteration_state(p, N, x0, r["trace"], r["scp_iters"])
    z0 = _pack(X, U, ws)
    nx = len(p["P_x"])
    scale = np.concatenate([np.tile(p["P_x"], N - 1), np.tile(p["P_u"][:p["nu"]], N),
                            np.ones(z0.size - (N - 1) * nx - N * p["nu"])])
    J = np.zeros((z0.size, z0.size))
    for j in range(z0.size):
        e = np.zeros(z0.size)
        e[j] = 1e-6 * scale[j]
        J[:, j] = (_scp_map(oracle, p, x0, z0 + e, X, U, ws, sig, n)
                   - _scp_map(oracle, p, x0, z0 - e, X, U, ws, sig, n)) / (2 * e[j])
    rho = np.abs(np.linalg.eigvals(J * scale[None, :] / scale[:, None])).max()
    assert rho >= 0.99, rho


def test_scp_creeps_at_tight_tolerance(oracle, inputs):
    """The total derivative through the SCP fixed point would need solves
    converged to that fixed point, e.g. to check it against differences of
    whole solves.  At a step tolerance of 1e-8 (PIPG converged to 1e-10 in
    every subproblem) the prox-linear iteration with its fixed prox weight
    does not get there: after 300 SCP iterations its scaled step is still
    above 1e-4, creeping down far slower than linearly."""
    p = inputs.load_params(model="3dof", scp_eps_step=1e-8, scp_eps_defect=1e-10, scp_jmax=300,
                           pipg_eps_rel=1e-10, pipg_eps_abs=1e-13, pipg_jmax=20000)
    x0 = inputs.dispersion(p, 1, 3, "bj")[0]
    r = oracle.solve(p, 10, x0)
    assert r["status"] == 1 and r["scp_iters"] == 300
    assert r["step"] > 1e-4 and r["defect"] < 1e-6
