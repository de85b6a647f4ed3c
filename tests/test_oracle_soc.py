"""Pins of the second-order-cone thrust variant (soc_thrust = 1): T_max and
the gimbal cone imposed by projection inside PIPG instead of CTCS rows."""
import math

import numpy as np
import pytest


def _in_sector(T, Tmax, tan_d, tol=1e-12):
    return np.linalg.norm(T) <= Tmax + tol and np.hypot(T[1], T[2]) <= tan_d * T[0] + tol


def test_sector_projection_is_the_euclidean_projection(oracle):
    """P(T) lies in the set, P is idempotent, and <T - P(T), Y - P(T)> <= 0 for
    every Y in the set (the variational inequality that characterizes the
    Euclidean projection onto a closed convex set)."""
    rng = np.random.default_rng(0)
    Tmax, d = 5.0, math.radians(20.0)
    a = math.tan(d)
    Ys = []
    while len(Ys) < 400:
        Y = rng.uniform(-6, 6, 3)
        if _in_sector(Y, Tmax, a):
            Ys.append(Y)
    Ys = np.array(Ys)
    for _ in range(300):
        T = rng.normal(size=3) * 4
        P = oracle.sector_project(T, Tmax, a)
        assert _in_sector(P, Tmax, a, 1e-9)
        np.testing.assert_allclose(oracle.sector_project(P, Tmax, a), P, atol=1e-12)
        assert np.max((Ys - P) @ (T - P)) <= 1e-9
        if _in_sector(T, Tmax, a):
            np.testing.assert_allclose(P, T, atol=0)


def test_sector_projection_matches_brute_force(oracle):
    scipy_opt = pytest.importorskip("scipy.optimize")
    Tmax, a = 5.0, math.tan(math.radians(20.0))
    rng = np.random.default_rng(1)
    cons = [{"type": "ineq", "fun": lambda y: Tmax ** 2 - y @ y},
            {"type": "ineq", "fun": lambda y: a * y[0] - math.hypot(y[1], y[2])}]
    for _ in range(12):
        T = rng.normal(size=3) * 5
        r = scipy_opt.minimize(lambda y: 0.5 * np.sum((y - T) ** 2), x0=np.array([1.0, 0.0, 0.0]),
                               constraints=cons, method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
        np.testing.assert_allclose(oracle.sector_project(T, Tmax, a), r.x, atol=1e-5)


def test_soc_pipgc_equals_alg1(oracle, inputs):
    p = inputs.load_params(soc_thrust=1)
    N, nu = 4, 4
    x0 = inputs.dispersion(p, 1, 5, "bj")[0]
    X, U = oracle.init_guess(p, N, x0)
    rng = np.random.default_rng(2)
    X[1:] += rng.normal(size=X[1:].shape) * 0.1 * p["P_x"]
    U += rng.normal(size=U.shape) * 0.1 * p["P_u"][:nu]
    A, Bm, Bp, xp = oracle.discretize(p, X, U)
    qp = oracle.scale(p, x0, X, U, A, Bm, Bp, xp)
    assert qp.soc == 1
    ws0 = oracle.PDState(N, nu)
    for k in ("xh", "uh", "mup", "mum", "phi", "th"):
        a = getattr(ws0, k)
        a[...] = np.abs(rng.normal(size=a.shape)) * 0.1
    sig, _ = oracle.power(p, qp, ws0)
    for J in (1, 9, 40):
        w1 = ws0.copy()
        oracle.pipgc(p, qp, sig, w1, force_iters=J)
        wp, om = p["w_prox"], p["pipg_omega"]
        alpha = 2.0 / (wp + np.sqrt(wp * wp + 4 * om * sig))
        z, w, v = oracle.pipg_generic(qp, alpha, om, p["pipg_rho"], J, oracle.z_pack(qp, ws0),
                                      ws0.phi.ravel().copy(), ws0.th.copy())
        np.testing.assert_allclose(oracle.z_pack(qp, w1), z, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w1.phi.ravel(), w, rtol=1e-12, atol=1e-12)


def test_soc_solution_keeps_thrust_in_the_sector(oracle, inputs):
    """Converged SOC solutions keep every node's thrust in the sector; FOH
    interpolation of points of a convex set stays in it between nodes."""
    p = inputs.load_params(soc_thrust=1)
    a = math.tan(p["delta_max"])
    x0 = inputs.dispersion(p, 3, 41, "bj")
    b = oracle.solve_batch(p, x0, np.full(3, 15, np.int32))
    assert np.all(b["status"] == 0)
    for i in range(3):
        for T in b["U"][i, :, :3]:
            assert _in_sector(T, p["T_max"], a, 1e-6)
        # the CTCS rows for T_max and the gimbal are off in this variant
        g = oracle.g(p, b["X"][i, 0], b["U"][i, 0])
        assert g[5] == -1.0 and g[6] == -1.0
