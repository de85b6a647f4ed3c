"""Pins of the oracle's glide-slope row and time-bound box (Sec. 2.2 time
bounds; the glide-slope bound gamma_gs named in Sec. 4), against their
definitions, finite differences and the converged solutions."""
import math

import numpy as np
import pytest

from conftest import rand_control, rand_state


@pytest.mark.parametrize("nu", [4, 7])
def test_glide_slope_row_on_the_cone(oracle, inputs, nu):
    """The row is zero on the cone tan(gamma_gs) ||(r_y, r_z)|| = r_x, negative
    inside (steeper), positive outside; it is the last row of g."""
    p = inputs.load_params(nu=nu, glide_slope=1)
    tg = math.tan(p["gamma_gs"])
    x = np.zeros(15); x[0] = 1.5; x[7] = 1.0
    u = np.zeros(nu); u[0] = 2.0; u[-1] = 1.0
    n_off = oracle.g(inputs.load_params(nu=nu), x, u).shape[0]
    for rho, phi in [(1.0, 0.3), (2.5, -2.0), (0.1, 1.1)]:
        for scale, sign in [(1.0, 0), (1.3, -1), (0.7, 1)]:
            x[1:4] = [scale * tg * rho, rho * math.cos(phi), rho * math.sin(phi)]
            g = oracle.g(p, x, u)
            assert g.shape[0] == n_off + 1
            ref = tg * tg * rho * rho - x[1] ** 2
            assert abs(g[-1] - ref) <= 1e-12 * max(1.0, abs(ref))
            assert (sign == 0 and abs(g[-1]) < 1e-12) or np.sign(g[-1]) == sign


@pytest.mark.parametrize("nu", [4, 7])
def test_jacobians_with_glide_slope_match_central_differences(oracle, inputs, nu):
    """df/dx with the glide-slope row active (states below the cone)."""
    p = inputs.load_params(nu=nu, glide_slope=1)
    rng = np.random.default_rng(10 + nu)
    for trial in range(4):
        x = rand_state(rng)
        x[1] = 0.2 * abs(x[1]) + 0.05  # low altitude: outside the cone
        u = rand_control(rng, nu)
        assert oracle.g(p, x, u)[-1] > 0
        A, B = oracle.jac(p, x, u)
        h = 1e-6
        for j in range(15):
            e = np.zeros(15); e[j] = h
            fd = (oracle.f(p, x + e, u) - oracle.f(p, x - e, u)) / (2 * h)
            np.testing.assert_allclose(A[:, j], fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(fd).max()))


def test_time_bound_box_is_sufficient(oracle, inputs):
    """The node box on s of the scaled subproblem is [max(s_min, dt_min (N-1)),
    min(s_max, dt_max (N-1), tf_max)], and every FOH dilation profile inside it
    satisfies dt_min <= Delta t_k <= dt_max and t_f <= tf_max (Sec. 2.2)."""
    p = inputs.load_params(dt_min=0.3, dt_max=0.5, tf_max=6.6)
    N, nu = 12, 4
    x0 = p["x0_nominal"]
    X, U = oracle.init_guess(p, N, x0)
    A, Bm, Bp, xp = oracle.discretize(p, X, U)
    qp = oracle.scale(p, x0, X, U, A, Bm, Bp, xp)
    lo = max(p["s_min"], 0.3 * (N - 1))
    hi = min(p["s_max"], 0.5 * (N - 1), 6.6)
    Ps = p["P_u"][nu - 1]
    np.testing.assert_allclose(qp.umin[:, -1], (lo - U[:, -1]) / Ps, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(qp.umax[:, -1], (hi - U[:, -1]) / Ps, rtol=1e-15, atol=1e-15)
    assert np.all(np.isinf(qp.umin[:, :-1]))
    rng = np.random.default_rng(3)
    for _ in range(200):
        s = rng.uniform(lo, hi, N)
        dt = (s[:-1] + s[1:]) / (2 * (N - 1))
        assert dt.min() >= 0.3 - 1e-12 and dt.max() <= 0.5 + 1e-12 and dt.sum() <= 6.6 + 1e-12


def test_converged_solution_meets_glide_slope_and_time_bounds(oracle, inputs):
    p = inputs.load_params(glide_slope=1, dt_min=0.3, dt_max=0.5, tf_max=6.6)
    N = 15
    x0s = inputs.dispersion(p, 8, 31, "bj")
    res = oracle.solve_batch(p, x0s, np.full(8, N, np.int32))
    ok = np.nonzero(res["status"] == 0)[0]
    assert len(ok) >= 3
    tg = math.tan(p["gamma_gs"])
    for b in ok:
        X, U = res["X"][b], res["U"][b]
        s = U[:, -1]
        dt = (s[:-1] + s[1:]) / (2 * (N - 1))
        assert dt.min() >= 0.3 - 1e-9 and dt.max() <= 0.5 + 1e-9 and res["tf"][b] <= 6.6 + 1e-9
        # glide slope between nodes: re-propagate each interval finely
        for k in range(N - 1):
            x = X[k].copy()
            for i in range(20):
                lp0, lp1 = i / 20, (i + 1) / 20
                a = (1 - lp0) * U[k] + lp0 * U[k + 1]
                c = (1 - lp1) * U[k] + lp1 * U[k + 1]
                a[-1] /= (N - 1) * 20; c[-1] /= (N - 1) * 20
                x = oracle.flow(p, x, a, c, 10)
                assert tg * math.hypot(x[2], x[3]) - x[1] <= 0.05, (b, k, i)
