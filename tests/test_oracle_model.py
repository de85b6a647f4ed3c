"""Pins of the oracle's model and discretization (Sec. 4, Sec. 2.1-2.3.1)
against closed forms, finite differences and invariants."""
import math

import numpy as np
import pytest

from conftest import rand_control, rand_state


def _fine_flow(O, p, x, u, t, nsub=4000):
    """Integrate the time-domain dynamics for duration t with constant u by
    running the tau-flow over a unit interval with dilation s = t."""
    u = np.array(u, dtype=np.float64)
    u[-1] = t
    return O.flow(p, x, u, u, nsub)


def test_rocket_equation(oracle, params):
    """Thrust along body x, identity attitude, no rotation: m(t) = m0 - a T t and
    v_x(t) = v0 + ln(m0/m(t))/a - g t (Tsiolkovsky with gravity)."""
    p = dict(params)
    p["T_min"], p["T_max"] = 0.0, 100.0
    x = np.zeros(15)
    x[0], x[1], x[4], x[7] = 2.0, 10.0, -0.5, 1.0
    T, t = 3.0, 2.5
    u = np.array([T, 0.0, 0.0, t])
    xt = _fine_flow(oracle, p, x, u, t)
    a, g0 = p["alpha_mdot"], -p["g_I"][0]
    m_t = 2.0 - a * T * t
    v_t = -0.5 + math.log(2.0 / m_t) / a - g0 * t
    assert abs(xt[0] - m_t) < 1e-12
    assert abs(xt[4] - v_t) < 1e-10
    np.testing.assert_allclose(xt[7:11], [1, 0, 0, 0], atol=1e-14)
    np.testing.assert_allclose(xt[11:14], 0.0, atol=1e-14)


def test_torque_free_principal_spin(oracle, params):
    """Zero thrust, spin about the body y principal axis: omega constant and
    q(t) = q0 (x) (cos(wt/2), sin(wt/2) e_y)."""
    x = np.zeros(15)
    x[0], x[7], x[12] = 2.0, 1.0, 0.4
    t = 3.0
    xt = _fine_flow(oracle, params, x, [0.0, 0.0, 0.0, t], t)
    np.testing.assert_allclose(xt[11:14], [0, 0.4, 0], atol=1e-14)
    ang = 0.4 * t
    np.testing.assert_allclose(xt[7:11], [math.cos(ang / 2), 0, math.sin(ang / 2), 0], atol=1e-12)


def test_symmetric_top_precession(oracle, params):
    """J = diag(Jx, Jt, Jt), no torque: omega_x constant and (omega_y, omega_z)
    rotates at rate k = (Jt - Jx) omega_x / Jt (Euler's equations): pins the
    sign of the gyroscopic term."""
    p = dict(params)
    Jx, Jt = p["J_B"][0], p["J_B"][1]
    assert p["J_B"][1] == p["J_B"][2] != Jx
    x = np.zeros(15)
    x[0], x[7] = 2.0, 1.0
    x[11:14] = [0.3, 0.1, -0.05]
    t = 2.0
    xt = _fine_flow(oracle, p, x, [0.0, 0.0, 0.0, t], t)
    k = (Jt - Jx) * 0.3 / Jt
    wy = 0.1 * math.cos(k * t) + (-0.05) * math.sin(k * t)
    wz = -0.05 * math.cos(k * t) - 0.1 * math.sin(k * t)
    np.testing.assert_allclose(xt[11:14], [0.3, wy, wz], atol=1e-11)


def test_quaternion_norm_and_mass_monotone(oracle, params):
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rand_state(rng)
        x[7:11] /= np.linalg.norm(x[7:11])
        u = rand_control(rng, 4, s=1.0)
        xt = oracle.flow(params, x, u, u, 2000)
        assert abs(np.linalg.norm(xt[7:11]) - 1.0) < 1e-12
        assert xt[0] <= x[0]
        assert oracle.F(params, x, u)[0] <= 0.0


def test_path_constraints_boundaries(oracle, params7):
    """Each row of g is zero exactly on its bound (Sec. 4; tilt row reading)."""
    p = params7
    x = np.zeros(15)
    x[0] = p["m_dry"]
    x[1] = 0.0
    x[4:7] = [p["v_max"], 0, 0]
    th = p["theta_max"]  # tilt about inertial y by theta_max
    x[7:11] = [math.cos(th / 2), 0, math.sin(th / 2), 0]
    x[11:14] = [0, p["omega_max"], 0]
    d = p["delta_max"]
    Tm = p["T_max"]
    u = np.array([Tm * math.cos(d), Tm * math.sin(d), 0.0, 0.0, p["gamma_max"], 0.0, 1.0])
    g = oracle.g(p, x, u)
    assert g.shape == (9,)
    np.testing.assert_allclose(g[[0, 1, 2, 3, 4, 5, 6, 8]], 0.0, atol=1e-12)
    assert abs(g[7] - (p["T_min"] - Tm)) < 1e-12
    # CTCS integrand: s * sum |g|_+^2
    x2 = x.copy()
    x2[0] = p["m_dry"] - 0.1
    f = oracle.f(p, x2, u)
    assert abs(f[14] - 1.0 * 0.1 ** 2) < 1e-12


@pytest.mark.parametrize("nu", [4, 7])
def test_jacobians_match_central_differences(oracle, inputs, nu):
    p = inputs.load_params(nu=nu)
    rng = np.random.default_rng(nu)
    for trial in range(4):
        x = rand_state(rng)
        u = rand_control(rng, nu)
        A, B = oracle.jac(p, x, u)
        h = 1e-6
        for j in range(15):
            e = np.zeros(15); e[j] = h
            fd = (oracle.f(p, x + e, u) - oracle.f(p, x - e, u)) / (2 * h)
            np.testing.assert_allclose(A[:, j], fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(fd).max()))
        for j in range(nu):
            e = np.zeros(nu); e[j] = h
            fd = (oracle.f(p, x, u + e) - oracle.f(p, x, u - e)) / (2 * h)
            np.testing.assert_allclose(B[:, j], fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(fd).max()))


def _tau_flow(O, p, N, xk, uk, uk1):
    """f_k of Eq. disc-dyn on the uniform grid (interval length 1/(N-1))."""
    uk = np.array(uk, dtype=np.float64); uk1 = np.array(uk1, dtype=np.float64)
    uk[-1] /= (N - 1); uk1[-1] /= (N - 1)
    return O.flow(p, xk, uk, uk1, p["rk4_substeps"])


@pytest.mark.parametrize("nu", [4, 7])
def test_stm_is_derivative_of_rk4_flow(oracle, inputs, nu):
    """A_k, B^-_k, B^+_k from the joint IVP (Sec. 2.3.1) integrated by the same
    RK4 are the exact derivatives of the discrete flow map: match central
    differences of f_k.  x-bar^k(tau_{k+1}) equals f_k itself."""
    p = inputs.load_params(nu=nu)
    rng = np.random.default_rng(10 + nu)
    N = 6
    X = rng.normal(size=(N, 15)) * 0.3
    X[:, 0] = 1.8
    X[:, 7] += 1.0
    U = np.tile(rand_control(rng, nu), (N, 1)) + rng.normal(size=(N, nu)) * 0.2
    A, Bm, Bp, xp = oracle.discretize(p, X, U)
    h = 1e-6
    for k in (0, 3):
        np.testing.assert_allclose(xp[k], _tau_flow(oracle, p, N, X[k], U[k], U[k + 1]), rtol=1e-13, atol=1e-13)
        for j in range(15):
            e = np.zeros(15); e[j] = h
            fd = (_tau_flow(oracle, p, N, X[k] + e, U[k], U[k + 1]) -
                  _tau_flow(oracle, p, N, X[k] - e, U[k], U[k + 1])) / (2 * h)
            np.testing.assert_allclose(A[k][:, j], fd, atol=2e-7 * (1 + np.abs(fd).max()))
        for j in range(nu):
            e = np.zeros(nu); e[j] = h
            fdm = (_tau_flow(oracle, p, N, X[k], U[k] + e, U[k + 1]) -
                   _tau_flow(oracle, p, N, X[k], U[k] - e, U[k + 1])) / (2 * h)
            fdp = (_tau_flow(oracle, p, N, X[k], U[k], U[k + 1] + e) -
                   _tau_flow(oracle, p, N, X[k], U[k], U[k + 1] - e)) / (2 * h)
            np.testing.assert_allclose(Bm[k][:, j], fdm, atol=2e-7 * (1 + np.abs(fdm).max()))
            np.testing.assert_allclose(Bp[k][:, j], fdp, atol=2e-7 * (1 + np.abs(fdp).max()))


def test_rk4_fourth_order(oracle, params):
    """The 10-substep flow agrees with a 2000-substep flow to O(h^4): halving
    h shrinks the error about 16x."""
    rng = np.random.default_rng(5)
    x = rand_state(rng)
    x[7:11] /= np.linalg.norm(x[7:11])
    uk, uk1 = rand_control(rng, 4, 0.5), rand_control(rng, 4, 0.6)
    ref = oracle.flow(params, x, uk, uk1, 2000)
    e1 = np.abs(oracle.flow(params, x, uk, uk1, 10) - ref)[:14].max()
    e2 = np.abs(oracle.flow(params, x, uk, uk1, 20) - ref)[:14].max()
    assert 10.0 < e1 / e2 < 22.0
