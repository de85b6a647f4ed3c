"""Pins of the oracle's second instance of the problem template of Sec. 2: the
translational 3-DoF powered-descent model (x = (m, r, v, y), inertial thrust).

The pins come from outside the oracle: the rocket equation integrated in
closed form under a constant inertial thrust, the 6-DoF model of Sec. 4 (a
separately pinned library) at level attitude and zero rate, central
differences, the dense canonical QP of Eq. parsed-data with Alg. 1, KKT
conditions, and an impulse bound that every feasible trajectory obeys."""
import math

import numpy as np
import pytest

NX3 = 8


@pytest.fixture(scope="module")
def p3(inputs):
    return inputs.load_params(model="3dof")


def _rand_state(rng, m=1.7):
    return np.concatenate([[m], rng.normal(size=3) * 3, rng.normal(size=3), [0.01]])


def _rand_control(rng, s=4.0):
    return np.concatenate([rng.normal(size=3) * 3, [s]])


def test_model_dimensions(oracle, p3):
    assert oracle.lib("3dof").orc_nx() == NX3 and oracle.lib("6dof").orc_nx() == 15
    x = _rand_state(np.random.default_rng(0))
    u = _rand_control(np.random.default_rng(1))
    assert oracle.F(p3, x, u).shape == (NX3 - 1,)
    assert oracle.f(p3, x, u).shape == (NX3,)
    assert oracle.g(p3, x, u).shape == (6,)
    assert oracle.g(dict(p3, glide_slope=1), x, u).shape == (7,)


def test_rocket_equation_with_inertial_thrust(oracle, p3):
    """Constant thrust T along a fixed inertial direction e, magnitude c:
    m(t) = m0 - a c t, v(t) = v0 + g t + (e / a) ln(m0 / m(t)),
    r(t) = r0 + v0 t + g t^2 / 2 + e (m(t) ln(m(t)/m0) + m0 - m(t)) / (a^2 c)."""
    p = dict(p3)
    p["T_min"], p["T_max"] = 0.0, 100.0
    a = p["alpha_mdot"]
    g = np.asarray(p["g_I"])
    e = np.array([0.8, -0.36, 0.48])
    e /= np.linalg.norm(e)
    c, t, m0 = 3.0, 2.5, 2.0
    r0, v0 = np.array([10.0, 2.0, -1.0]), np.array([-0.5, 0.3, 0.1])
    x = np.concatenate([[m0], r0, v0, [0.0]])
    u = np.concatenate([c * e, [t]])
    xt = oracle.flow(p, x, u, u, 4000)
    mt = m0 - a * c * t
    vt = v0 + g * t + e * math.log(m0 / mt) / a
    rt = r0 + v0 * t + 0.5 * g * t * t + e * (mt * math.log(mt / m0) + m0 - mt) / (a * a * c)
    assert abs(xt[0] - mt) < 1e-12
    np.testing.assert_allclose(xt[4:7], vt, atol=1e-10)
    np.testing.assert_allclose(xt[1:4], rt, atol=1e-10)


def test_matches_6dof_model_at_level_attitude(oracle, inputs, p3):
    """With q = identity and omega = 0 the 6-DoF model's body thrust is
    inertial and its attitude rows are inactive: its translational rows, CTCS
    rate and their derivatives in (m, r, v, y) and (T, s) are the 3-DoF
    model's (the 6-DoF gimbal row is the 3-DoF pointing row)."""
    rng = np.random.default_rng(4)
    for gs in (0, 1):
        p6 = inputs.load_params(nu=4, glide_slope=gs)
        p6["delta_max"] = p3["delta_max"]
        q3 = dict(p3, glide_slope=gs)
        for trial in range(6):
            x3 = _rand_state(rng)
            u = _rand_control(rng)
            if trial % 2:  # drive constraints active
                x3[0] = 0.9
                x3[1] = -0.5
                u[:3] = [0.2, 4.0, 3.0]
            x6 = np.concatenate([x3[:7], [1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0], x3[7:]])
            sel = [0, 1, 2, 3, 4, 5, 6, 14]
            np.testing.assert_allclose(oracle.f(q3, x3, u), oracle.f(p6, x6, u)[sel], rtol=1e-13, atol=1e-13)
            A3, B3 = oracle.jac(q3, x3, u)
            A6, B6 = oracle.jac(p6, x6, u)
            np.testing.assert_allclose(A3, A6[np.ix_(sel, sel)], rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(B3, B6[sel], rtol=1e-13, atol=1e-13)


def test_path_constraint_boundaries(oracle, p3):
    """Each row of the 3-DoF g is zero exactly on its bound."""
    p = p3
    d, Tm = p["delta_max"], p["T_max"]
    x = np.array([p["m_dry"], 0.0, 1.0, 2.0, p["v_max"], 0.0, 0.0, 0.0])
    u = np.array([Tm * math.cos(d), Tm * math.sin(d) * 0.6, Tm * math.sin(d) * 0.8, 1.0])
    g = oracle.g(p, x, u)
    np.testing.assert_allclose(g[:5], 0.0, atol=1e-12)
    assert abs(g[5] - (p["T_min"] - Tm)) < 1e-12
    # straight up: inside the pointing cone by 1 - sec(delta)
    g2 = oracle.g(p, x, np.array([2.0, 0.0, 0.0, 1.0]))
    assert abs(g2[3] - 2.0 * (1.0 - 1.0 / math.cos(d))) < 1e-12
    # glide slope on: zero on the cone tan(gamma_gs) ||(r_y, r_z)|| = r_x
    q = dict(p, glide_slope=1)
    gg = p["gamma_gs"]
    x3 = x.copy()
    x3[1:4] = [3.0 * math.tan(gg), 3.0 * 0.6, 3.0 * 0.8]
    assert abs(oracle.g(q, x3, u)[6]) < 1e-12
    # CTCS integrand: s * sum |g|_+^2
    x2 = x.copy()
    x2[0] = p["m_dry"] - 0.1
    assert abs(oracle.f(p, x2, u)[7] - 0.1 ** 2) < 1e-12


@pytest.mark.parametrize("gs", [0, 1])
def test_jacobians_match_central_differences(oracle, p3, gs):
    p = dict(p3, glide_slope=gs)
    rng = np.random.default_rng(30 + gs)
    for _ in range(6):
        x, u = _rand_state(rng), _rand_control(rng)
        A, B = oracle.jac(p, x, u)
        h = 1e-6
        for j in range(NX3):
            e = np.zeros(NX3); e[j] = h
            fd = (oracle.f(p, x + e, u) - oracle.f(p, x - e, u)) / (2 * h)
            np.testing.assert_allclose(A[:, j], fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(fd).max()))
        for j in range(4):
            e = np.zeros(4); e[j] = h
            fd = (oracle.f(p, x, u + e) - oracle.f(p, x, u - e)) / (2 * h)
            np.testing.assert_allclose(B[:, j], fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(fd).max()))


def test_stm_is_derivative_of_rk4_flow(oracle, p3):
    p = p3
    rng = np.random.default_rng(12)
    N = 5
    X = rng.normal(size=(N, NX3)) * 0.3
    X[:, 0] = 1.8
    U = np.tile(_rand_control(rng), (N, 1)) + rng.normal(size=(N, 4)) * 0.2
    A, Bm, Bp, xp = oracle.discretize(p, X, U)

    def fk(xk, uk, uk1):
        uk = np.array(uk); uk1 = np.array(uk1)
        uk[-1] /= (N - 1); uk1[-1] /= (N - 1)
        return oracle.flow(p, xk, uk, uk1, p["rk4_substeps"])

    h = 1e-6
    for k in (0, 2):
        np.testing.assert_allclose(xp[k], fk(X[k], U[k], U[k + 1]), rtol=1e-13, atol=1e-13)
        for j in range(NX3):
            e = np.zeros(NX3); e[j] = h
            fd = (fk(X[k] + e, U[k], U[k + 1]) - fk(X[k] - e, U[k], U[k + 1])) / (2 * h)
            np.testing.assert_allclose(A[k][:, j], fd, atol=2e-7 * (1 + np.abs(fd).max()))
        for j in range(4):
            e = np.zeros(4); e[j] = h
            fdm = (fk(X[k], U[k] + e, U[k + 1]) - fk(X[k], U[k] - e, U[k + 1])) / (2 * h)
            fdp = (fk(X[k], U[k], U[k + 1] + e) - fk(X[k], U[k], U[k + 1] - e)) / (2 * h)
            np.testing.assert_allclose(Bm[k][:, j], fdm, atol=2e-7 * (1 + np.abs(fdm).max()))
            np.testing.assert_allclose(Bp[k][:, j], fdp, atol=2e-7 * (1 + np.abs(fdp).max()))


def _subproblem(O, I, N, seed, perturb):
    p = I.load_params(model="3dof")
    x0 = I.dispersion(p, 1, seed, "bj")[0]
    X, U = O.init_guess(p, N, x0)
    rng = np.random.default_rng(seed)
    X[1:] += rng.normal(size=X[1:].shape) * perturb * p["P_x"]
    U += rng.normal(size=U.shape) * perturb * p["P_u"][:4]
    A, Bm, Bp, xp = O.discretize(p, X, U)
    return p, O.scale(p, x0, X, U, A, Bm, Bp, xp)


@pytest.mark.parametrize("N", [3, 6])
def test_pipgc_equals_alg1_on_dense_qp(oracle, inputs, N):
    """The block recursion of PIPG_custom on the 3-DoF subproblem produces the
    iterates of Alg. 1 on its dense canonical QP."""
    p, qp = _subproblem(oracle, inputs, N, 5, 0.1)
    assert qp.Am.shape == (N - 1, NX3, NX3)
    ws0 = oracle.PDState(N, 4, "3dof")
    rng = np.random.default_rng(6)
    for k in ("xh", "uh", "mup", "mum", "phi", "th"):
        a = getattr(ws0, k)
        a[...] = np.abs(rng.normal(size=a.shape)) * 0.1
    sig, _ = oracle.power(p, qp, ws0)
    D = oracle.qp_dense(qp)
    K = np.vstack([D["G"], D["H"]])
    assert sig / (1 + p["pow_eps_buff"]) <= np.linalg.eigvalsh(K.T @ K).max() * (1 + 1e-12)
    for J in (1, 9, 40):
        w1 = ws0.copy()
        assert oracle.pipgc(p, qp, sig, w1, force_iters=J) == J
        wp, om = p["w_prox"], p["pipg_omega"]
        alpha = 2.0 / (wp + np.sqrt(wp * wp + 4 * om * sig))
        z, w, v = oracle.pipg_generic(qp, alpha, om, p["pipg_rho"], J, oracle.z_pack(qp, ws0),
                                      ws0.phi.ravel().copy(), ws0.th.copy())
        np.testing.assert_allclose(oracle.z_pack(qp, w1), z, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w1.phi.ravel(), w, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w1.th, v, rtol=1e-12, atol=1e-12)


def test_pipgc_reaches_kkt_point(oracle, inputs):
    p, qp = _subproblem(oracle, inputs, 4, 7, 0.02)
    ws = oracle.PDState(4, 4, "3dof")
    sig, _ = oracle.power(p, qp, ws)
    oracle.pipgc(p, qp, sig, ws, force_iters=60000)
    D = oracle.qp_dense(qp)
    z, eta, chi = oracle.z_pack(qp, ws), ws.phi.ravel(), ws.th
    grad = D["P"] @ z + D["p"] + D["G"].T @ eta + D["H"].T @ chi
    assert np.abs(D["G"] @ z - D["g"]).max() < 1e-8
    assert max(0.0, (D["H"] @ z - D["h"]).max()) < 1e-8
    assert np.abs(z - np.clip(z - grad, D["lo"], D["hi"])).max() < 1e-8
    assert chi.min() >= 0.0
    assert np.abs(chi * (D["H"] @ z - D["h"])).max() < 1e-8


@pytest.mark.parametrize("soc", [0, 1])
def test_converged_solution_is_feasible(oracle, inputs, soc):
    """A converged 3-DoF solve meets the boundary conditions, the dynamics on
    re-propagation, the CTCS budget and the path constraints, and its
    propellant obeys the impulse bound of any feasible trajectory:
    m0 - m_f >= m0 (1 - exp(-a ||v_f - v0 - g t_f||)), since
    int T/m dt = v_f - v0 - g t_f and -dm/m = a ||T||/m dt."""
    p = inputs.load_params(model="3dof", soc_thrust=soc)
    N = 15
    x0s = inputs.dispersion(p, 3, 23, "bj")
    for x0 in x0s:
        r = oracle.solve(p, N, x0)
        assert r["status"] == 0, r
        X, U = r["X"], r["U"]
        np.testing.assert_allclose(X[0, :7], x0, atol=1e-12)
        fx = p["fix_f"].astype(bool)
        np.testing.assert_allclose(X[-1][fx], p["z_f"][fx], atol=1e-9)
        for k in range(N - 1):
            uk, uk1 = U[k].copy(), U[k + 1].copy()
            uk[-1] /= (N - 1); uk1[-1] /= (N - 1)
            d = np.abs(oracle.flow(p, X[k], uk, uk1, 200) - X[k + 1])[:7] / p["P_x"][:7]
            assert d.max() < 2e-3
        assert X[-1, 7] - X[0, 7] <= (N - 1) * p["eps_ctcs"] + 1e-9
        assert np.all(np.diff(X[:, 0]) <= 1e-12)
        for k in range(N):
            assert np.max(oracle.g(p, X[k], U[k])) < 0.05
        if soc:
            a = math.tan(p["delta_max"])
            for T in U[:, :3]:
                assert np.linalg.norm(T) <= p["T_max"] * (1 + 1e-6)
                assert np.linalg.norm(T[1:]) <= a * T[0] + 1e-6
        m0, a_m = x0[0], p["alpha_mdot"]
        dv = np.linalg.norm(X[-1, 4:7] - x0[4:7] - np.asarray(p["g_I"]) * r["tf"])
        assert r["fuel"] >= m0 * (1.0 - math.exp(-a_m * dv)) - 1e-3
        assert r["fuel"] <= m0 - p["m_dry"]


def test_paper_distribution_converges(oracle, inputs):
    p = inputs.load_params(model="3dof")
    x0 = inputs.dispersion(p, 32, inputs.config_seed(0), "paper256")
    b = oracle.solve_batch(p, x0, np.full(32, 15, np.int32))
    assert np.mean(b["status"] == 0) >= 0.9  # 250 of 256 at this seed
