"""Pins of the oracle's scaled subproblem and solver (Sec. 2.3.2, Sec. 3):
the scaling identity, the power iteration against dense eigenvalues, block
PIPG_custom against Alg. 1 on the dense canonical QP, KKT residuals at
convergence, and an equality-only instance solved by a library routine."""
import numpy as np
import pytest

from conftest import rand_control


def _subproblem(O, I, nu=4, N=4, seed=0, perturb=0.0):
    p = I.load_params(nu=nu)
    x0 = I.dispersion(p, 1, seed, "bj")[0]
    X, U = O.init_guess(p, N, x0)
    if perturb:
        rng = np.random.default_rng(seed)
        X[1:] += rng.normal(size=X[1:].shape) * perturb * p["P_x"]
        U += rng.normal(size=U.shape) * perturb * p["P_u"][:nu]
    A, Bm, Bp, xp = O.discretize(p, X, U)
    qp = O.scale(p, x0, X, U, A, Bm, Bp, xp)
    return p, x0, X, U, (A, Bm, Bp, xp), qp


@pytest.mark.parametrize("nu", [4, 7])
def test_scaling_identity(oracle, inputs, nu):
    """K(x_hat, u_hat, 0) + w_hat = P_x^{-1} (unscaled linearized residual)."""
    p, x0, X, U, (A, Bm, Bp, xp), qp = _subproblem(oracle, inputs, nu, N=5, seed=1, perturb=0.05)
    rng = np.random.default_rng(2)
    N = X.shape[0]
    xh = rng.normal(size=(N, 15)); uh = rng.normal(size=(N, nu))
    Px, Pu = p["P_x"], p["P_u"][:nu]
    x = X + xh * Px; u = U + uh * Pu
    for k in range(N - 1):
        lhs = qp.Am[k] @ xh[k] + qp.Ap[k] @ xh[k + 1] + qp.Bm[k] @ uh[k] + qp.Bp[k] @ uh[k + 1] + qp.w[k]
        res = A[k] @ (x[k] - X[k]) + Bm[k] @ (u[k] - U[k]) + Bp[k] @ (u[k + 1] - U[k + 1]) + xp[k] - x[k + 1]
        np.testing.assert_allclose(lhs, res / Px, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(qp.Ap[k], -np.eye(15))
        # relaxed CTCS row: y_{k+1} - y_k <= eps  <=>  E_y(xh_{k+1} - xh_k) <= eps_hat_k
        dy = x[k + 1, 14] - x[k, 14]
        dyh = xh[k + 1, 14] - xh[k, 14]
        assert abs((dyh - qp.eps[k]) * Px[14] - (dy - p["eps_ctcs"])) < 1e-12
    # box on the dilation only; boundary values
    s = nu - 1
    np.testing.assert_allclose(U[:, s] + qp.umin[:, s] * Pu[s], p["s_min"], atol=1e-12)
    np.testing.assert_allclose(U[:, s] + qp.umax[:, s] * Pu[s], p["s_max"], atol=1e-12)
    assert np.all(np.isinf(qp.umin[:, :s])) and np.all(np.isinf(qp.umax[:, :s]))
    xi = np.concatenate([x0, [0.0]])
    np.testing.assert_allclose(X[0] + qp.zi * Px, xi, atol=1e-12)
    fx = p["fix_f"].astype(bool)
    np.testing.assert_allclose((X[-1] + qp.zf * Px)[fx], p["z_f"][fx], atol=1e-12)


def test_jacobi_matches_library(oracle):
    rng = np.random.default_rng(4)
    M = rng.normal(size=(30, 30)); M = M + M.T
    assert abs(oracle.sym_eig_max(M) - np.linalg.eigvalsh(M).max()) < 1e-10


@pytest.mark.parametrize("nu", [4, 7])
def test_power_iteration_bounds(oracle, inputs, nu):
    """sigma*/(1+eps_buff) is a Rayleigh-type lower estimate of
    lambda_max(K^T K), K = [G; H_y]; it converges to it."""
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, nu, N=4, seed=3, perturb=0.05)
    D = oracle.qp_dense(qp)
    K = np.vstack([D["G"], D["H"]])
    lam = oracle.sym_eig_max(K.T @ K)
    assert abs(lam - np.linalg.eigvalsh(K.T @ K).max()) < 1e-9 * lam
    ws = oracle.PDState(qp.N, nu)
    sig, it = oracle.power(p, qp, ws)
    assert 1 <= it <= p["pow_jmax"]
    s0 = sig / (1 + p["pow_eps_buff"])
    assert s0 <= lam * (1 + 1e-12)
    sig2, it2 = oracle.power(p, qp, ws, force_iters=3000)
    assert it2 == 3000
    assert 0.0 <= lam - sig2 / (1 + p["pow_eps_buff"]) < 1e-3 * lam


def _random_ws(O, N, nu, seed):
    ws = O.PDState(N, nu)
    rng = np.random.default_rng(seed)
    for k in ("xh", "uh", "mup", "mum", "phi", "th"):
        a = getattr(ws, k)
        a[...] = np.abs(rng.normal(size=a.shape)) * 0.1
    return ws


@pytest.mark.parametrize("nu,N", [(4, 3), (4, 5), (7, 4)])
def test_pipgc_equals_alg1_on_dense_qp(oracle, inputs, nu, N):
    """The block recursion of PIPG_custom produces the iterates of Alg. 1 on
    the canonical QP assembled densely from Eq. parsed-data."""
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, nu, N=N, seed=5, perturb=0.1)
    ws0 = _random_ws(oracle, N, nu, 6)
    sig, _ = oracle.power(p, qp, ws0)
    for J in (1, 7, 41):
        w1 = ws0.copy()
        n = oracle.pipgc(p, qp, sig, w1, force_iters=J)
        assert n == J
        wp, om = p["w_prox"], p["pipg_omega"]
        alpha = 2.0 / (wp + np.sqrt(wp * wp + 4 * om * sig))
        z, w, v = oracle.pipg_generic(qp, alpha, om, p["pipg_rho"], J, oracle.z_pack(qp, ws0),
                                      ws0.phi.ravel().copy(), ws0.th.copy())
        np.testing.assert_allclose(oracle.z_pack(qp, w1), z, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w1.phi.ravel(), w, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w1.th, v, rtol=1e-12, atol=1e-12)


def _kkt(D, z, eta, chi):
    G, g, H, h, P, pv, lo, hi = (D[k] for k in ("G", "g", "H", "h", "P", "p", "lo", "hi"))
    grad = P @ z + pv + G.T @ eta + H.T @ chi
    return dict(prim=np.abs(G @ z - g).max(), ineq=max(0.0, (H @ z - h).max()),
                stat=np.abs(z - np.clip(z - grad, lo, hi)).max(),
                dual=max(0.0, -chi.min()), compl=np.abs(chi * (H @ z - h)).max())


@pytest.mark.parametrize("nu", [4, 7])
def test_pipgc_reaches_kkt_point(oracle, inputs, nu):
    """After enough iterations the PIPG_custom output satisfies the KKT
    conditions of Eq. cvx-subproblem-custom (box/nonnegativity normal cones,
    fixed boundary components, complementarity of the CTCS rows)."""
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, nu, N=4, seed=7, perturb=0.02)
    ws = oracle.PDState(qp.N, nu)
    sig, _ = oracle.power(p, qp, ws)
    oracle.pipgc(p, qp, sig, ws, force_iters=60000 if nu == 4 else 600000)
    D = oracle.qp_dense(qp)
    r = _kkt(D, oracle.z_pack(qp, ws), ws.phi.ravel(), ws.th)
    for k, v in r.items():
        assert v < 1e-8, (k, v)


def test_equality_only_subproblem_matches_linear_solve(oracle, inputs):
    """When no inequality is active (mu = 0, dilation box and CTCS rows slack)
    the QP is equality constrained; its solution solves the KKT linear system
    (numpy.linalg.solve)."""
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, 4, N=4, seed=8, perturb=0.0)
    qp.eps[:] = 10.0  # make the CTCS rows slack
    D = oracle.qp_dense(qp)
    nu, N = 4, qp.N
    nv = (15 + nu) * N  # x_hat, u_hat; mu fixed at 0
    G = D["G"][:, :nv]
    fixed = [i for i in range(nv) if D["lo"][i] == D["hi"][i]]
    E = np.zeros((len(fixed), nv))
    for r, i in enumerate(fixed):
        E[r, i] = 1.0
    Aeq = np.vstack([G, E])
    beq = np.concatenate([D["g"], D["lo"][fixed]])
    Pm = D["P"][:nv, :nv]
    c = D["p"][:nv]
    KKT = np.block([[Pm, Aeq.T], [Aeq, np.zeros((Aeq.shape[0], Aeq.shape[0]))]])
    sol = np.linalg.lstsq(KKT, np.concatenate([-c, beq]), rcond=None)[0]
    v = sol[:nv]
    ws = oracle.PDState(N, nu)
    sig, _ = oracle.power(p, qp, ws)
    oracle.pipgc(p, qp, sig, ws, force_iters=60000)
    z = oracle.z_pack(qp, ws)
    # the assumed active set holds at the PIPG solution
    assert np.abs(z[nv:]).max() < 1e-12
    assert np.abs(ws.phi).max() < p["w_ep"]
    s = z[15 * N + nu - 1: nv: nu]
    assert np.all(s > D["lo"][15 * N + nu - 1: nv: nu]) and np.all(s < D["hi"][15 * N + nu - 1: nv: nu])
    np.testing.assert_allclose(z[:nv], v, atol=1e-9)


def test_stop_test_fires_at_fixed_point(oracle, inputs):
    """Warm-started at a fixed point, PIPG_custom terminates at the first
    stopping check (iteration j_check, Alg. stopping)."""
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, 4, N=4, seed=9)
    ws = oracle.PDState(qp.N, 4)
    sig, _ = oracle.power(p, qp, ws)
    oracle.pipgc(p, qp, sig, ws, force_iters=60000)
    n = oracle.pipgc(p, qp, sig, ws)
    assert n == p["pipg_jcheck"]
    ws2 = oracle.PDState(qp.N, 4)
    assert oracle.pipgc(p, qp, sig, ws2) > p["pipg_jcheck"]
