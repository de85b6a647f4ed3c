"""Pins of the oracle's stop decisions (Alg. stopping, Alg. power, the SCP
test of reading R8), its touchdown error and its initial guess (reading R9),
and of the checker that holds the GPU's stop decisions to the oracle's.

Alg. stopping is pinned by constructed iterate pairs whose decision follows
from the definition by hand (the infinity norm over every primal and dual
block, the larger of the two iterates' norms in the relative term, ties
terminating), and by a run whose decisions and margins are recomputed from
the iterates themselves, unextrapolated as Alg. PIPG_custom passes them."""
import numpy as np
import pytest

from gpu_helpers import check_stop_decisions
from test_oracle_qp import _subproblem


def _pair(O, N=3, nu=4):
    a = O.PDState(N, nu)
    a.xh[0, 0] = 1.0
    a.phi[1, 1] = 1.0
    return a, a.copy()


@pytest.fixture()
def stop_qp(oracle, inputs):
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, 4, N=3, seed=2)
    return p, qp


def test_stop_identical_pair_terminates(oracle, stop_qp):
    p, qp = stop_qp
    a, b = _pair(oracle)
    stop, m = oracle.stop_custom(p, qp, a, b)
    assert stop and m == -1.0  # (0 - thr) / thr


@pytest.mark.parametrize("block,idx", [("phi", (0, 3)), ("th", (1,)), ("xh", (2, 5)), ("uh", (1, 2)),
                                       ("mup", (1, 7)), ("mum", (0, 14))])
def test_stop_every_block_counts(oracle, stop_qp, block, idx):
    """A change of 0.05 in one entry of any block, against the threshold
    eps_abs + eps_rel max(|a|, |b|) = 1e-3 + 1e-2 * 1 = 0.011 of its group
    (primal: x, u, mu+, mu-; dual: phi, theta), keeps the loop running, with
    margin (0.05 - 0.011) / 0.011; a change of 0.005 does not."""
    p = dict(stop_qp[0], pipg_eps_abs=1e-3, pipg_eps_rel=1e-2)
    qp = stop_qp[1]
    for delta, want in ((0.05, False), (0.005, True)):
        a, b = _pair(oracle)
        getattr(b, block)[idx] += delta
        stop, m = oracle.stop_custom(p, qp, a, b)
        assert stop is want, (block, delta)
        assert abs(m - (delta - 0.011) / 0.011) < 1e-12


def test_stop_uses_the_infinity_norm(oracle, stop_qp):
    """Every entry of x moves by 0.008: the infinity norm of the change (0.008)
    is below the threshold 1e-3 + 1e-2 * 1.008 = 0.01108, its 2-norm (0.054)
    is not.  Alg. stopping uses the infinity norm, so the loop terminates."""
    p = dict(stop_qp[0], pipg_eps_abs=1e-3, pipg_eps_rel=1e-2)
    a, b = _pair(oracle)
    b.xh += 0.008
    assert np.linalg.norm((b.xh - a.xh).ravel()) > 0.01108
    stop, m = oracle.stop_custom(p, stop_qp[1], a, b)
    assert stop
    assert abs(m - (0.008 - 0.01108) / 0.01108) < 1e-12


def test_stop_relative_term_takes_the_larger_iterate_and_ties_terminate(oracle, stop_qp):
    """eps_abs = 0, eps_rel = 1/4 (exact in binary): x moves from 3 to 4, so
    the change 1 equals 1/4 max(3, 4) exactly and the tie terminates (R7); with
    the smaller iterate's norm (1/4 * 3) it would not."""
    p = dict(stop_qp[0], pipg_eps_abs=0.0, pipg_eps_rel=0.25)
    a, b = _pair(oracle)
    a.xh[1, 4], b.xh[1, 4] = 3.0, 4.0
    stop, m = oracle.stop_custom(p, stop_qp[1], a, b)
    assert stop and m == 0.0
    stop, _ = oracle.stop_custom(p, stop_qp[1], b, a)  # symmetric in the pair
    assert stop
    b.xh[1, 4] = 4.0 + 2 ** -40  # just past the tie
    assert not oracle.stop_custom(p, stop_qp[1], a, b)[0]


def _state_vec(s):
    return (np.concatenate([s.xh.ravel(), s.uh.ravel(), s.mup.ravel(), s.mum.ravel()]),
            np.concatenate([s.phi.ravel(), s.th.ravel()]))


def _margin(p, a, b):
    """Alg. stopping on the pair (a, b) of (primal, dual) vectors, by hand."""
    out = []
    for u, v in zip(a, b):
        thr = p["pipg_eps_abs"] + p["pipg_eps_rel"] * max(np.abs(u).max(), np.abs(v).max())
        out.append((np.abs(u - v).max() - thr) / thr)
    return max(out)


def test_pipg_stops_at_the_first_passing_check_of_unextrapolated_iterates(oracle, inputs):
    """Warm-started near the solution, PIPG_custom stops at the first check
    j = c j_check at which the pair of iterates (j, j - 1) passes.  The
    iterates z^j are taken from runs forced to j iterations; the oracle's
    margins at every check equal the margins recomputed from those pairs, and
    differ from the margins of the extrapolated iterates
    z~^j = (1 - rho) z~^(j-1) + rho z^j (z~^0 the warm start), so the test
    is the one on unextrapolated iterates."""
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, 4, N=4, seed=9, perturb=0.02)
    p = dict(p, pipg_jcheck=5)
    ws = oracle.PDState(qp.N, 4)
    sig, _ = oracle.power(p, qp, ws)
    oracle.pipgc(p, qp, sig, ws, force_iters=60000)
    rng = np.random.default_rng(3)
    w0 = ws.copy()
    for k in ("xh", "uh", "phi"):
        getattr(w0, k)[...] += rng.normal(size=getattr(w0, k).shape) * 1e-5
    n_free = oracle.pipgc(p, qp, sig, w0.copy())
    jc = p["pipg_jcheck"]
    assert jc < n_free < p["pipg_jmax"] and n_free % jc == 0
    n, m = oracle.pipgc(p, qp, sig, w0.copy(), force_iters=n_free, margins=True)
    assert n == n_free
    seq = [_state_vec(w0)]
    for j in range(1, n_free + 1):
        w = w0.copy()
        oracle.pipgc(p, qp, sig, w, force_iters=j)
        seq.append(_state_vec(w))
    rho = p["pipg_rho"]
    ext = [seq[0]]
    for j in range(1, n_free + 1):
        ext.append(tuple((1 - rho) * e + rho * z for e, z in zip(ext[-1], seq[j])))
    differ = 0
    for c in range(1, n_free // jc + 1):
        j = c * jc
        mine = _margin(p, seq[j], seq[j - 1])
        assert abs(m[c - 1] - mine) <= 1e-9 * abs(mine), (c, m[c - 1], mine)
        assert (mine <= 0) == (j == n_free), (j, mine)
        mext = _margin(p, ext[j], ext[j - 1])
        differ += abs(mext - mine) > 1e-3 * abs(mine)
    assert differ >= 1


def test_power_iteration_stops_at_its_first_passing_test(oracle, inputs):
    """Alg. power stops after the first iteration whose estimate changed by at
    most eps_abs + eps_rel max(sigma*, sigma); the margins of a forced run
    are positive before that iteration and not after it, and a forced run of
    exactly that many iterations gives the free run's estimate."""
    p, x0, X, U, _, qp = _subproblem(oracle, inputs, 4, N=5, seed=3, perturb=0.05)
    ws = oracle.PDState(qp.N, 4)
    sig, n = oracle.power(p, qp, ws)
    assert 1 < n < p["pow_jmax"]
    sig_n, _ = oracle.power(p, qp, ws, force_iters=n)
    assert sig_n == sig
    r = oracle.solve(p, 5, x0, margins=True)
    j = 0
    n0 = int(r["trace"][j][0])
    pm = r["pow_margin"][j]
    assert np.all(pm[:n0 - 1] > 0) and (n0 == p["pow_jmax"] or pm[n0 - 1] <= 0)


# ---------------------------------------------------------------------------
# the checker of the GPU's stop decisions, against planted mistakes
# ---------------------------------------------------------------------------

def _free_and_replay(O, p, N, x0, trace=None, scp=None):
    r = O.solve(p, N, x0)
    tr = r["trace"].copy() if trace is None else trace
    J = r["scp_iters"] if scp is None else scp
    full = np.zeros((max(p["scp_jmax"], J), 2), np.int32)
    full[:J] = tr[:J]
    rr = O.solve(p, N, x0, trace=full, replay_scp=J, margins=True)
    return r, rr, full, J


@pytest.fixture(scope="module")
def loose(inputs):
    """PIPG tolerance 1e-4: most subproblems at N = 10 stop on their test
    before the iteration cap, so the PIPG decisions carry information."""
    return inputs.load_params(pipg_eps_rel=1e-4, pipg_eps_abs=1e-8)


def test_checker_accepts_the_oracles_own_decisions(oracle, inputs, loose):
    p = loose
    x0 = inputs.dispersion(p, 4, 5, "bj")
    total = early = 0
    for b in range(4):
        r, rr, tr, J = _free_and_replay(oracle, p, 10, x0[b])
        assert r["status"] == 0
        n, border = check_stop_decisions(p, rr, tr, J, r["status"])
        assert border == 0
        total += n
        early += int(np.sum(tr[:J, 1] < p["pipg_jmax"]))
    assert total > 200 and early >= 4


def _first_early(p, tr, J):
    for j in range(J):
        if tr[j, 1] < p["pipg_jmax"] and tr[j, 1] > p["pipg_jcheck"]:
            return j
    raise AssertionError("no PIPG loop stopped on its test")


@pytest.mark.parametrize("plant", ["pipg_early", "pipg_late", "power", "scp_early", "status"])
def test_checker_catches_planted_stop_mistakes(oracle, inputs, loose, plant):
    """A stop test that fires a check early or late, a power iteration that
    stops one iteration early, an SCP loop that stops one iteration early, and
    a converged run reported as not converged: each is caught."""
    p = loose
    x0 = inputs.dispersion(p, 1, 5, "bj")[0]
    r = oracle.solve(p, 10, x0)
    tr = r["trace"].copy()
    J, status = r["scp_iters"], r["status"]
    assert status == 0 and J > 2
    if plant == "pipg_early":
        j = _first_early(p, tr, J)
        tr[j, 1] -= p["pipg_jcheck"]
    elif plant == "pipg_late":
        j = _first_early(p, tr, J)
        tr[j, 1] += p["pipg_jcheck"]
    elif plant == "power":
        assert tr[1, 0] > 1
        tr[1, 0] -= 1
    elif plant == "scp_early":
        J -= 1
    else:
        status = 1
    _, rr, full, J = _free_and_replay(oracle, p, 10, x0, trace=tr, scp=J)
    with pytest.raises(AssertionError, match="oracle's test"):
        check_stop_decisions(p, rr, full, J, status)


# ---------------------------------------------------------------------------
# touchdown error
# ---------------------------------------------------------------------------

def _landing_on_target(O, p, N, x0):
    """A trajectory whose last interval's RK4 flow lands on z_f on every
    component E_f fixes: the guess with x_{N-1} corrected by minimum-norm
    Gauss-Newton steps, the Jacobian of the flow being the STM A_{N-1}."""
    X, U = O.init_guess(p, N, x0)
    fx = np.asarray(p["fix_f"][:X.shape[1]]).astype(bool)
    zf = np.asarray(p["z_f"][:X.shape[1]])
    for _ in range(30):
        A, Bm, Bp, xp = O.discretize(p, X, U)
        res = (xp[-1] - zf)[fx]
        if np.abs(res).max() < 1e-14:
            break
        X[-2] -= np.linalg.lstsq(A[-1][fx], res, rcond=None)[0]
    return X, U, fx


@pytest.mark.parametrize("model,nu", [("6dof", 4), ("6dof", 7), ("3dof", 4)])
def test_touchdown_zero_on_target_and_quadratic_off_it(oracle, inputs, model, nu):
    """On a trajectory whose last interval lands on z_f the touchdown error is
    zero; moving x_{N-1} by h d changes it by 0.5 h^2 ||S A_{N-1} d||^2 + O(h^3)
    with S = diag(1 / P_x) on the fixed components (the error's Hessian in
    x_{N-1}, since the residual is zero)."""
    p = inputs.load_params(model=model, nu=nu)
    N = 6
    x0 = inputs.dispersion(p, 1, 4, "bj")[0]
    X, U, fx = _landing_on_target(oracle, p, N, x0)
    assert oracle.touchdown(p, X, U) < 1e-26
    A = oracle.discretize(p, X, U)[0][-1]
    Px = np.asarray(p["P_x"][:X.shape[1]])
    rng = np.random.default_rng(0)
    d = rng.normal(size=X.shape[1])
    want = 0.5 * np.sum(((A @ d)[fx] / Px[fx]) ** 2)
    for h in (1e-3, 1e-4):
        Xh = X.copy()
        Xh[-2] += h * d
        assert abs(oracle.touchdown(p, Xh, U) / h ** 2 - want) <= 20 * h * want
    # nothing but x_{N-1}, u_{N-1} and u_N enters
    Xo = X.copy(); Uo = U.copy()
    Xo[:-2] += 0.1; Uo[:-2] += 0.1; Xo[-1] += 0.1
    assert oracle.touchdown(p, Xo, Uo) < 1e-26


def test_touchdown_two_nodes_by_hand(oracle, inputs):
    """N = 2: one interval of unit length in tau; the error is the hand sum
    over the fixed components of the flow's scaled miss."""
    p = inputs.load_params()
    x0 = inputs.dispersion(p, 1, 6, "bj")[0]
    X, U = oracle.init_guess(p, 2, x0)
    xp = oracle.flow(p, X[0], U[0], U[1], p["rk4_substeps"])
    want = sum(0.5 * ((xp[i] - p["z_f"][i]) / p["P_x"][i]) ** 2 for i in range(15) if p["fix_f"][i])
    assert abs(oracle.touchdown(p, X, U) - want) <= 1e-13 * want


# ---------------------------------------------------------------------------
# initial guess (reading R9)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nu", [4, 7])
def test_initial_guess_6dof(oracle, inputs, nu):
    p = inputs.load_params(nu=nu)
    N = 7
    x0 = inputs.dispersion(p, 1, 8, "bj")[0]
    X, U = oracle.init_guess(p, N, x0)
    zf = p["z_f"]
    np.testing.assert_array_equal(X[0, :14], x0)
    for sl in (slice(1, 4), slice(4, 7), slice(11, 14)):
        np.testing.assert_allclose(X[-1, sl], zf[sl], atol=1e-15)
        np.testing.assert_allclose(X[3, sl], 0.5 * (x0[sl] + zf[sl]), atol=1e-14)  # straight lines
        np.testing.assert_allclose(np.diff(X[:, sl], 2, axis=0), 0, atol=1e-14)
    assert abs(X[-1, 0] - 0.5 * (x0[0] + p["m_dry"])) < 1e-15
    np.testing.assert_allclose(np.diff(X[:, 0], 2), 0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(X[:, 7:11], axis=1), 1.0, atol=1e-15)
    qf = zf[7:11] * np.sign(np.dot(x0[7:11], zf[7:11]))
    np.testing.assert_allclose(X[-1, 7:11], qf, atol=1e-15)
    mid = x0[7:11] + qf
    np.testing.assert_allclose(X[3, 7:11], mid / np.linalg.norm(mid), atol=1e-15)
    assert np.all(X[:, 14] == 0)
    g0 = np.linalg.norm(p["g_I"])
    np.testing.assert_allclose(U[:, 0], X[:, 0] * g0, rtol=1e-15)  # hover thrust along body x
    assert np.all(U[:, 1:nu - 1] == 0) and np.all(U[:, -1] == p["tf_guess"])


def test_initial_guess_3dof(oracle, inputs):
    p = inputs.load_params(model="3dof")
    N = 5
    x0 = inputs.dispersion(p, 1, 8, "bj")[0]
    X, U = oracle.init_guess(p, N, x0)
    np.testing.assert_array_equal(X[0, :7], x0)
    np.testing.assert_allclose(X[-1, 1:7], p["z_f"][1:7], atol=1e-15)
    np.testing.assert_allclose(X[2, 1:7], 0.5 * (x0[1:7] + p["z_f"][1:7]), atol=1e-14)
    assert abs(X[-1, 0] - 0.5 * (x0[0] + p["m_dry"])) < 1e-15
    assert np.all(X[:, 7] == 0)
    np.testing.assert_allclose(U[:, 0], X[:, 0] * np.linalg.norm(p["g_I"]), rtol=1e-15)
    assert np.all(U[:, 1:3] == 0) and np.all(U[:, 3] == p["tf_guess"])
