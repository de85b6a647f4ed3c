"""Pins of the oracle's reference gradient (oracle/pdg_grad.py): the exact
subproblem solution it differentiates is a KKT point of Eq.
cvx-subproblem-custom that Alg. PIPG_custom converges to; its implicit-function
gradient equals central differences of the last SCP iteration with that
exact solution; and the gradient of the solver's own definition (the last
PIPG loop unrolled for a finite count, differentiated by central differences)
tends to it as the loop runs longer."""
import numpy as np
import pytest

from oracle import pdg_grad as G


def _last_iteration(O, p, N, seed, b=0):
    from paper_2404_18034_gb300 import inputs
    x0 = inputs.dispersion(p, b + 1, seed, "bj")[b]
    r = O.solve(p, N, x0)
    assert r["status"] == 0
    X, U, ws, sig, n = O.final_iteration_state(p, N, x0, r["trace"], r["scp_iters"])
    _, qp = G._qp_at(p, x0, X, U)
    return x0, X, U, ws, sig, n, qp


CASES = [("6dof", 4, 10, 3), ("6dof", 4, 15, 4), ("3dof", 4, 10, 3)]


@pytest.mark.parametrize("model,nu,N,seed", CASES)
def test_exact_subproblem_solution_is_the_pipg_limit(oracle, inputs, model, nu, N, seed):
    """The active-set solution satisfies every KKT condition of the full
    subproblem to rounding, and PIPG_custom run long from the solver's warm
    start reaches it."""
    p = inputs.load_params(model=model, nu=nu)
    x0, X, U, ws, sig, n, qp = _last_iteration(oracle, p, N, seed)
    guess = ws.copy()
    oracle.pipgc(p, qp, sig, guess, force_iters=20000)
    e = G.exact_qp(p, qp, guess)
    assert e["kkt"] <= 1e-12, e["kkt"]
    w = ws.copy()
    oracle.pipgc(p, qp, sig, w, force_iters=60000)
    assert np.abs(oracle.z_pack(qp, w) - e["z"]).max() <= 1e-12
    np.testing.assert_allclose(w.phi.ravel(), e["eta"], atol=1e-9)


@pytest.mark.parametrize("model,nu,N,seed", CASES)
def test_implicit_gradient_matches_differences(oracle, inputs, model, nu, N, seed):
    """grad_ift against central differences (h = 1e-6) of the last SCP
    iteration solved exactly on the same active set."""
    p = inputs.load_params(model=model, nu=nu)
    x0, X, U, ws, sig, n, qp = _last_iteration(oracle, p, N, seed)
    guess = ws.copy()
    oracle.pipgc(p, qp, sig, guess, force_iters=20000)
    g, e = G.grad_ift(p, x0, X, U, guess)
    assert e["kkt"] <= 1e-12
    h = 1e-6
    fd = np.zeros_like(g)
    for j in range(len(x0)):
        dx = np.zeros(len(x0)); dx[j] = h
        a = G.last_iteration_exact(p, x0 + dx, X, U, guess, active=e["active"])
        b = G.last_iteration_exact(p, x0 - dx, X, U, guess, active=e["active"])
        fd[j] = [(a[0] - b[0]) / (2 * h), (a[1] - b[1]) / (2 * h)]
    assert np.abs(g[:, 0] - fd[:, 0]).max() <= 1e-7 * np.abs(fd[:, 0]).max()
    assert np.abs(g[:, 1] - fd[:, 1]).max() <= 1e-14 + 1e-4 * np.abs(fd[:, 1]).max()


def test_unrolled_gradient_tends_to_the_implicit_one(oracle, inputs):
    """The solver's gradient definition differentiates the last PIPG loop
    unrolled for n iterations from its warm start; as n grows that loop
    converges to the exact solution and its derivative to the implicit one:
    the fuel gradient's relative gap shrinks from about 1e-2 at n = 2000 to
    below 1e-8 at n = 20000, the touchdown gradient's to below 1e-12."""
    p = inputs.load_params()
    N = 10
    x0, X, U, ws, sig, n, qp = _last_iteration(oracle, p, N, 3)
    guess = ws.copy()
    oracle.pipgc(p, qp, sig, guess, force_iters=20000)
    g, e = G.grad_ift(p, x0, X, U, guess)
    gaps = []
    for nn in (2000, 10000, 20000):
        h = 1e-6
        fd = np.zeros_like(g)
        for j in range(len(x0)):
            dx = np.zeros(len(x0)); dx[j] = h
            a = np.array(oracle.final_iteration_outputs(p, x0 + dx, X, U, ws, sig, nn))
            b = np.array(oracle.final_iteration_outputs(p, x0 - dx, X, U, ws, sig, nn))
            fd[j] = (a - b) / (2 * h)
        gaps.append((np.abs(fd[:, 0] - g[:, 0]).max() / np.abs(g[:, 0]).max(), np.abs(fd[:, 1] - g[:, 1]).max()))
    assert gaps[0][0] > gaps[1][0] > gaps[2][0] and gaps[2][0] < 1e-8, gaps
    assert gaps[2][1] < 1e-12, gaps
