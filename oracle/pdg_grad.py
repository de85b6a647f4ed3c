"""FP64 reference gradient of the last SCP iteration -- TEST INFRASTRUCTURE ONLY.

Only the test suite may import this module.  It gives an independent value of
the gradient that the CUDA solver's adjoint computes (pdg_mc_grad_batch): the
derivative, with respect to the initial condition x0, of the fuel m_1 - m_N
and of the touchdown error of the trajectory that the last SCP iteration
produces, the reference's first node moving with x0 (x_bar_1 = x0) and the
rest of the reference held.

The CUDA adjoint unrolls the PIPG_custom loop in reverse.  This module instead
solves the subproblem of Eq. cvx-subproblem-custom exactly and differentiates
its solution by the implicit function theorem:

1. Exact subproblem solution.  A PIPG_custom run (Alg. PIPG_custom) shows the
   active set: the bounds that hold with equality (the fixed boundary
   components, the dilation box, mu >= 0; Eq. parsed-data's projection set)
   and the CTCS rows with a positive multiplier theta.  On that active set the
   QP min 1/2 z'Pz + p'z s.t. G z = g, H_A z = h_A, z_B = bound is an
   equality-constrained QP, solved through its KKT system (a dense linear
   solve); an active CTCS row that the dynamics rows already imply is left out
   of that system (see exact_qp).  The solution is accepted only if it satisfies every KKT condition
   of the full QP: bounds and the inactive CTCS rows hold, theta_A >= 0, and
   the gradient P z + p + G'eta + H'theta lies in the box's normal cone
   (>= 0 at a lower bound, <= 0 at an upper one, 0 where free).
2. Sensitivity.  x0 enters the subproblem only through the first interval:
   hat A^-_1, hat B^-_1, hat B^+_1 and hat w_1 of the discretization (Sec.
   2.3.1) and the prescaling (Sec. 2.3.2) about x_bar_1 = x0 (hat z_i is then
   zero whatever x0 is).  Their derivatives come from central differences of
   the oracle's discretization and scaling (the STM itself is pinned against
   differences of the RK4 flow).  With the active set fixed, differentiating
   the KKT system gives K [dz_F; d eta; d theta_A] = -[dG_F' eta;
   dG z - dg; 0], one right-hand side per component of x0.
3. Outputs.  fuel = x0_m - (X_bar_N,m + P_m z_N,m); the touchdown error is
   1/2 sum over the components E_f fixes of ((x_prop,N - z_f) / P_x)^2 with
   x_prop,N the RK4 flow of the updated last interval, whose derivative is the
   STM (A, B^-, B^+) of that interval.

The exact solution differs from the solver's (the last PIPG loop stops after
a finite count from a warm start), so the unrolled and the implicit gradients
agree only as far as that loop has converged.
"""
from __future__ import annotations

import numpy as np

from . import pdg_oracle as O


def _qp_at(p, x0, X, U):
    """Scaled subproblem about (X, U) with the reference's first node at x0."""
    X = X.copy()
    X[0, :len(x0)] = x0
    A, Bm, Bp, xp = O.discretize(p, X, U)
    return X, O.scale(p, x0, X, U, A, Bm, Bp, xp)


def exact_qp(p, qp, guess: "O.PDState", tol: float = 1e-9, active=None):
    """Exact solution of the scaled subproblem on the active set that `guess`
    (a PIPG_custom solution) shows, or on `active` = (lower, upper, rows)
    when given.  Returns a dict with z (packed as orc_z_pack), eta (dynamics
    multipliers), theta (CTCS multipliers), the active set and the dense QP,
    and `kkt`, the largest violation of the full QP's KKT conditions."""
    D = O.qp_dense(qp)
    P, pv, G, g, H, h, lo, hi = (D[k] for k in ("P", "p", "G", "g", "H", "h", "lo", "hi"))
    nz = len(pv)
    fixed = lo == hi
    if active is None:
        z0 = O.z_pack(qp, guess)
        at_lo = ~fixed & (z0 - lo <= tol)
        at_hi = ~fixed & (hi - z0 <= tol)
        rows = np.asarray(guess.th) > tol
        active = (fixed | at_lo, at_hi & ~at_lo, rows)
    at_lo, at_hi, rows = active
    bound = at_lo | at_hi
    zB = np.where(at_hi, hi, lo)[bound]
    F = ~bound
    # An active CTCS row can be implied by the dynamics rows: on an interval
    # where no path constraint is violated, the CTCS integrand and its
    # derivatives vanish, so the y row of the dynamics fixes y_{k+1} - y_k by
    # itself.  Such a row changes neither the solution nor its derivative, but
    # would make K singular (its multiplier is not unique); it is left out.
    rows = rows.copy()
    base = G[:, F]
    rank = np.linalg.matrix_rank(base)
    for r in np.nonzero(rows)[0]:
        trial = np.vstack([base, H[r, F]])
        if np.linalg.matrix_rank(trial) > rank:
            base, rank = trial, rank + 1
        else:
            rows[r] = False
    active = (at_lo, at_hi, rows)
    HA = H[rows]
    nF, ng, na = int(F.sum()), G.shape[0], int(rows.sum())
    K = np.zeros((nF + ng + na, nF + ng + na))
    K[:nF, :nF] = P[np.ix_(F, F)]
    K[:nF, nF:nF + ng] = G[:, F].T
    K[:nF, nF + ng:] = HA[:, F].T
    K[nF:nF + ng, :nF] = G[:, F]
    K[nF + ng:, :nF] = HA[:, F]
    rhs = np.concatenate([-pv[F] - P[np.ix_(F, bound)] @ zB, g - G[:, bound] @ zB, h[rows] - HA[:, bound] @ zB])
    sol = np.linalg.solve(K, rhs)
    z = np.empty(nz)
    z[F] = sol[:nF]
    z[bound] = zB
    eta = sol[nF:nF + ng]
    theta = np.zeros(H.shape[0])
    theta[rows] = sol[nF + ng:]
    grad = P @ z + pv + G.T @ eta + H.T @ theta
    viol = [np.abs(G @ z - g).max(),
            max(0.0, (H @ z - h).max()),
            max(0.0, (lo - z).max()), max(0.0, (z - hi).max()),
            max(0.0, -theta.min()),
            np.abs(theta * (H @ z - h)).max(),
            np.abs(grad[F]).max() if nF else 0.0,
            max(0.0, -grad[at_lo & ~fixed].min()) if np.any(at_lo & ~fixed) else 0.0,
            max(0.0, grad[at_hi].max()) if np.any(at_hi) else 0.0]
    return dict(z=z, eta=eta, theta=theta, active=active, K=K, F=F, bound=bound, D=D, kkt=max(viol))


def _outputs(p, x0, X, U, z, N, nu, NX):
    """fuel and touchdown error of the reference updated by the packed step z."""
    Xn = X.copy(); Un = U.copy()
    Xn[0, :len(x0)] = x0
    Xn += z[:N * NX].reshape(N, NX) * np.asarray(p["P_x"][:NX])
    Un += z[N * NX:N * (NX + nu)].reshape(N, nu) * np.asarray(p["P_u"][:nu])
    return Xn[0, 0] - Xn[-1, 0], O.touchdown(p, Xn, Un), Xn, Un


def last_iteration_exact(p, x0, X, U, guess, active=None):
    """The last SCP iteration with its subproblem solved exactly: returns
    (fuel, touchdown error, exact-QP record)."""
    N, nu, NX = X.shape[0], int(p["nu"]), O.nx_of(p)
    Xr, qp = _qp_at(p, x0, X, U)
    e = exact_qp(p, qp, guess, active=active)
    fuel, touch, _, _ = _outputs(p, x0, Xr, U, e["z"], N, nu, NX)
    return fuel, touch, e


def grad_ift(p, x0, X, U, guess, h: float = 1e-6):
    """d(fuel, touchdown)/d x0 of the last SCP iteration with the exact
    subproblem solution, by the implicit function theorem (module docstring).
    X, U: the last iteration's reference; guess: a PIPG_custom solution of
    its subproblem, which fixes the active set.  Returns (grad [NX-1][2],
    exact-QP record); the record's kkt must be small for the result to hold."""
    N, nu, NX = X.shape[0], int(p["nu"]), O.nx_of(p)
    x0 = np.asarray(x0, np.float64)
    d = len(x0)
    Xr, qp = _qp_at(p, x0, X, U)
    e = exact_qp(p, qp, guess)
    D, F, z, eta = e["D"], e["F"], e["z"], e["eta"]
    nF, ng = int(F.sum()), D["G"].shape[0]
    R = np.zeros((e["K"].shape[0], d))
    for j in range(d):
        dx = np.zeros(d); dx[j] = h
        Dp = O.qp_dense(_qp_at(p, x0 + dx, X, U)[1])
        Dm = O.qp_dense(_qp_at(p, x0 - dx, X, U)[1])
        dG = (Dp["G"] - Dm["G"]) / (2 * h)
        dg = (Dp["g"] - Dm["g"]) / (2 * h)
        assert np.all(Dp["lo"] == D["lo"]) and np.all(Dp["hi"] == D["hi"]) and np.all(Dp["H"] == D["H"])
        R[:nF, j] = -(dG[:, F].T @ eta)
        R[nF:nF + ng, j] = -(dG @ z - dg)
    S = np.linalg.solve(e["K"], R)
    dz = np.zeros((len(z), d))
    dz[F] = S[:nF]
    fuel, touch, Xn, Un = _outputs(p, x0, Xr, U, z, N, nu, NX)
    Px, Pu = np.asarray(p["P_x"][:NX]), np.asarray(p["P_u"][:nu])
    g = np.zeros((d, 2))
    # fuel = x0_m - (X_bar_N,m + P_m z_N,m)
    g[0, 0] = 1.0
    g[:, 0] -= Px[0] * dz[(N - 1) * NX + 0]
    # touchdown: the residual of the last interval's flow, through its STM
    A, Bm, Bp, xp = O.discretize(p, Xn, Un)
    fx = np.asarray(p["fix_f"][:NX]).astype(bool)
    res = np.where(fx, (xp[-1] - np.asarray(p["z_f"][:NX])) / Px ** 2, 0.0)
    dxN1 = Px[:, None] * dz[(N - 2) * NX:(N - 1) * NX]
    duN1 = Pu[:, None] * dz[N * NX + (N - 2) * nu:N * NX + (N - 1) * nu]
    duN = Pu[:, None] * dz[N * NX + (N - 1) * nu:N * NX + N * nu]
    dxp = A[-1] @ dxN1 + Bm[-1] @ duN1 + Bp[-1] @ duN
    if N == 2:  # the last interval starts at the first node, which moves with x0 itself
        dxp += A[-1][:, :d]
    g[:, 1] = res @ dxp
    return g, e
