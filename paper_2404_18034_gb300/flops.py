"""Algorithmic operation counts of the solver (one FMA = 2 flops), used for
the roofline fraction.  They count the operations of the method itself, not
of any particular kernel:

* PIPG_custom iteration (Alg. PIPG_custom): the products K^T (phi, theta) and
  K (2 z - z~) over the blocks hat A^-_k (15 x 15), hat B^-_k, hat B^+_k
  (15 x nu), counting in hat A^-_k only its structural nonzeros (110 of 225
  for 6-DoF: the entries that can be nonzero for some state, control and
  parameter; the others are exactly zero in every interval STM), so
  2 (N-1)(110 + 30 nu) FMA; plus the vector work per scalar variable: 9 flops
  per x_hat / u_hat entry and per mu^+ / mu^- entry (gradient assembly, step,
  projection, 2z - z~, extrapolation), 8 per phi / theta entry.  With
  dense=True the products count every entry of hat A^-_k, 2 (N-1)(225 + 30 nu)
  FMA: the count of a solver that multiplies the structural zeros too.
* power iteration (Alg. power): the same two products plus the squared norm,
  2 flops per primal entry.
* discretization (Sec. 2.3.1 by RK4): per interval, substep and stage, the
  state-transition right-hand side J S for every one of the 15 + 2 nu STM
  columns through the structural nonzeros of df/dx (62 FMA), the df/du column
  term for the 2 nu control columns (15 FMA), the RK4 stage/accumulate updates
  (3 flops per entry), and one evaluation of f and its Jacobians (250 flops).

The 3-DoF model (NX = 8) has the same structure with its own constants: 13
structural nonzeros of df/dx in the STM right-hand side, 24 of the 64 entries
of its interval STM, and about 100 flops per evaluation of f and its
Jacobians.
"""

# model: (NX, structural nonzeros of df/dx used per STM column, flops of one
# model evaluation, structural nonzeros of the interval STM hat A^-_k)
MODELS = {"6dof": (15, 62, 250, 110), "3dof": (8, 13, 100, 24)}


def _blocks(nx: int, nu: int, nnz_a: int, dense: bool) -> int:
    return (nx * nx if dense else nnz_a) + 2 * nx * nu


def pipg_iter(N: int, nu: int, model: str = "6dof", dense: bool = False) -> int:
    nx, _, _, nnz_a = MODELS[model]
    mat = 2 * 2 * (N - 1) * _blocks(nx, nu, nnz_a, dense)
    vec = 9 * (nx + nu) * N + 9 * 2 * nx * (N - 1) + 8 * (nx + 1) * (N - 1)
    return mat + vec


def power_iter(N: int, nu: int, model: str = "6dof", dense: bool = False) -> int:
    nx, _, _, nnz_a = MODELS[model]
    mat = 2 * 2 * (N - 1) * _blocks(nx, nu, nnz_a, dense)
    return mat + 2 * ((nx + nu) * N + 2 * nx * (N - 1))


def discretization(N: int, nu: int, nsub: int, model: str = "6dof") -> int:
    nx, nnz, ev, _ = MODELS[model]
    ncol = nx + 2 * nu
    per_stage = ncol * (2 * nnz + 3 * nx) + 2 * nu * 2 * nx + ev
    return (N - 1) * nsub * 4 * per_stage


def solve_flops(N, nu, nsub, scp_iters, pow_iters, pipg_iters, model: str = "6dof", dense: bool = False) -> float:
    """Total algorithmic flops of a solve given its executed counters (arrays
    over instances are accepted)."""
    import numpy as np
    N = np.asarray(N)
    return float(np.sum(np.asarray(scp_iters) * np.vectorize(discretization)(N, nu, nsub, model)
                        + np.asarray(pow_iters) * np.vectorize(power_iter)(N, nu, model, dense)
                        + np.asarray(pipg_iters) * np.vectorize(pipg_iter)(N, nu, model, dense)))
