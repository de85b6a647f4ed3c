"""The structural sparsity that each built-in model declares for its interval
state-transition matrices (model_stm_row_mask, read by the PIPG products to
skip zeros) against the oracle: over random references that violate every
path constraint, random inertias and thrust points, both control sizes and
the glide slope on and off, every entry of the oracle's A_k outside the mask
is exactly zero, and every entry inside it is nonzero somewhere.  The mask is
printed by tests/stm_probe.cu, compiled on the host with the solver's own
headers."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2404_18034_gb300", "csrc")


def _probe(tmp_path, defs):
    nvcc = os.environ.get("NVCC", shutil.which("nvcc") or "nvcc")
    if not shutil.which(nvcc) and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "stm_probe")
    subprocess.check_call([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", SRC,
                           "-I", os.path.join(ROOT, "include")] + defs + [os.path.join(ROOT, "tests", "stm_probe.cu"),
                                                                         "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60, check=True).stdout.split("\n")
    nx = int(out[0].split()[1])
    mask = np.zeros((nx, nx), bool)
    order, offs, compact = [], [], None
    for line in out[1:]:
        f = line.split()
        if f and f[0] == "mask":
            i, m = int(f[1]), int(f[2])
            mask[i] = [(m >> c) & 1 for c in range(nx)]
        elif f and f[0] == "order":  # a, row_order[a], col_order[a], nnz of row a, of column a, their lists
            order.append([int(v) for v in f[2:]])
        elif f and f[0] == "compact":
            compact = (int(f[1]), int(f[2]))
        elif f and f[0] == "offsets":  # a, row_start[a], row_off[a][0..1], col_off[a][0..1]
            offs.append([int(v) for v in f[2:]])
    return mask, order, compact, offs


def _sampled_pattern(O, inputs, model, nx, trials=24):
    seen = np.zeros((nx, nx), bool)
    rng = np.random.default_rng(7)
    for nu, gs in ([(4, 0), (7, 0), (4, 1), (7, 1)] if model == "6dof" else [(4, 0), (4, 1)]):
        for t in range(trials):
            J = rng.uniform(0.05, 0.4, 3)
            p = inputs.load_params(model=model, nu=nu, glide_slope=gs, J_B=J, r_T_B=rng.normal(size=3) * 0.3)
            x0 = inputs.dispersion(p, 1, t, "bj")[0]
            X, U = O.init_guess(p, 6, x0)
            X[1:] += rng.normal(size=X[1:].shape) * 0.5 * p["P_x"][:nx]   # off the guess: g rows violated
            X[:, 0] = np.abs(X[:, 0]) + 0.5
            U += rng.normal(size=U.shape) * 1.5 * p["P_u"][:nu]
            U[:, -1] = np.abs(U[:, -1]) + 1.0
            A = O.discretize(p, X, U)[0]
            assert np.all(np.isfinite(A))
            seen |= np.any(A != 0.0, axis=0)
    return seen


@pytest.mark.parametrize("model,defs", [("6dof", []), ("3dof", ["-DPDG_MODEL_3DOF"])])
def test_declared_stm_sparsity_matches_oracle(tmp_path, oracle, inputs, model, defs):
    mask, order, compact, offs = _probe(tmp_path, defs)
    nx = mask.shape[0]
    seen = _sampled_pattern(oracle, inputs, model, nx)
    assert not np.any(seen & ~mask), np.argwhere(seen & ~mask)   # nothing nonzero outside the mask
    np.testing.assert_array_equal(seen, mask)                     # and the mask is no looser than needed
    from paper_2404_18034_gb300 import flops
    assert flops.MODELS[model][3] == int(mask.sum())              # the roofline's count of hat A^- nonzeros
    # the visiting order: rows and columns by nonzero count, largest first;
    # index lists hold exactly the nonzeros, then a structural zero
    rows = [o[0] for o in order]
    cols = [o[1] for o in order]
    assert sorted(rows) == list(range(nx)) and sorted(cols) == list(range(nx))
    rn, cn = mask.sum(1), mask.sum(0)
    assert all(rn[rows[a]] >= rn[rows[a + 1]] for a in range(nx - 1))
    assert all(cn[cols[a]] >= cn[cols[a + 1]] for a in range(nx - 1))
    for i in range(nx):
        rl, cl = order[i][4], order[i][5]
        ridx = [(rl >> (4 * j)) & 15 for j in range(nx)]
        cidx = [(cl >> (4 * j)) & 15 for j in range(nx)]
        assert order[i][2] == rn[i] and order[i][3] == cn[i]
        assert ridx[:rn[i]] == list(np.nonzero(mask[i])[0]) and all(not mask[i, c] for c in ridx[rn[i]:])
        assert cidx[:cn[i]] == list(np.nonzero(mask[:, i])[0]) and all(not mask[r, i] for r in cidx[cn[i]:])
    # compact storage: interval k keeps its nonzeros row by row, columns
    # ascending, then a zero, padded to an odd count; every list entry's
    # offset names that nonzero, and every padding entry the zero
    nnz, sas = compact
    assert nnz == int(mask.sum()) and sas == (nnz + 1) | 1
    pos = -np.ones((nx, nx), int)
    pos[mask] = np.arange(nnz)                       # row-major order of the nonzeros
    for i in range(nx):
        rs, r0, r1, c0, c1 = offs[i]
        ro = [((r0 if j < 8 else r1) >> (8 * (j % 8))) & 255 for j in range(nx)]
        co = [((c0 if j < 8 else c1) >> (8 * (j % 8))) & 255 for j in range(nx)]
        nz_c, nz_r = np.nonzero(mask[i])[0], np.nonzero(mask[:, i])[0]
        assert rs == (pos[i, nz_c[0]] if len(nz_c) else rs)
        assert ro[:len(nz_c)] == [pos[i, c] for c in nz_c] and all(o == nnz for o in ro[len(nz_c):])
        assert co[:len(nz_r)] == [pos[r, i] for r in nz_r] and all(o == nnz for o in co[len(nz_r):])
