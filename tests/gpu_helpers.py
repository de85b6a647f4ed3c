"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

# FP64 parity tolerance: |a - b| <= RTOL * max(|b|, scale) with scale the
# component's characteristic magnitude (its P_x / P_u entry).
RTOL = 1e-6


def assert_scaled_close(a, b, scale, rtol=RTOL, what=""):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    tol = rtol * np.maximum(np.abs(b), scale)
    err = np.abs(a - b)
    bad = ~(err <= tol)  # NaN anywhere counts as a mismatch
    assert not bad.any(), f"{what}: max err {err.max():.3e}, worst ratio {(err / tol).max():.3e} at {np.argwhere(bad)[:5]}"


def replay_instance(O, p, x0, N, trace, scp_iters):
    """Oracle solve of one instance forced to the GPU's recorded counts."""
    tr = np.zeros((max(int(p["scp_jmax"]), scp_iters), 2), np.int32)
    tr[:scp_iters] = trace[:scp_iters]
    return O.solve(p, N, x0, trace=tr, replay_scp=scp_iters)
