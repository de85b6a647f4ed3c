"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np

# FP64 parity tolerance: |a - b| <= RTOL * max(|b|, scale) with scale the
# component's characteristic magnitude (its P_x / P_u entry).
RTOL = 1e-6

# Stop decisions whose oracle margin (a - b) / b of the test a <= b lies
# within this band of zero are borderline: the two sides compute the tested
# quantities from iterates that differ by rounding, and a PIPG stop test
# compares a difference of consecutive iterates (about eps_rel |z|) against
# its threshold, so a discrepancy of 1e-12 |z| in the iterates moves its
# margin by about 1e-12 / eps_rel = 1e-6 at eps_rel = 1e-6.  1e-4 leaves a
# factor of 100 over that.
STOP_BAND = 1e-4


# FP32 tolerance: an FP32 solve against the FP64 oracle, on instances that
# converge on both sides in the same number of SCP iterations, in max |a - b| /
# max(|b|, P) over X and U and in relative t_f and fuel.  Measured on GB300
# (96 instances each): X 3.9e-5 to 6.8e-5, U 1.2e-4 to 3.4e-4, t_f and fuel
# below 2e-5, for 6-DoF at N = 15 and 30 and 3-DoF at N = 15.  The bound
# leaves a factor of about 6 over the largest.
FP32_TOL = 2e-3


def fp32_errors(p, o32, ref, idx):
    """Scaled trajectory, t_f and fuel errors of FP32 outputs o32 (numpy) against
    FP64 outputs ref on the instances idx: max over X and U of
    |a - b| / max(|b|, P), and the largest relative t_f and fuel errors."""
    nu = int(p["nu"])
    ex = max(np.max(np.abs(o32["X"][b] - ref["X"][b]) / np.maximum(np.abs(ref["X"][b]), p["P_x"])) for b in idx)
    eu = max(np.max(np.abs(o32["U"][b] - ref["U"][b]) / np.maximum(np.abs(ref["U"][b]), p["P_u"][:nu])) for b in idx)
    et = max(abs(o32["tf"][b] - ref["tf"][b]) / abs(ref["tf"][b]) for b in idx)
    ef = max(abs(o32["fuel"][b] - ref["fuel"][b]) / abs(ref["fuel"][b]) for b in idx)
    return dict(X=ex, U=eu, tf=et, fuel=ef)


def assert_scaled_close(a, b, scale, rtol=RTOL, what=""):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    tol = rtol * np.maximum(np.abs(b), scale)
    err = np.abs(a - b)
    bad = ~(err <= tol)  # NaN anywhere counts as a mismatch
    assert not bad.any(), f"{what}: max err {err.max():.3e}, worst ratio {(err / tol).max():.3e} at {np.argwhere(bad)[:5]}"


def replay_instance(O, p, x0, N, trace, scp_iters):
    """Oracle solve of one instance forced to the GPU's recorded counts, with
    the oracle's own stop-test margins at every point where a free-running
    solver evaluates its tests (see check_stop_decisions)."""
    tr = np.zeros((max(int(p["scp_jmax"]), scp_iters), 2), np.int32)
    tr[:scp_iters] = trace[:scp_iters]
    return O.solve(p, N, x0, trace=tr, replay_scp=scp_iters, margins=True)


def check_stop_decisions(p, r, trace, scp_iters, status, band=STOP_BAND, what=""):
    """The GPU's stop decisions against the oracle's own tests on the replayed
    iterates.  The GPU ran `trace[j] = (power, PIPG)` iterations in SCP
    iteration j, `scp_iters` SCP iterations and ended with `status`; r is the
    oracle replay of those counts with margins (replay_instance).  Every test
    the GPU evaluated must have decided as the oracle's test on the same
    iterates decides:
      - Alg. power: no stop after iterations 1 .. n-1, a stop after n unless n
        is the cap pow_jmax;
      - Alg. stopping (every pipg_jcheck iterations): no stop at the checks
        before the count n, a stop at n unless n is the cap pipg_jmax;
      - the SCP convergence test: not converged after iterations 1 .. J-1,
        converged after J exactly when the status is PDG_CONVERGED.
    A disagreement whose oracle margin lies within `band` of zero is
    borderline and is counted, not failed.  Returns (decisions checked,
    borderline count)."""
    jc, jmax, pmax = int(p["pipg_jcheck"]), int(p["pipg_jmax"]), int(p["pow_jmax"])
    checked = border = 0

    def decide(margin, want_stop, where):
        nonlocal checked, border
        checked += 1
        stop = bool(margin <= 0)
        if stop == want_stop:
            return
        assert np.isfinite(margin) and abs(margin) <= band, \
            f"{what}: {where}: the GPU {'stopped' if want_stop else 'went on'} but the oracle's test " \
            f"{'did not pass' if want_stop else 'passed'} (margin {margin:.3e})"
        border += 1

    J = int(scp_iters)
    for j in range(J):
        n = int(trace[j][0])
        assert 1 <= n <= pmax, f"{what}: SCP {j}: power iterations {n}"
        m = r["pow_margin"][j]
        for i in range(1, n):
            decide(m[i - 1], False, f"SCP {j} power iteration {i}")
        if n < pmax:
            decide(m[n - 1], True, f"SCP {j} power iteration {n}")
        n = int(trace[j][1])
        assert 1 <= n <= jmax, f"{what}: SCP {j}: PIPG iterations {n}"
        assert n == jmax or n % jc == 0, f"{what}: SCP {j}: PIPG stopped at {n}, not at a check"
        m = r["pipg_margin"][j]
        for c in range(1, n // jc + 1):
            if c * jc < n:
                decide(m[c - 1], False, f"SCP {j} PIPG check {c * jc}")
            elif n < jmax:
                decide(m[c - 1], True, f"SCP {j} PIPG check {c * jc}")
        if j < J - 1:
            decide(r["scp_margin"][j], False, f"SCP test after iteration {j + 1}")
    decide(r["scp_margin"][J - 1], int(status) == 0, f"SCP test after iteration {J}")
    return checked, border
