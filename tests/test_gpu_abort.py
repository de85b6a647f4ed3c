"""Failure handling on the host side of the boundary: pdg_mc_abort.

The abort word is pinned host memory mapped into the device's address space;
kernels read it at each SCP iteration boundary and never wait on it, so an
abort is tested by setting it from the host, before a launch or while a large
batch runs, and checking that every unfinished instance ends with
PDG_ABORTED promptly.  Nothing here faults or stalls the GPU."""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18034_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("mode", [0, 1, 2, "noalloc"])
def test_abort_before_launch(torch_cuda, oracle, inputs, mode):
    """With the request set before the call, every instance stops before its
    first SCP iteration with the initial guess as its output; after
    pdg_mc_clear_abort the same handle solves normally."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import PDG_ABORTED, Solver
    p = inputs.load_params()
    S = Solver(p, 12)
    B = 24
    x0 = inputs.dispersion(p, B, 5, "bj")
    Ns = inputs.node_counts(B, 5, (4, 8, 12))
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    run = (lambda: S.solve_noalloc(d(x0), d(Ns))) if mode == "noalloc" else (lambda: S.solve(d(x0), d(Ns), mode=mode))
    S.abort()
    out = {k: v.cpu().numpy() for k, v in run().items()}
    assert np.all(out["status"] == PDG_ABORTED) and np.all(out["scp_iters"] == 0) and np.all(out["pipg_iters"] == 0)
    for b in range(B):
        X, U = oracle.init_guess(p, int(Ns[b]), x0[b])
        np.testing.assert_allclose(out["X"][b, :Ns[b]], X, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(out["U"][b, :Ns[b]], U, rtol=1e-12, atol=1e-12)
    S.clear_abort()
    out = run()
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() <= 1)
    S.close()


@pytest.mark.parametrize("mode", [1, 0])
def test_abort_while_a_large_batch_runs(torch_cuda, inputs, mode):
    """B = 16384, N = 15 takes about 8 s.  A host thread sets the request
    0.5 s after the launch: the call returns well before the full solve
    would, the instances finished by then keep their outcome, the others are
    PDG_ABORTED with fewer than scp_jmax iterations and finite outputs."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import PDG_ABORTED, Solver
    p = inputs.load_params()
    S = Solver(p, 15)
    B = 16384
    x0 = torch.from_numpy(inputs.dispersion(p, B, 7, "bj")).cuda()
    S.solve(x0[:64], mode=mode)  # loads the kernels
    torch.cuda.synchronize()
    timer = threading.Timer(0.5, S.abort)
    t0 = time.perf_counter()
    timer.start()
    out = S.solve(x0, mode=mode)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    timer.join()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    st = o["status"]
    ab = st == PDG_ABORTED
    print(f"mode {mode}: returned after {dt:.2f} s; aborted {ab.sum()}, finished {np.sum(st <= 1)}")
    assert dt < 3.0
    assert ab.sum() > B // 2 and np.all((st == PDG_ABORTED) | (st <= 1))
    assert np.all(o["scp_iters"][ab] < p["scp_jmax"])
    assert np.all(np.isfinite(o["X"][ab])) and np.all(np.isfinite(o["U"][ab]))
    np.testing.assert_allclose(o["X"][ab, 0, :14], x0.cpu().numpy()[ab], atol=1e-12)
    S.clear_abort()
    S.close()


def test_abort_gives_zero_gradients(torch_cuda, inputs):
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import PDG_ABORTED, Solver
    p = inputs.load_params()
    S = Solver(p, 10)
    x0 = torch.from_numpy(inputs.dispersion(p, 4, 9, "bj")).cuda()
    S.abort()
    g = S.grad(x0, None, torch.ones(4, dtype=torch.float64, device="cuda"), None)
    torch.cuda.synchronize()
    assert np.all(g["status"].cpu().numpy() == PDG_ABORTED)
    assert np.all(g["grad"].cpu().numpy() == 0.0)
    S.clear_abort()
    S.close()
