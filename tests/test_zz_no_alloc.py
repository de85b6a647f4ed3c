"""pdg_mc_solve_batch_noalloc: the solve for callers that cannot allocate.

Some callers cannot call cudaMalloc while they run: code inside a region whose
device memory an allocator or memory pool owns, or a service that must not
grow its device footprint after start-up.  For them the library keeps the
plain-form workspace in a fixed device array and this entry point allocates
nothing.  The test calls it through the C ABI and checks it against the
regular entry point (pdg_mc_solve_batch, plain form) on two calls in a row;
the second call uses a different batch, so leftovers of the first call in the
shared array would show.  The same check also runs in a fresh child process,
where the no-allocation call comes first (before any other solve has loaded
the library's kernels), and a warmed-up call is checked to leave the device's
free memory unchanged.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_helpers import assert_scaled_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18034_gb300 import build
    build.build()
    return torch


def _batch(inputs, p, B, seed):
    x0 = inputs.dispersion(p, B, seed, "bj")
    Ns = inputs.node_counts(B, seed, (2, 10, 15))
    return x0, Ns


def _two_calls(torch, inputs, model):
    """Two no-allocation calls in a row, each before the regular solve of the
    same batch, compared with it."""
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params(model=model)
    S = Solver(p, 15)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for call, (B, seed) in enumerate([(48, 101), (29, 202)]):
        x0, Ns = _batch(inputs, p, B, seed)
        out = S.solve_noalloc(d(x0), d(Ns))
        ref = S.solve(d(x0), d(Ns), mode=0)
        torch.cuda.synchronize()
        for k in ("status", "scp_iters", "pipg_iters"):
            np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=f"{k} call {call}")
        ok = ref["status"].cpu().numpy() != 2
        assert_scaled_close(out["X"].cpu().numpy()[ok], ref["X"].cpu().numpy()[ok], p["P_x"], what=f"X call {call}")
        assert_scaled_close(out["U"].cpu().numpy()[ok], ref["U"].cpu().numpy()[ok], p["P_u"][:4], what=f"U call {call}")
        assert_scaled_close(out["tf"].cpu().numpy()[ok], ref["tf"].cpu().numpy()[ok], 1.0, what=f"tf call {call}")
        assert_scaled_close(out["fuel"].cpu().numpy()[ok], ref["fuel"].cpu().numpy()[ok], 0.5, what=f"fuel call {call}")
    S.close()


@pytest.mark.parametrize("model", ["6dof", "3dof"])
def test_noalloc_matches_regular_solve_on_two_calls(torch_cuda, inputs, model):
    _two_calls(torch_cuda, inputs, model)


def test_noalloc_in_a_fresh_process(torch_cuda):
    """The two-call check in a child process whose first solve of all is the
    no-allocation one (both models, one process each)."""
    here = os.path.dirname(os.path.abspath(__file__))
    for model in ("6dof", "3dof"):
        code = ("import sys, torch; sys.path[:0] = [%r, %r]; "
                "from paper_2404_18034_gb300 import inputs; import test_zz_no_alloc as t; "
                "t._two_calls(torch, inputs, %r); print('fresh ok')") % (here, os.path.dirname(here), model)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


def test_noalloc_leaves_free_device_memory_unchanged(torch_cuda, inputs):
    """After a first call on the device, a call changes neither the device's
    free memory (cudaMemGetInfo) nor what torch's allocator holds."""
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params()
    S = Solver(p, 15)
    x0, Ns = _batch(inputs, p, 40, 303)
    x0, Ns = torch.from_numpy(x0).cuda(), torch.from_numpy(Ns).cuda()
    out = S.alloc_outputs(40, x0.device)
    S.solve_noalloc(x0, Ns, out=out)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    S.solve_noalloc(x0, Ns, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    S.close()


def test_noalloc_rejects_batches_beyond_the_scratch(torch_cuda, inputs):
    torch = torch_cuda
    from paper_2404_18034_gb300.pdg_mc import Solver
    p = inputs.load_params()
    S = Solver(p, 15)
    x0 = torch.zeros(4000, 14, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="static scratch"):
        S.solve_noalloc(x0)
    S.close()
