"""The per-instance shared-memory layouts hold every region the kernels
index (tests/layout_probe.cu, compiled on the host with the solver's own
headers), for both models, every node count up to 32, both control sizes
and every CTA size the library accepts."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2404_18034_gb300", "csrc")


@pytest.mark.parametrize("defs", [[], ["-DPDG_MODEL_3DOF"]], ids=["6dof", "3dof"])
def test_layouts_hold_what_the_kernels_index(tmp_path, defs):
    nvcc = os.environ.get("NVCC", shutil.which("nvcc") or "nvcc")
    if not shutil.which(nvcc) and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "layout_probe")
    subprocess.check_call([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", SRC,
                           "-I", os.path.join(ROOT, "include")] + defs +
                          [os.path.join(ROOT, "tests", "layout_probe.cu"), "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout
    assert int(r.stdout.split()[1]) > 500
