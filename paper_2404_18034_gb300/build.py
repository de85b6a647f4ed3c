"""Build the CUDA libraries in-tree for sm_103a (GB300) with nvcc.

One library per model of the problem template (the model is a compile-time
choice of csrc/pdg_device.cuh): libpdg_mc.so holds the 6-DoF model of Sec. 4,
libpdg_mc_3dof.so the translational 3-DoF model.  Both compile from the same
sources, in parallel.  build_model() compiles a library for a model header of
the caller's (the interface is listed in csrc/pdg_device.cuh).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpdg_mc.so")
LIBS = {"6dof": LIB, "3dof": os.path.join(HERE, "libpdg_mc_3dof.so")}
DEFS = {"6dof": [], "3dof": ["-DPDG_MODEL_3DOF"]}
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
GENCODE = "arch=compute_103a,code=sm_103a"


def _sources():
    return [os.path.join(SRC, f) for f in sorted(os.listdir(SRC)) if f.endswith((".cu", ".cuh"))] + \
        [os.path.join(INCLUDE, "pdg_mc.h")]


def _stale(path: str) -> bool:
    if not os.path.exists(path):
        return True
    return os.path.getmtime(path) < max(os.path.getmtime(p) for p in _sources())


def build(force: bool = False, verbose: bool = False, models=("6dof", "3dof")) -> str:
    """Compile csrc/pdg_mc.cu into one library per model (in parallel);
    returns the 6-DoF library's path."""
    nvcc = os.environ.get("NVCC", "nvcc")
    procs = []
    for m in models:
        out = LIBS[m]
        if not force and not _stale(out):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc, "-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
               "-I", INCLUDE] + DEFS[m] + [os.path.join(SRC, "pdg_mc.cu"), "-o", tmp]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((subprocess.Popen(cmd), tmp, out, cmd))
    failed = []
    for p, tmp, out, cmd in procs:
        if p.wait() != 0:
            failed.append(" ".join(cmd))
        else:
            os.replace(tmp, out)
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    return LIB


def build_model(header: str, out: str, force: bool = False) -> str:
    """Compile the solver for the model in `header` (passed to the device code
    as PDG_MODEL_HEADER) into the library `out`; returns `out`.  The header may
    include the solver's own headers by name (csrc is on the include path)."""
    header = os.path.abspath(header)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            [os.path.getmtime(header)] + [os.path.getmtime(p) for p in _sources()]):
        return out
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc, "-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", INCLUDE, "-I", SRC, f'-DPDG_MODEL_HEADER="{header}"', os.path.join(SRC, "pdg_mc.cu"), "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
