"""The C-ABI library builds, loads and exports every entry point that
include/pdg_mc.h declares; argument errors come back as codes (no GPU work)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_18034_gb300 import build, pdg_mc
    build.build()
    return pdg_mc.load_library()


def test_exports_match_header(lib):
    hdr = open(os.path.join(ROOT, "include", "pdg_mc.h")).read()
    declared = set(re.findall(r"\b(pdg_mc_\w+)\s*\(", hdr))
    from paper_2404_18034_gb300 import pdg_mc
    assert declared == set(pdg_mc.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_param_struct_layout_matches_header(lib):
    from paper_2404_18034_gb300 import pdg_mc
    hdr = open(os.path.join(ROOT, "include", "pdg_mc.h")).read()
    body = hdr[hdr.index("typedef struct pdg_params {"):hdr.index("} pdg_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for line in body.splitlines()[1:]:
        line = line.strip().rstrip(";")
        if not line:
            continue
        for part in line.split(None, 1)[1].split(","):
            names.append(part.strip().split("[")[0])
    assert names == [f[0] for f in pdg_mc.PdgParams._fields_]


def test_init_rejects_bad_arguments(lib, params):
    from paper_2404_18034_gb300 import pdg_mc
    h = C.c_void_p()
    p = pdg_mc.make_params(params)
    assert lib.pdg_mc_init(C.byref(p), 1, C.byref(h)) == -1
    assert b"n_max" in lib.pdg_mc_last_error(None)
    p.nu = 5
    assert lib.pdg_mc_init(C.byref(p), 10, C.byref(h)) == -1
    assert b"nu" in lib.pdg_mc_last_error(None)
    p = pdg_mc.make_params(params)
    p.P_x[3] = 0.0
    assert lib.pdg_mc_init(C.byref(p), 10, C.byref(h)) == -1
    assert lib.pdg_mc_solve_batch(None, 1, None, None, 1, *([None] * 9)) == -1


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2404_18034_gb300 import pdg_mc
    with pytest.raises(RuntimeError, match="not built"):
        pdg_mc.load_library(str(tmp_path / "missing.so"))


def test_3dof_library_exports_and_checks(lib, inputs):
    """The 3-DoF model's library exports the same entry points, reports its
    state size, and rejects nu = 7 (the model has no RCS torque) and a
    non-positive P_x entry among its 8 states; the binding refuses to load a
    library under the wrong model."""
    from paper_2404_18034_gb300 import pdg_mc
    L3 = pdg_mc.load_library(model="3dof")
    assert lib.pdg_mc_model_nx() == 15 and L3.pdg_mc_model_nx() == 8
    for name in pdg_mc.EXPORTS:
        assert hasattr(L3, name), name
    p3 = inputs.load_params(model="3dof")
    h = C.c_void_p()
    p = pdg_mc.make_params(p3)
    p.nu = 7
    assert L3.pdg_mc_init(C.byref(p), 10, C.byref(h)) == -1
    assert b"nu must be 4" in L3.pdg_mc_last_error(None)
    p = pdg_mc.make_params(p3)
    p.P_x[7] = 0.0
    assert L3.pdg_mc_init(C.byref(p), 10, C.byref(h)) == -1
    assert b"P_x" in L3.pdg_mc_last_error(None)
    with pytest.raises(RuntimeError, match="not the 3dof model"):
        pdg_mc.load_library(pdg_mc.LIB_PATHS["6dof"], model="3dof")
