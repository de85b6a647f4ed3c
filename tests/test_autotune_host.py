"""Host side of the launch-shape autotuner: the candidate list (the register
PIPG forms' thread rules and the shared-memory fit), the cache keys of both
models, and the committed cache's entries."""
import json

from paper_2404_18034_gb300 import autotune as A


def test_register_form_thread_rule():
    # one thread per dual row in whole warps, plus 4 (nu = 4) or 8 (nu = 7) lanes per node
    assert A.reg_threads(15, 4) == 224 + 64
    assert A.reg_threads(30, 4) == 448 + 128
    assert A.reg_threads(15, 7) == 224 + 128
    assert A.reg_threads(15, 4, "3dof") == 128 + 64


def test_tiled_form_thread_rule():
    # 8 lanes per node (4 when NX <= 8) in whole warps
    assert A.ks_threads(15) == 128 and A.ks_threads(30) == 256 and A.ks_threads(32) == 256
    assert A.ks_threads(15, "3dof") == 64 and A.ks_threads(10, "3dof") == 64


def test_candidates_fit_and_cover_every_form():
    c6 = A.candidates(15, 4, 0)
    assert (1, 128) in c6 and (1, 512) in c6 and (2, 288) in c6
    assert all(t % 32 == 0 and 128 <= t <= 576 for _, t in c6)
    # FP64 at N = 30: the image fills most of an SM, but one CTA still fits
    assert A.candidates(30, 4, 0)
    # FP32 allows the register form up to 576 threads
    assert (2, 576) in A.candidates(15, 4, 1) and (2, 576) not in c6
    c3 = A.candidates(15, 4, 0, model="3dof")
    assert (1, 128) in c3 and (2, 192) in c3 and (2, 160) not in c3
    assert (3, 128) in c6 and (3, 96) not in c6 and (3, 512) in c6 and (3, 544) not in c6
    assert (3, 64) in c3


def test_cache_keys_and_committed_entries():
    assert A.cache_key("GPU", 15, 4, 0, 1) == "GPU|15|4|fp64|persistent"
    assert A.cache_key("GPU", 15, 4, 1, 0, "3dof") == "GPU|15|4|fp32|plain|3dof"
    cache = json.load(open(A.DEFAULT_CACHE))
    for key, e in cache.items():
        dev, n, nu, prec, mode = key.split("|")[:5]
        model = key.split("|")[5] if key.count("|") == 5 else "6dof"
        assert (e["form"], e["threads"]) in A.candidates(int(n), int(nu), 0 if prec == "fp64" else 1, model=model), key
    assert A.lookup("NVIDIA GB300", 15, 4, 0, 1, model="3dof") == (128, 1)
