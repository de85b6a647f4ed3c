"""Autotuner for the launch shape of the batched solver.

For one (device, n_max, nu, precision, execution form) the library's
pdg_mc_autotune times a solve of a seeded batch at every candidate (PIPG
layout, CTA size) pair -- the shared-memory PIPG form at 128..512 threads, the
register forms 2 and 3 from the threads they need up to their limits,
candidates that do not fit skipped -- and keeps the fastest by converged solves per second; this
module records the choice in a JSON cache keyed by
"device|n_max|nu|precision|mode".  Solver(tune_cache=...) applies a cached
choice through pdg_mc_set_pipg_form and pdg_mc_set_threads.  candidates()
lists the pairs that fit, for tests and reports.  Keys of models other than
the 6-DoF one end in "|<model>" (e.g. "|3dof").

  python -m paper_2404_18034_gb300.autotune --nodes 15 --precision fp64 --batch 2048
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Dict, Iterable, Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "autotune_cache.json")
NXS = {"6dof": 15, "3dof": 8}
NNZA = {"6dof": 110, "3dof": 24}  # structural nonzeros of the interval STM
SMEM_MAX = 232448


def cache_key(device_name: str, n_max: int, nu: int, precision: int, mode: int, model: str = "6dof") -> str:
    k = f"{device_name}|{n_max}|{nu}|{'fp64' if precision == 0 else 'fp32'}|{'persistent' if mode == 1 else 'plain'}"
    return k if model == "6dof" else f"{k}|{model}"


def load_cache(path: str = DEFAULT_CACHE) -> Dict:
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def lookup(device_name: str, n_max: int, nu: int, precision: int, mode: int,
           path: str = DEFAULT_CACHE, model: str = "6dof") -> Optional[Tuple[int, int]]:
    """(threads, PIPG form) of a cached choice, or None.  Entries written
    before the register form existed carry no form: they are form 1."""
    e = load_cache(path).get(cache_key(device_name, n_max, nu, precision, mode, model))
    return (int(e["threads"]), int(e.get("form", 1))) if e else None


def round32(x: int) -> int:
    return (x + 31) // 32 * 32


def reg_threads(n_max: int, nu: int, model: str = "6dof") -> int:
    """Threads the register PIPG form needs (one per dual row, whole warps,
    plus 4 or 8 lanes per node for the controls)."""
    return round32((n_max - 1) * NXS[model]) + round32(n_max * (4 if nu <= 4 else 8))


def ks_threads(n_max: int, model: str = "6dof") -> int:
    """Threads PIPG form 3 needs (8 lanes per node, 4 when NX <= 8, whole
    warps)."""
    return round32(n_max * (4 if NXS[model] <= 8 else 8))


def candidates(n_max: int, nu: int, precision: int, forms: Iterable[int] = (1, 2, 3),
               model: str = "6dof") -> Iterable[Tuple[int, int]]:
    """(form, CTA size) pairs with at least one discretization interval per
    wave whose shared-memory image fits on an SM (mirrors the kernel's layout
    rule); form 2 from its minimum up to 576 (FP32) or 512 threads, form 3
    from its minimum up to 512."""
    out = []
    if 1 in forms:
        out += [(1, t) for t in _fitting(range(128, 513, 32), n_max, nu, precision, model)]
    if 2 in forms:
        hi = 576 if precision == 1 else 512
        out += [(2, t) for t in _fitting(range(reg_threads(n_max, nu, model), hi + 1, 32), n_max, nu, precision,
                                         model)]
    if 3 in forms:
        out += [(3, t) for t in _fitting(range(ks_threads(n_max, model), 513, 32), n_max, nu, precision, model)]
    return out


def _fitting(ts: Iterable[int], n_max: int, nu: int, precision: int, model: str = "6dof") -> Iterable[int]:
    NX = NXS[model]
    sa = {"6dof": 42, "3dof": 12}[model]
    ncol = NX + 2 * nu
    esz = 8 if precision == 0 else 4
    for t in ts:
        ipw = min(32, (t - 32) // ncol)
        if ipw < 1:
            continue
        n = n_max
        sas = (NNZA[model] + 1) | 1  # compact hat A^-: nonzeros, a zero, odd count
        img = 8 + 16 + n * NX + n * nu + (n - 1) * (sas + 2 * ((NX * nu) | 1) + NX + 1) + 2 * n + 2 * NX + \
            n * NX + n * nu + 3 * (n - 1) * NX + (n - 1)
        uni = max(2 * n * NX + 2 * n * nu + 4 * (n - 1) * NX + (n - 1), ipw * (2 * (sa + NX * nu) + 3 * NX))
        if (img + uni + 210) * esz > SMEM_MAX:
            continue
        yield t


def autotune(params: Dict, n_max: int, precision: int = 0, mode: int = 1, batch: int = 2048, seed: int = 7,
             path: str = DEFAULT_CACHE) -> Dict:
    """Run the library's autotuner (pdg_mc_autotune: every (PIPG form, CTA
    size) candidate timed on a seeded batch) and record its choice."""
    import torch

    from . import inputs
    from .pdg_mc import Solver
    dev = torch.device("cuda")
    name = torch.cuda.get_device_name(dev)
    x0 = torch.from_numpy(inputs.dispersion(params, batch, seed, "bj")).to(dev)
    S = Solver(params, n_max, precision)
    threads, form, rate = S.autotune(x0, None, mode)
    S.close()
    entry = {"threads": int(threads), "form": int(form), "solves_per_s": float(rate), "batch": batch}
    cache = load_cache(path)
    cache[cache_key(name, n_max, int(params["nu"]), precision, mode, params.get("model", "6dof"))] = entry
    with open(path, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    return entry


def main():
    from . import inputs
    ap = argparse.ArgumentParser()
    ap.add_argument("--nodes", type=int, nargs="+", default=[15])
    ap.add_argument("--precision", nargs="+", default=["fp64"], choices=["fp64", "fp32"])
    ap.add_argument("--mode", nargs="+", default=["persistent"], choices=["persistent", "plain"])
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--nu", type=int, default=4)
    ap.add_argument("--model", default="6dof", choices=["6dof", "3dof"])
    ap.add_argument("--cache", default=DEFAULT_CACHE)
    a = ap.parse_args()
    p = inputs.load_params(nu=a.nu, model=a.model)
    for n in a.nodes:
        for pr in a.precision:
            for m in a.mode:
                e = autotune(p, n, 0 if pr == "fp64" else 1, 1 if m == "persistent" else 0, a.batch, path=a.cache)
                print(json.dumps({"nodes": n, "precision": pr, "mode": m, **e}))


if __name__ == "__main__":
    main()
