"""Autotuner for the launch shape of the batched solver.

For one (device, n_max, nu, precision, form) it times a solve of a seeded
batch at every candidate CTA size (multiples of 32 that leave room for at
least one discretization interval and fit in shared memory), keeps the
fastest by converged solves per second, and records it in a JSON cache keyed
by "device|n_max|nu|precision|mode".  Solver(tune_cache=...) applies a cached
choice through pdg_mc_set_threads.

  python -m paper_2404_18034_gb300.autotune --nodes 15 --precision fp64 --batch 2048
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Dict, Iterable, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "autotune_cache.json")
NX = 15
SMEM_MAX = 232448


def cache_key(device_name: str, n_max: int, nu: int, precision: int, mode: int) -> str:
    return f"{device_name}|{n_max}|{nu}|{'fp64' if precision == 0 else 'fp32'}|{'persistent' if mode == 1 else 'plain'}"


def load_cache(path: str = DEFAULT_CACHE) -> Dict:
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def lookup(device_name: str, n_max: int, nu: int, precision: int, mode: int, path: str = DEFAULT_CACHE) -> Optional[int]:
    e = load_cache(path).get(cache_key(device_name, n_max, nu, precision, mode))
    return int(e["threads"]) if e else None


def candidates(n_max: int, nu: int, precision: int) -> Iterable[int]:
    """CTA sizes with at least one discretization interval per wave whose
    shared-memory image fits on an SM (mirrors the kernel's layout rule)."""
    ncol = NX + 2 * nu
    esz = 8 if precision == 0 else 4
    for t in range(128, 513, 32):
        ipw = min(32, (t - 32) // ncol)
        if ipw < 1:
            continue
        n = n_max
        img = 8 + 16 + n * NX + n * nu + (n - 1) * (NX * NX + 2 * NX * nu + NX + 1) + 2 * n + 2 * NX + \
            n * NX + n * nu + 3 * (n - 1) * NX + (n - 1)
        uni = max(2 * n * NX + 2 * n * nu + 4 * (n - 1) * NX + (n - 1), ipw * (40 + NX * nu + 3 * NX))
        if (img + uni + 210) * esz > SMEM_MAX:
            continue
        yield t


def autotune(params: Dict, n_max: int, precision: int = 0, mode: int = 1, batch: int = 2048, seed: int = 7,
             reps: int = 2, path: str = DEFAULT_CACHE, cands: Optional[Iterable[int]] = None) -> Dict:
    import torch

    from . import inputs
    from .pdg_mc import Solver
    dev = torch.device("cuda")
    name = torch.cuda.get_device_name(dev)
    x0 = torch.from_numpy(inputs.dispersion(params, batch, seed, "bj")).to(dev)
    S = Solver(params, n_max, precision)
    results = {}
    for t in (cands or candidates(n_max, int(params["nu"]), precision)):
        S.set_threads(t)
        try:
            S.solve(x0, mode=mode)
            torch.cuda.synchronize()
        except RuntimeError:
            continue
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            out = S.solve(x0, mode=mode)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            conv = int((out["status"] == 0).sum().item())
            rate = conv / dt
            best = rate if best is None else max(best, rate)
        results[t] = best
    S.close()
    t_best = max(results, key=results.get)
    entry = {"threads": int(t_best), "solves_per_s": results[t_best], "batch": batch,
             "swept": {str(k): v for k, v in sorted(results.items())}}
    cache = load_cache(path)
    cache[cache_key(name, n_max, int(params["nu"]), precision, mode)] = entry
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
    ap.add_argument("--cache", default=DEFAULT_CACHE)
    a = ap.parse_args()
    p = inputs.load_params(nu=a.nu)
    for n in a.nodes:
        for pr in a.precision:
            for m in a.mode:
                e = autotune(p, n, 0 if pr == "fp64" else 1, 1 if m == "persistent" else 0, a.batch, path=a.cache)
                print(json.dumps({"nodes": n, "precision": pr, "mode": m, **e}))


if __name__ == "__main__":
    main()
