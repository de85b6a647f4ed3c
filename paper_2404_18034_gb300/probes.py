"""Device probes behind the roofline denominators and the instruction counts.

  python -m paper_2404_18034_gb300.probes
      FP64 and FP32 FMA-chain throughput (TFLOP/s) and the FMA-chain time with
      32, 16, 8, 4, 2 and 1 active lanes per warp: on a pipe whose cost is per
      warp instruction the time does not depend on the active lanes.

  python -m paper_2404_18034_gb300.probes --pipg-step B
      one SCP iteration of B instances (N = 15, FP64) through pdg_mc_scp_step
      with forced counts (power iteration 10, PIPG 2000), about the solved
      trajectories of the same batch, so that a profiler capture of the
      plain-form PIPG kernel covers exactly 2000 iterations per instance.
"""
from __future__ import annotations

import argparse
import json

from . import build, inputs
from .pdg_mc import Solver, probe_fma, probe_fma_lanes


def pipg_step(B: int, N: int = 15, precision: int = 0, iters: int = 2000):
    import numpy as np
    import torch
    p = inputs.load_params()
    S = Solver(p, N, precision)
    dev = torch.device("cuda")
    x0 = torch.from_numpy(inputs.dispersion(p, B, 5, "bj")).to(dev)
    sol = S.solve(x0, mode=1)
    nu = int(p["nu"])
    shapes = {"xh": (N, 15), "uh": (N, nu), "mup": (N - 1, 15), "mum": (N - 1, 15), "phi": (N - 1, 15),
              "th": (N - 1,)}
    ws = {k: torch.zeros(B, *s, dtype=torch.float64, device=dev) for k, s in shapes.items()}
    force = torch.from_numpy(np.array([[10, iters]] * B, np.int32)).to(dev)
    o = S.scp_step(x0, sol["X"], sol["U"], ws, None, force)
    torch.cuda.synchronize()
    S.close()
    return {"instances": B, "nodes": N, "forced_pipg_iterations": int(o["iters"][0, 1].item())}


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pipg-step", type=int, default=0, metavar="B")
    a = ap.parse_args()
    build.build()
    torch.cuda.init()
    if a.pipg_step:
        print(json.dumps(pipg_step(a.pipg_step)))
        return
    out = {"device": torch.cuda.get_device_name()}
    for prec, name in ((0, "fp64"), (1, "fp32")):
        out[f"{name}_tflops"] = probe_fma(prec)
        out[f"{name}_ms_by_active_lanes"] = probe_fma_lanes(prec, (32, 16, 8, 4, 2, 1))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
