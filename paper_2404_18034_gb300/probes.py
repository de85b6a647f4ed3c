"""Device probes behind the roofline denominators.

  python -m paper_2404_18034_gb300.probes

prints the FP64 and FP32 FMA-chain throughput (TFLOP/s) and the FMA-chain
time with 32, 16, 8, 4, 2 and 1 active lanes per warp: on a pipe whose cost is
per warp instruction the time does not depend on the active lanes.
"""
from __future__ import annotations

import json

from . import build
from .pdg_mc import probe_fma, probe_fma_lanes


def main():
    import torch
    build.build()
    torch.cuda.init()
    out = {"device": torch.cuda.get_device_name()}
    for prec, name in ((0, "fp64"), (1, "fp32")):
        out[f"{name}_tflops"] = probe_fma(prec)
        out[f"{name}_ms_by_active_lanes"] = probe_fma_lanes(prec, (32, 16, 8, 4, 2, 1))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
