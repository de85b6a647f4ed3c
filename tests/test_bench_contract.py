"""The benchmark's reference arm (the oracle on the host cores) prints one JSON
line with the contract's keys, for both models; the workload naming and the
algorithmic flop counts the roofline divides by are consistent with the
documented per-unit figures."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("model", ["6dof", "3dof"])
def test_reference_arm_prints_one_contract_line(model):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--model", model, "--steps", "1",
                        "--warmup", "0", "--cpu-sample", "4"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"].startswith(f"pdg{model}_")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_algorithmic_flop_counts():
    """The per-iteration and per-discretization figures the roofline uses
    (one FMA = 2 flops) at N = 15, nu = 4."""
    from paper_2404_18034_gb300 import flops
    # 6-DoF: 4 (N-1)(110 + 30 nu) block-product flops (110 structural nonzeros
    # of hat A^-) plus the vector work; dense: 225 entries
    assert flops.pipg_iter(15, 4) == 4 * 14 * (110 + 120) + 9 * 19 * 15 + 9 * 2 * 15 * 14 + 8 * 16 * 14
    assert flops.pipg_iter(15, 4, dense=True) == 4 * 14 * (225 + 120) + 9 * 19 * 15 + 9 * 2 * 15 * 14 + 8 * 16 * 14
    assert flops.pipg_iter(15, 4, dense=True) == 27457
    assert abs(flops.discretization(15, 4, 10) - 2.45e6) < 0.01e6
    # 3-DoF: the same formulas with NX = 8
    assert flops.pipg_iter(15, 4, "3dof") == 4 * 14 * (24 + 64) + 9 * 12 * 15 + 9 * 2 * 8 * 14 + 8 * 9 * 14
    assert flops.discretization(2, 4, 10, "3dof") == 10 * 4 * (16 * (2 * 13 + 24) + 2 * 4 * 2 * 8 + 100)
    # a solve's flops are the sums over its executed counters
    assert flops.solve_flops([15], 4, 10, [2], [3], [5]) == \
        2 * flops.discretization(15, 4, 10) + 3 * flops.power_iter(15, 4) + 5 * flops.pipg_iter(15, 4)
