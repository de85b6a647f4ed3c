#!/usr/bin/env python
"""Benchmark: converged 6-DoF powered-descent SCP solves per second on GB300
(--model 3dof: the translational 3-DoF instance of the same problem template).

One step = one full batched solve (every SCP iteration of every instance:
RK4 discretization with STMs, prescaling, power iteration, PIPG, update) of
a batch of seeded synthetic dispersed initial conditions (the "bj"
dispersion), inputs resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|fp32] [--mode persistent|plain]
                  [--batch B] [--nodes N]

Under torchrun each rank solves its own batch (weak scaling, no collective on
the data path); the timed region is bracketed by barriers and the max over
ranks is reported.  --impl reference times the FP64 CPU oracle on the host
cores (rank 0 only) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged PDG SCP solves/s on 1 GB300, batch 16384, N=15; % FP64/FP32 peak"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the solve
# kernel per instance, from ncu captures of the kernel sources with the given
# hash (profiles/ has the summaries); reported only while the sources match.
PROFILED_TRAFFIC = {
    # ncu (dram__bytes_read.sum, dram__bytes_write.sum) of k_persistent<double,4,1> at
    # its tuned 128 threads, 608 instances (one per CTA slot, four per SM):
    # 6-DoF 14.10 MB read + 171.12 MB written; 3-DoF 3.107 MB read + 0.046 MB written
    "40b1c3098dc7d69a": {("6dof", "fp64", 4, 15, "persistent"): 185.22e6 / 608,
                         ("3dof", "fp64", 4, 15, "persistent"): 3.153e6 / 608},
}


def kernel_source_hash() -> str:
    import glob
    import hashlib
    h = hashlib.sha1()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2404_18034_gb300", "csrc", "*.cu*"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]
SMS = 152
MAX_SM_MHZ = 2070.0
FMA_PER_CLK = {"fp64": 2, "fp32": 128}  # per SM, GB300


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--mode", default="persistent", choices=["persistent", "plain", "classed"])
    ap.add_argument("--batch", type=int, default=None, help="instances (default 16384; 4096 with --grad)")
    ap.add_argument("--nodes", type=int, default=15)
    ap.add_argument("--dispersion", default="bj", choices=["bj", "paper256", "nominal"])
    ap.add_argument("--nu", type=int, default=4, choices=[4, 7], help="7: the paper's model with the RCS torque")
    ap.add_argument("--model", default="6dof", choices=["6dof", "3dof"],
                    help="3dof: the translational instance of the problem template (nu = 4)")
    ap.add_argument("--uneven", action="store_true", help="N per instance uniform in {10, 15, 20, 30}")
    ap.add_argument("--grad", action="store_true", help="time gradients (pdg_mc_grad_batch) instead of solves")
    ap.add_argument("--soc", action="store_true",
                    help="thrust magnitude and gimbal bounds as a second-order-cone projection in PIPG")
    ap.add_argument("--glide-slope", action="store_true", help="add the glide-slope CTCS row (gamma_gs)")
    ap.add_argument("--dt-min", type=float, default=0.0, help="Delta t_k lower bound (0: off)")
    ap.add_argument("--dt-max", type=float, default=0.0, help="Delta t_k upper bound (0: off)")
    ap.add_argument("--tf-max", type=float, default=0.0, help="final-time bound (0: off)")
    ap.add_argument("--pipg-form", type=int, default=0, choices=[0, 1, 2, 3],
                    help="PIPG layout: 0 autotune cache / automatic, 1 shared memory, 2 registers, "
                         "3 register tiles over lane groups")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: autotune cache / automatic)")
    ap.add_argument("--err-sample", type=int, default=512,
                    help="fp32: instances re-solved in fp64 on the GPU to report the fp32 error (0: off)")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle sample size (0: automatic, at least 256)")
    ap.add_argument("--scp-tol-scale", type=float, default=1.0,
                    help="divide the SCP step and defect tolerances (reading R8) by this factor")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def shard_seed(base_seed: int, rank: int) -> int:
    """Each rank draws its own dispersed batch (weak scaling: no data exchange)."""
    return base_seed + 1000 * rank


def reduce_over_ranks(total_ms: float, converged: int, solved: int, dist, device):
    """Whole-job figures: the slowest rank's time and the instances of all ranks."""
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    c = torch.tensor([converged, solved], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), int(c[0]), int(c[1])


def workload_name(a):
    n = "Nuneven10-30" if a.uneven else f"N{a.nodes}"
    nu = "" if a.nu == 4 else f"_nu{a.nu}"
    soc = "_soc" if getattr(a, "soc", False) else ""
    gs = "_gs" if getattr(a, "glide_slope", False) else ""
    tb = "_tbounds" if (getattr(a, "dt_min", 0) or getattr(a, "dt_max", 0) or getattr(a, "tf_max", 0)) else ""
    tol = f"_scptol/{a.scp_tol_scale:g}" if getattr(a, "scp_tol_scale", 1.0) != 1.0 else ""
    return f"pdg{getattr(a, 'model', '6dof')}_{a.dispersion}_B{a.batch}_{n}{nu}{soc}{gs}{tb}{tol}_{a.precision}_{a.mode}"


def load_workload_params(a):
    """Parameters of the workload the flags name (the SCP tolerances divided
    by --scp-tol-scale)."""
    from paper_2404_18034_gb300 import inputs
    p = inputs.load_params(nu=a.nu, model=a.model, soc_thrust=int(getattr(a, "soc", False)),
                           glide_slope=int(getattr(a, "glide_slope", False)), dt_min=getattr(a, "dt_min", 0.0),
                           dt_max=getattr(a, "dt_max", 0.0), tf_max=getattr(a, "tf_max", 0.0))
    k = float(getattr(a, "scp_tol_scale", 1.0))
    p["scp_eps_step"] = p["scp_eps_step"] / k
    p["scp_eps_defect"] = p["scp_eps_defect"] / k
    return p


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join("/tmp", f"pdg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_run(p, x0, N, nthreads):
    """Oracle solves of the rows of x0 (N: one node count, or one per row);
    returns (converged, wall seconds)."""
    import oracle
    oracle.build()
    Ns = np.broadcast_to(np.asarray(N, np.int32), (x0.shape[0],)).copy()
    t = time.perf_counter()
    r = oracle.solve_batch(p, x0, Ns, nthreads=nthreads)
    dt = time.perf_counter() - t
    return int(np.sum(r["status"] == 0)), dt


def cpu_baseline(p, a, seed, sample, budget_s: float = 12.0):
    """The oracle on the host cores, on a seeded random subsample of the batch
    (at least 256 instances, else as many as fit in about budget_s), with
    OpenMP over instances on every core; then the same oracle on one core, on
    the first 16 instances of that subsample: the per-solve time of a serial
    CPU solver, the comparison Sec. 6 makes."""
    cores = os.cpu_count() or 1
    from paper_2404_18034_gb300 import inputs
    x0 = inputs.dispersion(p, a.batch, seed, a.dispersion)
    Ns = inputs.node_counts(a.batch, seed) if a.uneven else np.full(a.batch, a.nodes, np.int32)
    order = np.random.default_rng(seed).permutation(a.batch)
    if sample <= 0:
        probe = order[:cores * 2]
        conv, dt = cpu_oracle_run(p, x0[probe], Ns[probe], cores)
        per = dt / len(probe)
        sample = int(min(a.batch, max(256, round(budget_s / max(per, 1e-6)))))
    pick = np.sort(order[:sample])
    conv, dt = cpu_oracle_run(p, x0[pick], Ns[pick], cores)
    one = pick[:16]
    conv1, dt1 = cpu_oracle_run(p, x0[one], Ns[one], 1)
    return {"value": conv / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample} of the {a.batch} instances of {workload_name(a)}, drawn by a seeded permutation "
                      f"(FP64 oracle, OpenMP over instances, {cores} threads, {dt:.1f} s); converged solves / wall "
                      f"time",
            "converged_in_sample": conv,
            "single_core": {"value": conv1 / dt1, "unit": "solves/s", "ms_per_solve": 1e3 * dt1 / len(one),
                            "sample": f"the first {len(one)} instances of that sample on one thread",
                            "converged_in_sample": conv1}}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2404_18034_gb300 import inputs
    p = load_workload_params(a)
    seed = inputs.config_seed(2)
    x0 = inputs.dispersion(p, a.batch, seed, a.dispersion)
    cores = os.cpu_count() or 1
    per_step = a.cpu_sample or max(cores * 4, 64)
    per_step = min(per_step, a.batch)
    times, convs = [], []
    for s in range(a.warmup + a.steps):
        lo = (s * per_step) % max(1, a.batch - per_step + 1)
        conv, dt = cpu_oracle_run(p, x0[lo:lo + per_step], a.nodes, cores)
        if s >= a.warmup:
            times.append(dt)
            convs.append(conv)
    value = sum(convs) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(a), "batch": a.batch, "nodes": a.nodes,
                                            "precision": "fp64", "dispersion": a.dispersion,
                                            "parallelism": f"dp{a.gpus}"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} instances of {workload_name(a)} per step (FP64 oracle, "
                                       f"OpenMP over instances, {cores} threads)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_grad(a):
    """Gradient workload: B dispersed instances, d(fuel, touchdown)/d(x0, m_wet)."""
    import torch

    from paper_2404_18034_gb300 import build, flops, inputs
    from paper_2404_18034_gb300.pdg_mc import Solver
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p = inputs.load_params(model=a.model)
    x0 = torch.from_numpy(inputs.dispersion(p, a.batch, inputs.config_seed(3), a.dispersion)).to(dev)
    S = Solver(p, a.nodes, 0)
    gf = torch.ones(a.batch, dtype=torch.float64, device=dev)
    gt = torch.ones(a.batch, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(a.warmup):
        o = S.grad(x0, None, gf, gt)
    torch.cuda.synchronize(dev)
    ms, ok = [], 0
    with ClockSampler(0) as clk:
        for _ in range(a.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o = S.grad(x0, None, gf, gt)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
            ok += int((o["status"] <= 1).sum().item())
    # algorithmic flops of one step from the counters of the same solve: the
    # forward solve, plus the adjoint of its last SCP iteration counted as the
    # PIPG loop twice (recomputed from checkpoints, then reversed), the
    # first interval's discretization in dual arithmetic (3 flops per real
    # flop) along the NX - 1 directions of x0, and the touchdown interval twice
    sol = S.solve(x0, mode=1, trace=True)
    torch.cuda.synchronize(dev)
    scp = sol["scp_iters"].cpu().numpy()
    tr = sol["trace"].cpu().numpy()
    live = o["status"].cpu().numpy() <= 1
    N, nu, nsub = a.nodes, p["nu"], p["rk4_substeps"]
    fwd = flops.solve_flops(np.full(a.batch, N), nu, nsub, scp, tr[:, :, 0].sum(1), sol["pipg_iters"].cpu().numpy(),
                            a.model)
    last_pipg = tr[np.arange(a.batch), np.maximum(scp - 1, 0), 1]
    one = flops.discretization(2, nu, nsub, a.model)
    adj = float(np.sum(live * (2.0 * last_pipg * flops.pipg_iter(N, nu, a.model)
                               + (3.0 * (S.nx - 1) + 2.0) * one)))
    achieved = (fwd + adj) / (float(np.mean(ms)) * 1e-3) / 1e12
    peak = SMS * FMA_PER_CLK["fp64"] * 2 * MAX_SM_MHZ * 1e6 / 1e12
    cpu = None if a.no_cpu else cpu_grad_baseline(p, a, x0.cpu().numpy())
    line = {"metric": f"gradients d(fuel, touchdown)/d(x0, m_wet) per second on 1 GB300, batch {a.batch}, N={a.nodes}",
            "value": ok / (sum(ms) * 1e-3), "unit": "grads/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"pdg{a.model}_grad_{a.dispersion}_B{a.batch}_N{a.nodes}_fp64", "batch": a.batch,
                       "nodes": a.nodes, "model": a.model, "l2": "256 MiB buffer written between timed steps",
                       "includes": "the forward solve and the adjoint of its last SCP iteration"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "k_persistent + k_grad (one gradient step)",
                         "flops_per_launch": fwd + adj, "flops_forward": fwd, "flops_adjoint": adj,
                         "peak_source": f"derived: {SMS} SMs x 2 FP64 FMA/clk x 2 flop x {MAX_SM_MHZ:.0f} MHz"},
            "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": 2 * a.steps}
    print(json.dumps(line), flush=True)
    S.close()


def cpu_grad_baseline(p, a, x0h, budget_s: float = 12.0):
    """The oracle's gradient as the tests take it -- a free solve, then
    central differences (h = 1e-6) of its last SCP iteration along every
    direction of x0 -- on the first instances of the batch, one thread per
    host core (the oracle's ctypes calls release the GIL)."""
    import concurrent.futures as cf

    import oracle
    oracle.build()
    cores = os.cpu_count() or 1

    def grad_one(x):
        r = oracle.solve(p, a.nodes, x)
        X, U, ws, sig, n = oracle.final_iteration_state(p, a.nodes, x, r["trace"], r["scp_iters"])
        g = np.zeros((len(x), 2))
        for j in range(len(x)):
            e = np.zeros(len(x)); e[j] = 1e-6
            g[j] = (np.array(oracle.final_iteration_outputs(p, x + e, X, U, ws, sig, n))
                    - np.array(oracle.final_iteration_outputs(p, x - e, X, U, ws, sig, n))) / 2e-6
        return r["status"] <= 1

    t0 = time.perf_counter()
    grad_one(x0h[0])
    per = time.perf_counter() - t0
    sample = int(min(a.batch, max(cores, round(budget_s * cores / max(per, 1e-6)))))
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        done = sum(ex.map(grad_one, list(x0h[:sample])))
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "grads/s", "cores": cores, "kind": "oracle",
            "sample": f"first {sample} of the {a.batch} instances (FP64 oracle: free solve, then central differences "
                      f"of its last SCP iteration along the {x0h.shape[1]} directions of x0; {cores} threads, "
                      f"{dt:.1f} s)"}


def fp32_error(p, a, S32, x0, Ns, out32, mode, dev):
    """Re-solve the first instances in FP64 on the GPU and report the FP32 path's
    largest deviation on instances that converged in both with equal SCP
    counts: trajectories scaled per component by max(|x64|, P), final time
    and fuel relative."""
    import torch

    from paper_2404_18034_gb300.pdg_mc import Solver
    n = min(a.err_sample, a.batch)
    S64 = Solver(p, a.nodes, 0, mode=mode)
    o64 = S64.solve(x0[:n].contiguous(), None if Ns is None else Ns[:n].contiguous(), mode=mode)
    torch.cuda.synchronize(dev)
    # compared as the tests compare: converged in both with equal SCP counts
    # (an instance that stops one SCP iteration apart differs by up to the
    # SCP step tolerance, which is not rounding)
    ok = ((o64["status"] == 0) & (out32["status"][:n] == 0)
          & (o64["scp_iters"] == out32["scp_iters"][:n])).cpu().numpy()
    Px = np.asarray(p["P_x"])
    Pu = np.asarray(p["P_u"])[:p["nu"]]
    X32, X64 = out32["X"][:n].cpu().numpy()[ok], o64["X"].cpu().numpy()[ok]
    U32, U64 = out32["U"][:n].cpu().numpy()[ok], o64["U"].cpu().numpy()[ok]
    ex = np.abs(X32 - X64) / np.maximum(np.abs(X64), Px)
    eu = np.abs(U32 - U64) / np.maximum(np.abs(U64), Pu)
    if Ns is not None:  # nodes past an instance's N are padding
        nn = Ns[:n].cpu().numpy()[ok]
        live = np.arange(X32.shape[1])[None, :] < nn[:, None]
        ex, eu = ex[live], eu[live]
    rel = lambda k: float(np.max(np.abs(out32[k][:n].cpu().numpy()[ok] - o64[k].cpu().numpy()[ok])
                                 / np.abs(o64[k].cpu().numpy()[ok]))) if ok.any() else None
    S64.close()
    return {"instances": int(ok.sum()), "of": n, "max_scaled_err_X": float(ex.max()) if ok.any() else None,
            "max_scaled_err_U": float(eu.max()) if ok.any() else None, "max_rel_err_tf": rel("tf"),
            "max_rel_err_fuel": rel("fuel"),
            "note": "first instances of the batch re-solved by the FP64 kernel; both converged in the same "
                    "number of SCP iterations"}


def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_2404_18034_gb300 import build, flops, inputs
    from paper_2404_18034_gb300.pdg_mc import Solver, probe_fma

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    prec = 0 if a.precision == "fp64" else 1
    p = load_workload_params(a)
    seed = shard_seed(inputs.config_seed(2), rank)
    x0h = inputs.dispersion(p, a.batch, seed, a.dispersion)
    x0 = torch.from_numpy(x0h).to(dev)
    Ns_h = inputs.node_counts(a.batch, seed) if a.uneven else None
    Ns = torch.from_numpy(Ns_h).to(dev) if a.uneven else None
    if a.uneven:
        a.nodes = int(Ns_h.max())
    mode = {"plain": 0, "persistent": 1, "classed": 2}[a.mode]
    from paper_2404_18034_gb300.autotune import DEFAULT_CACHE
    S = Solver(p, a.nodes, prec, tune_cache=DEFAULT_CACHE, mode=mode)
    if a.pipg_form:
        S.set_pipg_form(a.pipg_form)
        if S.tuned_form != a.pipg_form:  # cached threads were tuned for the other layout
            S.set_threads(0)
            S.tuned_threads = None
    if a.threads:
        S.set_threads(a.threads)
        S.tuned_threads = None
    out = S.alloc_outputs(a.batch, dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step(trace=False):
        return S.solve(x0, Ns, mode=mode, out=out, trace=trace, stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize(dev)
    info = S.launch_info()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    conv_counts = []
    traces = None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            o = step(trace=True)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    st = out["status"].cpu().numpy()
    conv = int(np.sum(st == 0))
    tr = o["trace"].cpu().numpy()
    scp = out["scp_iters"].cpu().numpy()
    pipg = out["pipg_iters"].cpu().numpy()
    pow_it = tr[:, :, 0].sum(1)
    total_ms = float(np.sum(ms))
    total_ms_max, conv_all, solved_all = reduce_over_ranks(total_ms, conv * a.steps, a.batch * a.steps,
                                                           dist if world > 1 else None, dev)
    value = conv_all / (total_ms_max * 1e-3)

    # roofline of the dominant kernel (the persistent solve kernel is the whole step)
    Nv = Ns_h if a.uneven else np.full(a.batch, a.nodes)
    fl = flops.solve_flops(Nv, p["nu"], p["rk4_substeps"], scp, pow_it, pipg, a.model)
    fl_dense = flops.solve_flops(Nv, p["nu"], p["rk4_substeps"], scp, pow_it, pipg, a.model, dense=True)
    launch_s = float(np.mean(ms)) * 1e-3
    achieved = fl / launch_s / 1e12
    clocks = clk.summary()
    peak_nominal = SMS * FMA_PER_CLK[a.precision] * 2 * MAX_SM_MHZ * 1e6 / 1e12
    try:
        probe = probe_fma(prec, stream)
    except RuntimeError:
        probe = None

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not a.no_e2e:
        pin = torch.from_numpy(x0h).pin_memory()
        x0_pinned = pin.numpy()
        outs = {k: torch.empty(tuple(v.shape), dtype=v.dtype).pin_memory().numpy() for k, v in out.items()
                if k != "trace"}
        S.solve_host(x0_pinned, Ns_h, mode=mode, out=outs, stream=stream)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_conv = 0
        for _ in range(a.steps):
            r = S.solve_host(x0_pinned, Ns_h, mode=mode, out=outs, stream=stream)
            e2e_conv += int(np.sum(r["status"] == 0))
        e2e_s = time.perf_counter() - t0
        e2e_ms_max, e2e_conv_all, _ = reduce_over_ranks(1e3 * e2e_s, e2e_conv, a.batch * a.steps,
                                                        dist if world > 1 else None, dev)
        h2d = x0h.nbytes + (Ns_h.nbytes if a.uneven else 0)
        d2h = sum(v.nbytes for v in outs.values())
        e2e = {"value": e2e_conv_all / (e2e_ms_max * 1e-3), "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    err = None
    if prec == 1 and a.err_sample > 0 and rank == 0:
        err = fp32_error(p, a, S, x0, Ns, out, mode, dev)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_baseline(p, a, inputs.config_seed(2), a.cpu_sample)

    launches = a.steps * (1 if mode == 1 else (1 + 4 * int(scp.max()) if mode == 0 else 1 + len(set(Ns_h.tolist()))
                                                if a.uneven else 1))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "batch_per_gpu": a.batch, "global_batch": a.batch * world,
                       "nodes": "uniform in {10,15,20,30}" if a.uneven else a.nodes, "model": a.model, "nu": p["nu"],
                       "precision": a.precision, "mode": a.mode,
                       "dispersion": a.dispersion, "parallelism": f"dp{world}",
                       "scp_eps_step": p["scp_eps_step"], "scp_eps_defect": p["scp_eps_defect"],
                       "l2": "256 MiB buffer written between timed steps",
                       "threads_per_cta": info["threads"], "ctas_per_sm": info["ctas_per_sm"],
                       "pipg_form": {1: "shared-memory blocks", 2: "register-resident blocks"}.get(info["pipg_form"]),
                       "threads_from_autotune_cache": S.tuned_threads is not None,
                       "smem_bytes_per_cta": info["smem_bytes"]},
            "converged_fraction": conv / a.batch,
            "all_solves_per_s": solved_all / (total_ms_max * 1e-3),
            "mean_scp_iters": float(scp.mean()), "mean_pipg_iters_per_solve": float(pipg.mean()),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_nominal, "unit": "TFLOP/s",
                         "frac": achieved / peak_nominal,
                         "traffic": (PROFILED_TRAFFIC.get(kernel_source_hash(), {}).get(
                             (a.model, a.precision, p["nu"], a.nodes, a.mode)) or 0) * a.batch or None,
                         "traffic_algorithmic_bytes": int(x0h.nbytes + a.batch * a.nodes * (S.nx + p["nu"]) * 8
                                                          + a.batch * 28),
                         "kernel": "whole plain-form step" if mode == 0 else "k_persistent",
                         "flops_per_launch": fl,
                         "flops_count": "structural nonzeros of hat A^- only (flops.py); frac_dense_count counts "
                                        "every entry, as a solver multiplying the zeros would",
                         "frac_dense_count": fl_dense / launch_s / 1e12 / peak_nominal,
                         "peak_source": f"derived: {SMS} SMs x {FMA_PER_CLK[a.precision]} "
                                        f"{a.precision.upper()} FMA/clk x 2 flop x {MAX_SM_MHZ:.0f} MHz",
                         "probe_tflops": probe,
                         "frac_of_probe": (achieved / probe) if probe else None},
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": launches,
        }
        if err is not None:
            line["fp32_vs_fp64"] = err
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.batch is None:
        a.batch = 4096 if a.grad else 16384
    if a.impl == "reference":
        run_reference(a)
    elif a.grad:
        run_grad(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
