#!/usr/bin/env python
"""QPE emulator benchmark: runs/s on the 22-qubit workload (Nmat=6, Nmeas=16,
64 x 64 Haar-eigenbasis U with phases uniform in [0,1), psi = V[:,0]).

One step = one whole QPE run (U^(2^k) squaring chain, Hadamard layer +
controlled-U^(2^k) gates, QFT^-1, |amp|^2 histogram + readout) through the C
ABI, U and psi resident on the device. The complex64 path (FP32 gates and
transform, FP64 squaring and readout) is the headline; the all-FP64 path on
the same device is reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPE runs/s + % roofline; mixed-prec & batched vs FP64 at ≤1e-6 L1 prob error"
WORKLOAD = "qpe Nmat=6 Nmeas=16 (22 qubits), Haar 64x64 U, phases U[0,1), psi=V[:,0]"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return {"hbm_gbs": j["hbm_gbs"], "bf16_tflops": j["bf16_tflops"], "sm_max_mhz": j.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def fp64_alu_peak_tflops() -> float:
    """Nominal GB300 FP64 rate (1.25 TFLOP/s); no measured figure exists."""
    return 1.25


def csrc_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2507_17175_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(stage: str):
    """DRAM bytes per launch of `stage` from the committed ncu summary, or None
    if the sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = csrc_hash()
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 3 and not line.startswith("#") and parts[0] == stage and parts[1] == cur:
                return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, device) -> float:
    """MAX of a per-rank scalar across the process group (a single rank: x)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world: int, steps_per_rank: int, local_ms: float, device) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: every rank ran
    ``steps_per_rank`` steps; the job took the slowest rank's time.
    Returns (runs per second over all ranks, max ms over ranks)."""
    slowest = max_over_ranks(local_ms, device)
    return world * steps_per_rank / (slowest / 1e3), slowest


# ------------------------------------------------------------ CPU baseline
def oracle_cost(n: int, d: int) -> float:
    """Amplitude-gate operations of the gate-by-gate oracle: n Hadamards
    (N d each), n controlled gates (N/2 rows x d^2), n(n-1)/2 controlled
    phases and n/2 swaps (N d each)."""
    N = 1 << n
    return n * N * d + n * (N / 2) * d * d + (n * (n - 1) / 2 + n / 2) * N * d


def time_oracle(inst, budget_s: float):
    """Run the FP64 gate-by-gate oracle on the full workload if one run fits
    the budget, else on the largest Nmeas that does, and express the result
    as full-workload runs/s (scaled by the oracle's operation count)."""
    from oracle import gates
    d = inst.d
    n_full = inst.nmeas
    # calibrate on a small register
    ns = min(n_full, 8)
    t0 = time.perf_counter()
    gates.qpe_probabilities(inst.U, inst.psi, ns)
    t_small = time.perf_counter() - t0
    n_s = ns
    while n_s < n_full and t_small * oracle_cost(n_s + 1, d) / oracle_cost(ns, d) <= budget_s:
        n_s += 1
    runs, elapsed = 0, 0.0
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        gates.qpe_probabilities(inst.U, inst.psi, n_s)
        elapsed += time.perf_counter() - t0
        runs += 1
        if time.perf_counter() - t_start >= budget_s or runs >= 1000:
            break
    t_run = elapsed / runs
    scale = oracle_cost(n_full, d) / oracle_cost(n_s, d)
    rps = 1.0 / (t_run * scale)
    if n_s == n_full:
        sample = f"{runs} full gate-by-gate oracle run(s) of the workload"
    else:
        sample = (f"{runs} oracle run(s) at Nmeas={n_s} (same U, psi), scaled to Nmeas={n_full} by the "
                  f"oracle's operation count x{scale:.1f} (extrapolated)")
    return rps, t_run * scale, sample


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ ours
def bench_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe, workloads

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    inst = workloads.c2()
    U_d = torch.from_numpy(inst.U).to(dev)
    psi_d = torch.from_numpy(inst.psi).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def make(prec, flags):
        p = qpe.Plan(inst.nmat, inst.nmeas, prec, flags, device=dev, stream=stream)
        p.load(U_d, psi_d)
        return p

    plan = make(qpe.C64_FP32, qpe.FLAG_GRAPH | qpe.FLAG_TIMING)

    def timed_steps(p, K, W, stage_acc=None, kern_acc=None):
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        with torch.cuda.stream(stream):
            for _ in range(W):
                flush.zero_()
                p.run()
            stream.synchronize()
            for i in range(K):
                flush.zero_()  # L2 flush between timed steps (outside the events)
                ev0[i].record(stream)
                p.run()
                ev1[i].record(stream)
                if stage_acc is not None:
                    st = p.stage_times()
                    for j in range(4):
                        stage_acc[j].append(st[j])
                if kern_acc is not None:
                    kern_acc.append(p.kernel_time())
            stream.synchronize()
        return [a.elapsed_time(b) for a, b in zip(ev0, ev1)]

    # ---------------- headline: complex64 path, K steps
    stage_acc = [[], [], [], []]
    kern_acc = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    gpu_id = f"GPU-{uuid}" if uuid is not None else str(local_rank)
    with ClockSampler(gpu_id) as clk:
        times = timed_steps(plan, args.steps, args.warmup, stage_acc, kern_acc)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches_per_run = plan.query(qpe.INFO_LAST_LAUNCHES)
    memory = {"workspace_bytes": int(plan.ws_bytes),
              "state_bytes_if_materialised": int(inst.N * (1 << inst.nmat) * 8),
              "peak_allocated_bytes": int(torch.cuda.max_memory_allocated(dev)),
              "note": "the library allocates nothing itself: its device footprint is the workspace; the peak "
                      "includes U, psi and the 512 MiB L2-flush buffer"}
    value, total_ms = aggregate(world, args.steps, float(sum(times)), dev)
    ms_per_step = total_ms / args.steps

    P, am, pa, pm = plan.probs()

    # ---------------- FP64 path on the same device
    plan64 = make(qpe.FP64, qpe.FLAG_GRAPH | qpe.FLAG_TIMING)
    k64 = max(3, min(args.steps, 20))
    st64 = [[], [], [], []]
    t64 = timed_steps(plan64, k64, 3, st64)
    P64, am64, _, _ = plan64.probs()
    fp64 = {"runs_per_s": 1e3 / (sum(t64) / k64), "ms_per_run": sum(t64) / k64, "steps": k64,
            "stage_ms": [statistics.median(s) for s in st64],
            "argmax": int(am64)}
    mixed_vs_fp64 = {"l1": float(np.abs(P - P64).sum()), "max_abs": float(np.abs(P - P64).max()),
                     "argmax_equal": bool(am == am64),
                     "phase_mean_diff": float(abs(pm - plan64.probs(want_hist=False)[3]))}
    del plan64

    # ---------------- end to end through the C ABI with host buffers
    U_h = torch.from_numpy(inst.U).pin_memory()
    psi_h = torch.from_numpy(inst.psi).pin_memory()
    hist_h = torch.empty(inst.N, dtype=torch.float64).pin_memory()
    e2e_plan = make(qpe.C64_FP32, qpe.FLAG_GRAPH)
    ke = max(3, min(args.steps, 200))
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            e2e_plan.load(U_h, psi_h)
            e2e_plan.run()
            e2e_plan.probs(hist_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_plan.load(U_h, psi_h)   # H2D of U and psi from pinned memory
            e2e_plan.run()
            e2e_plan.probs(hist_h)      # D2H of the histogram + readout (synchronises)
        t_e2e = time.perf_counter() - t0
    e2e_value, _ = aggregate(world, ke, t_e2e * 1e3, dev)
    e2e = {"value": e2e_value, "unit": "runs/s",
           "h2d_bytes_per_step": int(inst.U.nbytes + inst.psi.nbytes),
           "d2h_bytes_per_step": int(inst.N * 8 + 40)}

    # ---------------- roofline of the dominant stage
    pk = peaks()
    clocks = clk.summary()
    stage_names = ["powers", "sweep", "fft", "reduce"]
    stage_ms = [statistics.median(s) for s in stage_acc]
    dom = int(np.argmax(stage_ms))
    N, d, n = inst.N, inst.d, inst.nmeas
    S_B = N * d * 8
    fp32_peak = fp32_alu_peak_tflops(pk["sm_max_mhz"])
    # algorithmic work per run of each stage
    work = {
        "powers": ("alu", (n - 1) * 8.0 * d ** 3, fp64_alu_peak_tflops() * 1e3, "GFLOP/s",
                   "FP64 squaring: (n-1) x 8 d^3 flop vs nominal 1.25 TFLOP/s FP64"),
        "sweep": ("alu", (N - 1) * 8.0 * d * d, fp32_peak * 1e3, "GFLOP/s",
                  "controlled gates: (N-1) matvecs x 8 d^2 flop vs FP32 FMA peak from unit counts"),
        "fft": ("hbm", 2.0 * S_B * plan.query(qpe.INFO_FFT_PASSES), pk["hbm_gbs"], "GB/s",
                "QFT^-1: passes x (read + write of the state) vs measured HBM copy bandwidth"),
        "reduce": ("hbm", float(S_B + N * 8), pk["hbm_gbs"], "GB/s",
                   "histogram: one read of the state + N doubles vs measured HBM copy bandwidth"),
    }
    bound, amount, peak, unit, note = work[stage_names[dom]]
    achieved = amount / (stage_ms[dom] * 1e-3) / 1e9
    stage_roofline = {"bound": bound, "achieved": round(achieved, 2), "peak": round(peak, 2), "unit": unit,
                      "frac": round(achieved / peak, 4), "stage": stage_names[dom], "note": note}
    # dominant kernel: the top level of the fused schedule, timed by its own
    # CUDA event pair on the launching stream inside every timed step
    kms = [k[0] for k in kern_acc if k[1] == 1]
    if kms:
        t_k = statistics.mean(kms)
        flops = 8.0 * N * d * d  # every one of the N rows receives one d x d complex matvec in this launch
        ach = flops / (t_k * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": round(ach, 2), "peak": round(fp32_peak * 1e3, 2),
                    "unit": "GFLOP/s", "frac": round(ach / (fp32_peak * 1e3), 4),
                    "traffic": recorded_traffic("level2_top"), "kernel": "level2_kernel (top level, fused)",
                    "kernel_ms": round(t_k, 5), "algorithmic_flop_per_launch": flops,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock",
                    "note": "flop counts only the controlled-gate matvecs (8 d^2 per row), not the DFT"}
    else:
        roofline = dict(stage_roofline, traffic=recorded_traffic(stage_names[dom]))

    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "runs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nmat": inst.nmat, "nmeas": inst.nmeas,
                   "precision": "complex64 state, FP32 gates + QFT^-1, FP64 squaring + readout",
                   "parallelism": f"replicas x{world}", "graph": True,
                   "l2": "flushed between timed steps (512 MiB write outside the timed events)"},
        "stage_ms": dict(zip(stage_names, [round(x, 5) for x in stage_ms])),
        "fp64_path": fp64, "complex64_vs_fp64": mixed_vs_fp64, "e2e": e2e,
        "roofline": roofline, "stage_roofline": stage_roofline,
        "gpu_launches": int(launches_per_run * args.steps),
        "clocks": clocks,
        "memory": memory,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rps, t_run, sample = time_oracle(inst, budget_s=args.cpu_budget)
        res["cpu_baseline"] = {"value": rps, "unit": "runs/s", "cores": host_cores(), "kind": "oracle",
                               "sample": sample, "s_per_run": t_run}
    return res


# ------------------------------------------------------------- reference
def bench_reference(args):
    """The CPU oracle as it stands (FP64 gate-by-gate numpy), each step a
    bounded sample of the same workload."""
    from paper_2507_17175_gb300 import workloads
    inst = workloads.c2()
    per_step = max(0.05, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    from oracle import gates
    # choose the sample size once, then time exactly K steps of it
    d, n_full = inst.d, inst.nmeas
    t0 = time.perf_counter()
    gates.qpe_probabilities(inst.U, inst.psi, 8)
    t8 = time.perf_counter() - t0
    n_s = 8
    while n_s < n_full and t8 * oracle_cost(n_s + 1, d) / oracle_cost(8, d) <= per_step:
        n_s += 1
    for _ in range(args.warmup):
        gates.qpe_probabilities(inst.U, inst.psi, n_s)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        gates.qpe_probabilities(inst.U, inst.psi, n_s)
        ts.append(time.perf_counter() - t0)
    scale = oracle_cost(n_full, d) / oracle_cost(n_s, d)
    t_run = sum(ts) / len(ts) * scale
    value = 1.0 / t_run
    sample = ("full gate-by-gate oracle runs" if n_s == n_full else
              f"oracle at Nmeas={n_s} per step, scaled to Nmeas={n_full} by its operation count x{scale:.1f} "
              "(extrapolated)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "runs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_run * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nmat": inst.nmat, "nmeas": inst.nmeas},
            "cpu_baseline": {"value": value, "unit": "runs/s", "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "runs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(bench_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res = bench_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
