#!/usr/bin/env python
"""QPE emulator benchmark: runs/s on the largest workload, 34 qubits (Nmat=4,
Nmeas=30; 16 x 16 Haar-eigenbasis U with phases uniform in [0,1), psi a
Dirichlet(1)-weighted superposition of all 16 eigenvectors with uniform
phases), on the FP64 path (complex128 state, FP64-accurate arithmetic: the
paper's precision; the top level's contraction runs as exact integer digit
products on the tensor cores, QPE_FLAG_LEVEL_TC, everything else in FP64).

One step = one whole QPE run (U^(2^k) squaring chain, Hadamard layer +
controlled-U^(2^k) gates, QFT^-1, |amp|^2 histogram + readout) through the C
ABI, U and psi resident on the device. Beside the headline: the complex64 and
split-precision paths on the same workload with their L1 / max-abs histogram
difference against the FP64 histogram, end-to-end runs/s with host buffers,
the same FP64 run with every level on the CUDA cores (FP64 FMA), the
top-level kernel's roofline against the measured FP64 peak, and the CPU
oracle on a bounded sample.

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
WORKLOAD = ("qpe Nmat=4 Nmeas=30 (34 qubits), Haar 16x16 U, phases U[0,1), psi = Dirichlet(1)-weighted "
            "superposition of the eigenvectors")
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return {"hbm_gbs": j["hbm_gbs"], "bf16_tflops": j["bf16_tflops"], "sm_max_mhz": j.get("sm_max_mhz", 2070.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# the sources that make up each recorded kernel (its translation unit and the
# headers it includes); a traffic record holds while their code is unchanged
KERNEL_SOURCES = {
    "level_oz_top_c5_fp64": ["paper_2507_17175_gb300/csrc/qpe_oztop.cu", "paper_2507_17175_gb300/csrc/qpe_internal.cuh",
                             "paper_2507_17175_gb300/csrc/qpe_tcgen05.cuh", "include/qpe.h"],
}


def _code_only(text: str) -> str:
    """C / C++ source without its comments (string literals kept as they are);
    csrc_hash also drops blank lines and trailing blanks."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "".join(out)


def csrc_hash(stage: str = "level_oz_top_c5_fp64") -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[stage]:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as fh:
            code = "\n".join(ln.rstrip() for ln in _code_only(fh.read()).splitlines() if ln.strip())
            h.update(rel.encode() + code.encode())
    return h.hexdigest()[:16]


def recorded_traffic(stage: str):
    """DRAM bytes per launch of `stage` from the committed ncu summary, or None
    if the sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = csrc_hash(stage) if stage in KERNEL_SOURCES else None
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
def level_flops(N: int, d: int, r_top: int) -> float:
    """Algorithmic flops of the fused schedule's top level: every one of the N
    rows receives one d x d complex matvec (8 d^2 flop: the controlled gates of
    the top level's measurement qubits applied to Z) and every (y, column) one
    length-2^r_top DFT share (5 r_top flop per complex point, the usual
    5 n log2 n count)."""
    return 8.0 * N * d * d + 5.0 * N * d * r_top


def bench_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe, workloads

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    inst = workloads.c5()
    N, d, n = inst.N, inst.d, inst.nmeas
    U_d = torch.from_numpy(inst.U).to(dev)
    psi_d = torch.from_numpy(inst.psi).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def make(prec, flags):
        p = qpe.Plan(inst.nmat, inst.nmeas, prec, flags, device=dev, stream=stream)
        p.load(U_d, psi_d)
        return p

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

    # ---------------- headline: the FP64 path, K steps
    plan = make(qpe.FP64, qpe.FLAG_GRAPH | qpe.FLAG_TIMING | qpe.FLAG_LEVEL_TC)
    top_on_tc = bool(plan.query(qpe.INFO_TC_TOP_LEVEL))
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
    r_top = plan.query(qpe.INFO_TOP_LEVEL_BITS)
    levels = plan.query(qpe.INFO_LEVELS)
    value, total_ms = aggregate(world, args.steps, float(sum(times)), dev)
    ms_per_step = total_ms / args.steps
    P64 = torch.empty(N, dtype=torch.float64, device=dev)
    _, am64, pa64, pm64 = plan.probs(P64)
    memory = {"workspace_bytes": int(plan.ws_bytes),
              "state_bytes_if_materialised": int(N * d * 16),
              "peak_allocated_bytes": int(torch.cuda.max_memory_allocated(dev)),
              "note": "the library allocates nothing itself: its device footprint is the workspace (powers, level "
                      "buffers, histogram); the fused schedule never holds the N x d state"}

    # ---------------- end to end through the C ABI with host buffers (FP64)
    # host buffers from the library's page-locked allocator (qpe_host_alloc):
    # the copies run at the host link's rate
    U_h = qpe.host_array(inst.U.shape, np.complex128)
    U_h[...] = inst.U
    psi_h = qpe.host_array(inst.psi.shape, np.complex128)
    psi_h[...] = inst.psi
    hist_h = qpe.host_array(N, np.float64)
    # every run copies its histogram into hist_h (on a second stream while the
    # tensor-core top level computes, eight parts); qpe_probs then returns the
    # readout without a second copy
    plan.set_host_histogram(hist_h)
    ke = max(1, min(args.steps, 3))
    with torch.cuda.stream(stream):
        plan.load(U_h, psi_h)
        plan.run()
        plan.probs(hist_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            plan.load(U_h, psi_h)   # H2D of U and psi from page-locked memory
            plan.run()              # ... and the D2H of the histogram into hist_h
            plan.probs(hist_h)      # readout (synchronises)
        t_e2e = time.perf_counter() - t0
    e2e_equal = bool(np.array_equal(hist_h, P64.cpu().numpy()))
    plan.set_host_histogram(None)
    e2e_value, _ = aggregate(world, ke, t_e2e * 1e3, dev)
    e2e = {"value": e2e_value, "unit": "runs/s",
           "h2d_bytes_per_step": int(inst.U.nbytes + inst.psi.nbytes),
           "d2h_bytes_per_step": int(N * 8 + 40), "steps": ke,
           "host_histogram_equals_device": e2e_equal,
           "d2h": "histogram copied by qpe_set_host_histogram during the run (overlapped with the top level's "
                  "computation where it runs on the tensor cores), into qpe_host_alloc memory"}
    del hist_h

    # ---------------- mixed precision on the same workload, against this FP64 histogram
    def compare(P):
        diff = (P - P64).abs()
        return {"l1_vs_fp64": float(diff.sum().item()), "max_abs_vs_fp64": float(diff.max().item())}

    # the same FP64 run with the top level on the CUDA cores (FP64 FMA)
    kcc = max(1, min(args.steps, 3))
    plancc = make(qpe.FP64, qpe.FLAG_GRAPH | qpe.FLAG_TIMING)
    kerncc = []
    tcc = timed_steps(plancc, kcc, 1, kern_acc=kerncc)
    Pcc = torch.empty(N, dtype=torch.float64, device=dev)
    _, amcc, _, pmcc = plancc.probs(Pcc)
    fp64_cc = {"runs_per_s": 1e3 / (sum(tcc) / kcc), "ms_per_run": sum(tcc) / kcc, "steps": kcc,
               "top_level_kernel_ms": statistics.mean(k[0] for k in kerncc if k[1] == 1),
               "precision": "complex128 state, FP64 FMA everywhere",
               "argmax_equal": bool(amcc == am64), "phase_mean_diff": float(abs(pmcc - pm64)), **compare(Pcc)}
    del plancc, Pcc
    k32 = max(3, min(4 * args.steps, 40))
    plan32 = make(qpe.C64_FP32, qpe.FLAG_GRAPH | qpe.FLAG_TIMING)
    kern32 = []
    t32 = timed_steps(plan32, k32, 3, kern_acc=kern32)
    P32 = torch.empty(N, dtype=torch.float64, device=dev)
    _, am32, pa32, pm32 = plan32.probs(P32)
    c64 = {"runs_per_s": 1e3 / (sum(t32) / k32), "ms_per_run": sum(t32) / k32, "steps": k32,
           "top_level_kernel_ms": statistics.mean(k[0] for k in kern32 if k[1] == 1),
           "precision": "complex64 state, FP32 gates + QFT^-1, FP64 squaring + readout",
           "argmax_equal": bool(am32 == am64), "phase_mean_diff": float(abs(pm32 - pm64)), **compare(P32)}
    c64["speedup_vs_fp64"] = c64["runs_per_s"] / (1e3 / ms_per_step)
    del plan32, P32
    split = {}
    for name, prec in (("fp16x2", qpe.C64_FP16X2), ("tf32x3", qpe.C64_TF32X3)):
        try:
            ps = make(prec, qpe.FLAG_GRAPH | qpe.FLAG_TIMING)
        except qpe.QpeError as e:
            split[name] = {"available": False, "reason": str(e)}
            continue
        ks = []
        ts = timed_steps(ps, k32, 3, kern_acc=ks)
        Ps = torch.empty(N, dtype=torch.float64, device=dev)
        _, ams, _, _ = ps.probs(Ps)
        tc_top = bool(ps.query(qpe.INFO_TC_TOP_LEVEL))
        split[name] = {"runs_per_s": 1e3 / (sum(ts) / k32), "ms_per_run": sum(ts) / k32, "steps": k32,
                       "top_level_kernel_ms": statistics.mean(k[0] for k in ks if k[1] == 1),
                       "top_level_on_tensor_cores": tc_top,
                       "argmax_equal": bool(ams == am64), **compare(Ps)}
        split[name]["speedup_vs_fp64"] = split[name]["runs_per_s"] / (1e3 / ms_per_step)
        if not tc_top:
            split[name]["note"] = "Nmat = 4 under this precision runs the fused complex64 levels on the CUDA cores"
        del ps, Ps
    torch.cuda.empty_cache()

    # ---------------- roofline of the dominant kernel (top level of the fused schedule)
    pk = peaks()
    fp64_peak = qpe.measure_fma_peak(True, 4096, 5, device=dev)
    fp32_peak = qpe.measure_fma_peak(False, 65536, 5, device=dev)
    clocks = clk.summary()
    stage_names = ["powers", "sweep", "fft", "reduce"]
    stage_ms = [statistics.median(s) for s in stage_acc]
    kms = [k[0] for k in kern_acc if k[1] == 1]
    t_k = statistics.mean(kms)
    flops = level_flops(N, d, r_top)
    if top_on_tc:
        # the method's own HBM bound for C5: the final state (N x d complex128) written once and read once,
        # 2 S_B per run; the top level produces and consumes every amplitude of it, so its launch carries
        # those bytes (the fused kernel itself moves only Z in and the histogram out: `traffic`)
        state_bytes = float(N) * d * 16
        alg_bytes = 2.0 * state_bytes
        ach = alg_bytes / (t_k * 1e-3) / 1e9
        tensor_flop = 8 * 28 * 2 * (2.0 * 128 * 32 * 16) * (N // (1 << r_top) // 128)
        roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": round(pk["hbm_gbs"], 1),
                    "unit": "GB/s", "frac": round(ach / pk["hbm_gbs"], 4),
                    "traffic": recorded_traffic("level_oz_top_c5_fp64"),
                    "kernel": "level_oz_kernel<1> (tcgen05 digit products + fixed-point twiddle / DFT, FP64 |X|^2)",
                    "kernel_ms": round(t_k, 3), "algorithmic_bytes_per_launch": alg_bytes,
                    "algorithmic_bytes": f"2 x state bytes = 2 x 2^{n} x {d} x 16 B (the C5 roofline's 2 S_B: "
                                         "final state written once and read once)",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)",
                    "tensor_tflops": round(tensor_flop / (t_k * 1e-3) / 1e12, 1),
                    "tensor_frac_of_bf16_peak": round(tensor_flop / (t_k * 1e-3) / 1e12 / pk["bf16_tflops"], 4),
                    "algorithmic_flop_per_launch": flops,
                    "algorithmic_equiv_gflops": round(flops / (t_k * 1e-3) / 1e9, 1),
                    "flop_count": f"8 N d^2 + 5 N d r_top with N = 2^{n}, d = {d}, r_top = {r_top}",
                    "fp64_fma_peak_gflops_measured": round(fp64_peak * 1e3, 1),
                    "fp32_fma_peak_gflops_measured": round(fp32_peak * 1e3, 1)}
    else:
        ach = flops / (t_k * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": round(ach, 2), "peak": round(fp64_peak * 1e3, 2),
                    "unit": "GFLOP/s", "frac": round(ach / (fp64_peak * 1e3), 4),
                    "traffic": recorded_traffic("level2_top_c5_fp64"),
                    "kernel": "level2_kernel<double2, 4, 1> (top level of the fused schedule)",
                    "kernel_ms": round(t_k, 3), "algorithmic_flop_per_launch": flops,
                    "flop_count": f"8 N d^2 + 5 N d r_top with N = 2^{n}, d = {d}, r_top = {r_top}",
                    "peak_source": "measured: FP64 FMA loop on every SM, CUDA events (qpe_measure_fma_peak)",
                    "fp32_fma_peak_gflops_measured": round(fp32_peak * 1e3, 1)}
    # the FP64 CUDA-core top level against the same peak (the level's flops, FMA = 2)
    cc_ach = flops / (fp64_cc["top_level_kernel_ms"] * 1e-3) / 1e9
    fp64_cc["roofline"] = {"bound": "alu", "achieved": round(cc_ach, 2), "peak": round(fp64_peak * 1e3, 2),
                           "unit": "GFLOP/s", "frac": round(cc_ach / (fp64_peak * 1e3), 4),
                           "traffic": recorded_traffic("level2_top_c5_fp64"),
                           "kernel": "level2_kernel<double2, 4, 1> (top level of the fused schedule)"}
    whole = flops / (ms_per_step * 1e-3) / 1e9
    stage_roofline = {"fp64_equiv_gflops_whole_run": round(whole, 2),
                      "fp64_fma_peak_gflops": round(fp64_peak * 1e3, 2),
                      "note": "whole run (squaring chain, every level, readout) credited with the top level's "
                              "8 N d^2 + 5 N d r_top flops only; above the FP64 peak because the contraction "
                              "runs on the tensor cores"}
    c64_flops_ach = flops / (c64["top_level_kernel_ms"] * 1e-3) / 1e9
    c64["roofline"] = {"bound": "alu", "achieved": round(c64_flops_ach, 1), "peak": round(fp32_peak * 1e3, 1),
                       "unit": "GFLOP/s", "frac": round(c64_flops_ach / (fp32_peak * 1e3), 4),
                       "kernel": "level2_kernel<float2, 4, 1> (top level)", "note": "same flop count as the FP64 line"}
    if split.get("fp16x2", {}).get("top_level_on_tensor_cores"):
        # the contraction runs as fp16 products on the tensor cores (hi.hi over K = 2d, cross terms over
        # K = 4d: 3 x 2 x N x 2d x 2d flop); the twiddle, the 16-point DFT and |X|^2 (31 flop per complex
        # point: 6 + 20 + 3, plus 2 for the operand scale) run on the FP32 units of the drain warps
        t_tc = split["fp16x2"]["top_level_kernel_ms"] * 1e-3
        tensor_flop = 3.0 * 2.0 * N * (2 * d) * (2 * d)
        alu_flop = 31.0 * N * d
        split["fp16x2"]["roofline"] = {
            "bound": "alu", "achieved": round(alu_flop / t_tc / 1e9, 1), "peak": round(fp32_peak * 1e3, 1),
            "unit": "GFLOP/s", "frac": round(alu_flop / t_tc / 1e9 / (fp32_peak * 1e3), 4),
            "tensor_tflops": round(tensor_flop / t_tc / 1e12, 1),
            "tensor_frac_of_bf16_peak": round(tensor_flop / t_tc / 1e12 / pk["bf16_tflops"], 4),
            "kernel": "level_tc_top_kernel (tcgen05 fp16 split products + FP32 drain)",
            "algorithmic_equiv_gflops": round(flops / t_tc / 1e9, 1),
            "note": "FP32 work of the drain (31 flop per complex point) against the measured FP32 FMA peak; the "
                    "contraction's tensor-core flops beside it against the measured bf16 peak (fp16 runs at the "
                    "same rate)"}
    hbm_term_ms = 2.0 * N * d * 16 / (pk["hbm_gbs"] * 1e9) * 1e3

    res = {
        "metric": METRIC, "value": round(value, 4), "unit": "runs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nmat": inst.nmat, "nmeas": inst.nmeas,
                   "precision": "complex128 state, FP64-accurate: every level of >= 128 pencils as exact integer "
                                "digit products on the tensor cores (7 x 8-bit digits, Ozaki scheme) with the "
                                "twiddles and the 8-point DFT in 64-bit fixed point; squaring chain, the deepest "
                                "levels, |X|^2 and readout in FP64" if top_on_tc else
                                "complex128 state, FP64 arithmetic everywhere (the paper's)",
                   "schedule": f"fused levels ({levels} levels, top level 2^{r_top}-point DFT"
                               f"{' on the tensor cores' if top_on_tc else ''})",
                   "parallelism": f"replicas x{world}", "graph": True,
                   "l2": "inputs and level buffers far larger than L2; also flushed between timed steps "
                         "(512 MiB write outside the timed events)"},
        "stage_ms": dict(zip(stage_names, [round(x, 3) for x in stage_ms])),
        "readout": {"argmax": int(am64), "phase_argmax": pa64, "phase_mean": pm64},
        "fp64_cuda_cores": fp64_cc,
        "complex64_path": c64, "split_precision_paths": split, "e2e": e2e,
        "roofline": roofline, "stage_roofline": stage_roofline,
        "hbm_term_ms": round(hbm_term_ms, 2),
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
    inst = workloads.c5()
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
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
