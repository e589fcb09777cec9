"""Scaling, memory footprint and profiler split of the GPU path: the GB300
counterpart of the measurements in Sec. 4.1 (time and memory against the
total qubit count) and Sec. 4.3 (allocation, host-to-device copy and matrix
application, Tables 1-2).

Inputs are the paper's analytically solvable family (Sec. 3): phases
j / 2^Nmat, psi = its eigenvector x_1, so every run has a known exact answer
(the argmax is checked). For each (Nmat, Nmeas, precision, schedule) one JSON
line reports:

* ``workspace_bytes``: the path's whole device footprint (the library
  allocates nothing itself); ``peak_vram_bytes``: torch's peak while the plan
  runs (workspace + the caller's U/psi/histogram buffers);
* ``alloc_ms``: allocating the workspace from an emptied caching allocator
  (a cudaMalloc), plus ``plan_bind_ms`` for qpe_plan + qpe_bind;
* ``load_ms``: qpe_load of U and psi from pinned host memory, synchronised;
* ``stage_ms``: CUDA-event times of the four stages of one run (squaring
  chain, controlled gates, QFT^-1, histogram) and ``run_ms`` for the whole
  run, medians over ``--repeat`` runs after a warm-up.

Schedules: ``gate`` applies the controlled gates one measurement qubit at a
time over the materialised state (the paper's gate sequence; Nmat <= 6);
``fused`` is the default schedule; ``plain`` materialises the state with the
doubling schedule.

    python -m paper_2507_17175_gb300.scaling_study --tables
    python -m paper_2507_17175_gb300.scaling_study --sweep 10:30 --nmat 2,4,6
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

# the (Nmat, Nmeas) shapes of the paper's profiler tables (Tables 1 and 2)
TABLE_SHAPES = [(2, 18), (2, 19), (4, 14), (4, 15), (4, 16), (5, 15), (5, 16),
                (6, 14), (6, 15), (8, 12), (8, 13)]

SCHEDULE_FLAGS = {"fused": 0, "gate": 0x1, "plain": 0x8}


def measure(nmat: int, nmeas: int, prec: int, schedule: str, repeat: int = 5) -> dict:
    import torch
    from . import qpe, workloads
    inst = workloads.analytic_instance(nmat, nmeas, 1)
    flags = SCHEDULE_FLAGS[schedule] | qpe.FLAG_TIMING
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)

    U_h = torch.from_numpy(inst.U).pin_memory()
    psi_h = torch.from_numpy(inst.psi).pin_memory()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()

    t0 = time.perf_counter()
    st, ws_bytes, h = qpe.plan_workspace(nmat, nmeas, prec, flags)
    if st != qpe.OK:
        raise qpe.QpeError(st, f"qpe_plan: {qpe.status_string(st)}")
    qpe.LIB.qpe_destroy(h)
    t1 = time.perf_counter()
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    plan = qpe.Plan(nmat, nmeas, prec, flags, stream=stream, workspace=ws)
    t3 = time.perf_counter()

    torch.cuda.synchronize()
    t4 = time.perf_counter()
    plan.load(U_h, psi_h)
    torch.cuda.synchronize()
    t5 = time.perf_counter()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.run()
    plan.sync()
    runs, stages = [], []
    for _ in range(repeat):
        e0.record(stream)
        plan.run()
        e1.record(stream)
        plan.sync()
        runs.append(e0.elapsed_time(e1))
        stages.append(plan.stage_times())
    _, am, pa, pm = plan.probs(want_hist=False)
    expect = (1 << nmeas) >> nmat  # y = N j / d with j = 1
    peak = torch.cuda.max_memory_allocated(dev)
    del plan, ws
    torch.cuda.empty_cache()
    return {
        "nmat": nmat, "nmeas": nmeas, "n_total": nmat + nmeas,
        "prec": {qpe.FP64: "fp64", qpe.C64_FP32: "c64"}.get(prec, str(prec)),
        "schedule": schedule,
        "workspace_bytes": int(ws_bytes),
        "state_bytes": (1 << (nmat + nmeas)) * (16 if prec == qpe.FP64 else 8),
        "peak_vram_bytes": int(peak),
        "alloc_ms": (t2 - t1) * 1e3,
        "plan_bind_ms": ((t1 - t0) + (t3 - t2)) * 1e3,
        "load_ms": (t5 - t4) * 1e3,
        "stage_ms": [float(x) for x in np.median(np.array(stages), axis=0)],
        "run_ms": float(np.median(runs)),
        "argmax_exact": int(am) == expect,
    }


def schedules_for(nmat: int, nmeas: int, prec: int, which):
    out = []
    for s in which:
        if s == "gate" and nmat > 6:
            continue
        if s == "fused" and nmat > 6:
            continue
        out.append(s)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--tables", action="store_true", help="the shapes of the paper's profiler tables")
    ap.add_argument("--sweep", default=None, help="first:last total qubit count (step 2)")
    ap.add_argument("--nmat", default="2,4,6", help="Nmat values of the sweep")
    ap.add_argument("--prec", default="fp64,c64")
    ap.add_argument("--schedules", default="gate,fused,plain")
    ap.add_argument("--repeat", type=int, default=5)
    args = ap.parse_args(argv)

    import torch
    from . import qpe
    t0 = time.perf_counter()
    torch.cuda.init()
    torch.empty(1, device="cuda")
    torch.cuda.synchronize()
    print(json.dumps({"context_init_ms": (time.perf_counter() - t0) * 1e3,
                      "device": torch.cuda.get_device_name(0)}), flush=True)

    precs = [{"fp64": qpe.FP64, "c64": qpe.C64_FP32}[p] for p in args.prec.split(",")]
    which = args.schedules.split(",")
    shapes = []
    if args.tables:
        shapes += TABLE_SHAPES
    if args.sweep:
        a, b = (int(x) for x in args.sweep.split(":"))
        for nt in range(a, b + 1, 2):
            for nmat in (int(x) for x in args.nmat.split(",")):
                nmeas = nt - nmat
                if nmat <= nmeas <= 30:
                    shapes.append((nmat, nmeas))
    for nmat, nmeas in shapes:
        for prec in precs:
            for s in schedules_for(nmat, nmeas, prec, which):
                print(json.dumps(measure(nmat, nmeas, prec, s, args.repeat)), flush=True)


if __name__ == "__main__":
    main()
