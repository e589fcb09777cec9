"""Time the batched form on the 512-instance workload (Nmat uniform in
{3..10}, Nmeas in {8..18}, seeded Haar eigenbases) and compare it with running
the same instances one plan at a time.

    python -m paper_2507_17175_gb300.run_batched --prec c64 --count 512 --repeat 3

Prints one JSON line: batched runs/s (all instances per run), the one-by-one
time, and launch counts. Inputs are resident on the device before timing.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", choices=["fp64", "c64", "fp16x2", "tf32x3"], default="c64")
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--single", action="store_true", help="also time one plan per instance")
    ap.add_argument("--autotune", action="store_true", help="let qpe_bind pick the squaring tiles")
    ap.add_argument("--square-tc", action="store_true", help="square U^(2^k) of d >= 256 on the tensor cores")
    ap.add_argument("--level-tc", action="store_true",
                    help="FP64: doubling levels of d >= 256 as exact digit products on the tensor cores")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="also run the plain FP64 batched plan and report the histograms' L1 difference")
    args = ap.parse_args(argv)

    import torch
    from . import qpe, workloads
    insts = workloads.c4(args.count)
    prec = {"fp64": qpe.FP64, "c64": qpe.C64_FP32, "fp16x2": qpe.C64_FP16X2,
            "tf32x3": qpe.C64_TF32X3}[args.prec]
    shapes = [(i.nmat, i.nmeas) for i in insts]
    stream = torch.cuda.Stream()
    flags = (qpe.FLAG_GRAPH | qpe.FLAG_TIMING | (qpe.FLAG_AUTOTUNE if args.autotune else 0) |
             (qpe.FLAG_SQUARE_TC if args.square_tc else 0) | (qpe.FLAG_LEVEL_TC if args.level_tc else 0))
    bp = qpe.BatchedPlan(shapes, prec, flags, stream=stream)
    dev_inputs = [(torch.from_numpy(i.U).cuda(), torch.from_numpy(i.psi).cuda()) for i in insts]
    for k, (U, psi) in enumerate(dev_inputs):
        bp.load(k, U, psi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    with torch.cuda.stream(stream):
        bp.run()  # capture + first replay
        stream.synchronize()
        for _ in range(args.repeat):
            e0.record(stream)
            bp.run()
            e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1))
    hists = [bp.probs(k)[0] for k in range(len(insts))] if args.compare_fp64 else None
    res = {"workload": f"{args.count} instances, Nmat 3..10, Nmeas 8..18", "prec": args.prec,
           "square_tc": bool(args.square_tc),
           "batched_ms": min(times), "batched_runs_per_s": 1e3 / min(times),
           "launches_per_run": bp.query(qpe.INFO_LAST_LAUNCHES),
           "stage_ms": dict(zip(["squarings", "gates (fused levels whole, plain doubling levels)",
                                 "plain QFT^-1 passes", "plain histograms + every readout"],
                                [round(x, 3) for x in bp.stage_times()])),
           "plain_instances": sum(1 for a, _ in shapes if a > 6),
           "square_tile": bp.query(qpe.INFO_SQUARE_TILE),
           "workspace_gib": bp.ws_bytes / 2 ** 30}
    del bp
    torch.cuda.empty_cache()
    if hists is not None:
        ref = qpe.BatchedPlan(shapes, qpe.FP64, qpe.FLAG_GRAPH, stream=stream)
        for k, (U, psi) in enumerate(dev_inputs):
            ref.load(k, U, psi)
        with torch.cuda.stream(stream):
            ref.run()
            e0.record(stream)
            ref.run()
            e1.record(stream)
            stream.synchronize()
        l1, mx, same = [], [], 0
        for k in range(len(insts)):
            Pr, amr, *_ = ref.probs(k)
            l1.append(float(np.abs(hists[k] - Pr).sum()))
            mx.append(float(np.abs(hists[k] - Pr).max()))
            same += int(np.argmax(hists[k]) == amr)
        res.update({"fp64_batched_ms": e0.elapsed_time(e1), "l1_vs_fp64_max": max(l1),
                    "l1_vs_fp64_median": float(np.median(l1)), "maxabs_vs_fp64": max(mx),
                    "argmax_equal": f"{same}/{len(insts)}"})
        del ref
        torch.cuda.empty_cache()
    if args.single:
        plans = []
        total_launches = 0
        t_single = 0.0
        for inst, (U, psi) in zip(insts, dev_inputs):
            p = qpe.Plan(inst.nmat, inst.nmeas, prec, qpe.FLAG_SQUARE_TC if args.square_tc else 0, stream=stream)
            p.load(U, psi)
            with torch.cuda.stream(stream):
                p.run()
                stream.synchronize()
                t0 = time.perf_counter()
                e0.record(stream)
                p.run()
                e1.record(stream)
                stream.synchronize()
                t_single += e0.elapsed_time(e1)
            total_launches += p.query(qpe.INFO_LAST_LAUNCHES)
            del p
        res["one_by_one_ms"] = t_single
        res["one_by_one_launches"] = total_launches
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
