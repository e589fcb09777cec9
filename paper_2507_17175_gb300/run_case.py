"""Run one QPE problem through the C ABI from the command line and print the
per-stage times (for profiling a kernel on a chosen size).

    python -m paper_2507_17175_gb300.run_case --nmat 4 --nmeas 24 --prec c64 --repeat 3

The problem is a seeded Haar-eigenbasis instance (superposition input); the
output is one JSON line per repetition with the four stage times in ms.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nmat", type=int, default=None)
    ap.add_argument("--nmeas", type=int, default=None)
    ap.add_argument("--workload", choices=["c2", "c3", "c5"], default=None,
                    help="one of the seeded workloads instead of a random superposition input")
    ap.add_argument("--prec", choices=["fp64", "c64", "tf32x3", "fp16x2"], default="c64")
    ap.add_argument("--flags", type=lambda s: int(s, 0), default=0)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--seed", type=int, default=12345)
    args = ap.parse_args(argv)

    from . import qpe, workloads
    if args.workload:
        inst = workloads.by_name(args.workload)
        args.nmat, args.nmeas = inst.nmat, inst.nmeas
    else:
        if args.nmat is None or args.nmeas is None:
            ap.error("--nmat and --nmeas, or --workload")
        inst = workloads.haar_instance(np.random.default_rng(args.seed), args.nmat, args.nmeas, superposition=True)
    prec = {"fp64": qpe.FP64, "c64": qpe.C64_FP32, "tf32x3": qpe.C64_TF32X3,
            "fp16x2": qpe.C64_FP16X2}[args.prec]
    plan = qpe.Plan(args.nmat, args.nmeas, prec, args.flags | qpe.FLAG_TIMING)
    plan.load(inst.U, inst.psi)
    for i in range(args.repeat):
        plan.run()
        st = plan.stage_times()
        _, am, pa, pm = plan.probs(want_hist=False)
        print(json.dumps({"rep": i, "stage_ms": [round(x, 5) for x in st], "argmax": am,
                          "launches": plan.query(qpe.INFO_LAST_LAUNCHES)}), flush=True)


if __name__ == "__main__":
    main()
