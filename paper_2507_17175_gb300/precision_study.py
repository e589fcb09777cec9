"""Estimation accuracy versus the number of measurement qubits (the study of
Sec. 4.2), run on the GPU path.

A seeded 16 x 16 unitary U = V diag(exp(2 pi i phi)) V^dagger (Nmat = 4) is
given each of its 16 eigenvectors as input in turn (one batched plan of 16
instances per Nmeas). For each Nmeas the two estimators of Sec. 4.2, the
most probable outcome and the probability-weighted average, are compared with
the eigenphase the matrix was built from, and the errors are averaged over
the 16 eigenvectors: both as the plain absolute difference Sec. 4.2 uses and
as the distance on the circle (phases live on [0, 1) with 0 = 1).

    python -m paper_2507_17175_gb300.precision_study --nmeas 4:24 --prec fp64

Prints one JSON line per Nmeas.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def circ(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)) % 1.0
    return np.minimum(d, 1.0 - d)


def study_rows(nmeas_list, prec, seed=12345, nmat=4):
    from . import qpe, workloads
    rng = np.random.default_rng(seed)
    d = 1 << nmat
    V = workloads.haar_unitary(rng, d)
    phases = rng.random(d)
    U = workloads.unitary_from_eigen(V, phases)
    rows = []
    for n in nmeas_list:
        bp = qpe.BatchedPlan([(nmat, n)] * d, prec)
        for j in range(d):
            bp.load(j, U, np.ascontiguousarray(V[:, j]))
        bp.run()
        est_max, est_mean = [], []
        for j in range(d):
            _, am, pa, pm = bp.probs(j, want_hist=False)
            est_max.append(pa)
            est_mean.append(pm)
        est_max, est_mean = np.array(est_max), np.array(est_mean)
        rows.append({
            "nmeas": n,
            "err_max_norm": float(np.mean(np.abs(est_max - phases))),
            "err_weighted_mean": float(np.mean(np.abs(est_mean - phases))),
            "circ_err_max_norm": float(np.mean(circ(est_max, phases))),
            "circ_err_weighted_mean": float(np.mean(circ(est_mean, phases))),
        })
        del bp
    return rows, phases


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nmeas", default="4:24", help="first:last (inclusive)")
    ap.add_argument("--prec", choices=["fp64", "c64"], default="fp64")
    args = ap.parse_args(argv)
    from . import qpe
    a, b = (int(x) for x in args.nmeas.split(":"))
    rows, _ = study_rows(range(a, b + 1), qpe.FP64 if args.prec == "fp64" else qpe.C64_FP32)
    for r in rows:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
