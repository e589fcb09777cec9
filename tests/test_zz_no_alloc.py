"""The readout entry point that allocates nothing (qpe_readout_static).

It exists for callers that cannot allocate device memory, so it takes no
workspace and keeps its scratch in a fixed array inside the library. Its
histogram and readout must equal what the regular plan path produces for the
same final statevector, on two calls in a row (the second call reuses the
scratch the first one left behind). This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2507_17175_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {0: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe
    return qpe


def regular_path(q, inst, prec):
    """Histogram, readout and final state from the plan-based entry points."""
    import torch
    plan = q.Plan(inst.nmat, inst.nmeas, prec, 0x10)  # QPE_FLAG_KEEP_STATE
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, pa, pm = plan.probs()
    dt = torch.complex128 if prec == q.FP64 else torch.complex64
    X = torch.empty((inst.N, inst.d), dtype=dt, device="cuda")
    plan.state(X)
    torch.cuda.synchronize()
    return P, am, pa, pm, X


@pytest.mark.parametrize("prec", [0, 1])
def test_static_readout_matches_regular_path_twice(q, prec):
    import torch
    rng = np.random.default_rng(2024)
    cases = [W.haar_instance(rng, 3, 12, superposition=True), W.haar_instance(rng, 5, 9, superposition=True)]
    for inst in cases:  # two calls in a row, different problems, shared scratch
        P, am, pa, pm, X = regular_path(q, inst, prec)
        probs = torch.full((inst.N,), -1.0, dtype=torch.float64, device="cuda")
        ro = torch.zeros(4, dtype=torch.float64, device="cuda")
        st = q.readout_static(X, inst.nmat, inst.nmeas, prec, probs, ro)
        assert st == q.OK, q.status_string(st)
        torch.cuda.synchronize()
        Ps = probs.cpu().numpy()
        r = ro.cpu().numpy()
        am_s = int(r[:1].view(np.int64)[0])
        assert np.abs(Ps - P).max() <= TOL[prec]
        assert am_s == am
        assert abs(r[1] - pa) <= 1e-12 and abs(r[2] - pm) <= TOL[prec] * 10
        assert abs(r[3] - P.sum()) <= TOL[prec] * 10


def test_static_readout_rejects_oversized_problems(q):
    import torch
    X = torch.zeros(8, dtype=torch.complex64, device="cuda")
    probs = torch.zeros(8, dtype=torch.float64, device="cuda")
    ro = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert q.readout_static(X, 1, 22, 1, probs, ro) == q.ERR_WORKSPACE
    assert q.readout_static(X, 0, 3, 1, probs, ro) == q.ERR_ARG
