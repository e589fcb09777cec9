"""The readout entry point that allocates nothing (qpe_readout_static).

It exists for callers that cannot allocate device memory, so it takes no
workspace and keeps its scratch in a fixed array inside the library. Given a
final statevector it must produce the oracle's histogram and readout of that
same state, and equal what the regular plan path produces, on calls in a row
(each call reuses the scratch the previous one left behind). The shapes cover
rows narrower than a warp, rows of several elements per lane (Nmat 7 and 12),
and Nmeas = 21, where all 8192 scratch slots are filled. This file is
collected last on purpose.
"""
import numpy as np
import pytest

from oracle import gates, readout
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


def static_readout(q, X, nmat, nmeas, prec):
    import torch
    N = 1 << nmeas
    probs = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
    ro = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = q.readout_static(X, nmat, nmeas, prec, probs, ro)
    assert st == q.OK, q.status_string(st)
    torch.cuda.synchronize()
    r = ro.cpu().numpy()
    return probs.cpu().numpy(), int(r[:1].view(np.int64)[0]), r[1], r[2], r[3]


@pytest.mark.parametrize("prec", [0, 1])
def test_static_readout_matches_oracle_on_the_same_state(q, prec):
    """The oracle's readout (oracle.gates.probabilities + oracle.readout) of a
    final statevector against qpe_readout_static of the same state, for the
    QPE circuit's own final state and for seeded random states of larger
    rows, on calls in a row."""
    import torch
    rng = np.random.default_rng(99)
    states = []
    inst = W.haar_instance(rng, 3, 10, superposition=True)
    states.append((inst.nmat, inst.nmeas, gates.qpe_final_state(inst.U, inst.psi, inst.nmeas)))
    for nmat, nmeas in ((1, 9), (7, 6), (12, 3), (1, 21)):
        S = W.random_state(rng, 1 << nmeas, 1 << nmat)
        states.append((nmat, nmeas, S / np.linalg.norm(S)))
    dt = torch.complex128 if prec == 0 else torch.complex64
    for nmat, nmeas, S in states:
        Sd = np.ascontiguousarray(S.astype(np.complex128 if prec == 0 else np.complex64))
        X = torch.from_numpy(Sd).cuda()
        assert X.dtype == dt
        Ps, am, pa, pm, tot = static_readout(q, X, nmat, nmeas, prec)
        ref = gates.probabilities(Sd.astype(np.complex128))  # the same (rounded) state, in FP64
        # a pure reduction of the same numbers: summation order is the only difference
        assert np.abs(Ps - ref).max() <= 1e-13 * ref.max()
        top2 = np.sort(ref)[-2:]
        if len(ref) == 1 or top2[1] - top2[0] > 1e-6 * top2[1]:
            assert am == readout.argmax_lowest(ref)
        assert pa == am / (1 << nmeas)
        assert abs(pm - readout.phase_weighted_mean(ref)) <= 1e-9
        assert abs(tot - ref.sum()) <= 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_static_readout_matches_regular_path_twice(q, prec):
    import torch
    rng = np.random.default_rng(2024)
    cases = [W.haar_instance(rng, 3, 12, superposition=True), W.haar_instance(rng, 5, 9, superposition=True),
             W.haar_instance(rng, 1, 21, superposition=True)]
    for inst in cases:  # calls in a row, different problems, shared scratch
        P, am, pa, pm, X = regular_path(q, inst, prec)
        Ps, am_s, pa_s, pm_s, tot = static_readout(q, X, inst.nmat, inst.nmeas, prec)
        assert np.abs(Ps - P).max() <= TOL[prec]
        assert am_s == am
        assert abs(pa_s - pa) <= 1e-12 and abs(pm_s - pm) <= TOL[prec] * 10
        assert abs(tot - P.sum()) <= TOL[prec] * 10
        del X
        torch.cuda.empty_cache()


def test_static_readout_non_finite_state(q):
    """A NaN in the state: total is NaN and argmax is -1 (no defined outcome)."""
    import torch
    X = torch.full((16, 2), float("nan"), dtype=torch.complex64, device="cuda")
    _, am, pa, _, tot = static_readout(q, X, 1, 4, 1)
    assert am == -1 and np.isnan(pa) and np.isnan(tot)


def test_static_readout_rejects_oversized_problems(q):
    import torch
    X = torch.zeros(8, dtype=torch.complex64, device="cuda")
    probs = torch.zeros(8, dtype=torch.float64, device="cuda")
    ro = torch.zeros(4, dtype=torch.float64, device="cuda")
    ptr = X.data_ptr(), probs.data_ptr(), ro.data_ptr()
    assert q.LIB.qpe_readout_static(ptr[0], 1, 22, 1, ptr[1], ptr[2], None) == q.ERR_WORKSPACE
    assert q.LIB.qpe_readout_static(ptr[0], 0, 3, 1, ptr[1], ptr[2], None) == q.ERR_ARG
    with pytest.raises(ValueError):  # the binding checks sizes before any device access
        q.readout_static(X, 1, 3, 1, probs, ro)
