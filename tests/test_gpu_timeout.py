"""Failure detection on the device: a bounded wait that runs out.

Every mbarrier wait in the library's tensor-core kernels has a poll limit;
when it expires the CTA records QPE_ERR_TIMEOUT in the instance's error word,
frees its tensor memory and returns. qpe_selftest_timeout takes that exit on
purpose (a barrier nothing arrives at, a short poll limit, nothing in flight),
so these tests check that the host sees the error and that the next run is
clean again. No GPU fault is involved.
"""
import numpy as np
import pytest

from oracle import gates
from paper_2507_17175_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe
    return qpe


# FP64 fused, complex64 plain, FP16x2 on the tensor cores (with tensor-core
# squaring), and a graph-replayed plan
CASES = [(0, 2, 6, 0), (1, 3, 9, 0x8), (3, 8, 8, 0x100), (1, 4, 10, 0x2)]


@pytest.mark.parametrize("prec,nmat,nmeas,flags", CASES)
def test_expired_wait_is_reported_and_cleared(q, prec, nmat, nmeas, flags):
    rng = np.random.default_rng(nmat * 10 + nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    tol = 1e-10 if prec == 0 else 1e-4
    plan = q.Plan(nmat, nmeas, prec, flags)
    plan.load(inst.U, inst.psi)
    plan.run()
    plan.sync()
    for polls in (1, 64):
        plan.selftest_timeout(polls)
        with pytest.raises(q.QpeError) as e:
            plan.sync()
        assert e.value.status == q.ERR_TIMEOUT
        with pytest.raises(q.QpeError) as e:
            plan.probs()
        assert e.value.status == q.ERR_TIMEOUT
        # the next whole run starts with a clean error word and is correct
        plan.run()
        plan.sync()
        P, am, _, _ = plan.probs()
        assert np.abs(P - ref).max() <= tol


def test_selftest_arguments(q):
    plan = q.Plan(2, 4, q.FP64)
    for bad in (0, (1 << 20) + 1):
        with pytest.raises(q.QpeError) as e:
            plan.selftest_timeout(bad)
        assert e.value.status == q.ERR_ARG
    bp = q.BatchedPlan([(2, 4), (3, 5)], q.C64_FP32)
    assert q.LIB.qpe_selftest_timeout(bp.handle, 0, 8) == q.ERR_UNSUPPORTED
