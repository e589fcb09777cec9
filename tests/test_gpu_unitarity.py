"""QPE_FLAG_CHECK_UNITARY: the POWERS stage measures max |(U^dagger U - I)_ij|
in FP64 and reports QPE_ERR_NUMERIC above 1e-8.

QPE is defined for a unitary U (Sec. 2); the check guards the squaring chain,
which amplifies non-unitarity by ~2^k. The paper's own analytic family
(Sec. 3, U = P Lambda P^{-1} with non-orthogonal P) is the natural negative
case. The threshold is pinned exactly with a scaled unitary: for
U' = (1 + delta) U the only non-zero entries of U'^dagger U' - I are the
diagonal ones, 2 delta + delta^2.
"""
import numpy as np
import pytest

from oracle import fejer
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


def run(q, inst, prec, flags, U=None):
    plan = q.Plan(inst.nmat, inst.nmeas, prec, flags)
    plan.load(inst.U if U is None else U, inst.psi)
    plan.run()
    return plan


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("extra", [0, 0x8, 0x2])  # fused, plain, graph replay
def test_unitary_input_passes_and_results_unchanged(q, prec, extra):
    inst = W.c2()
    P0, am0, *_ = run(q, inst, prec, extra).probs()
    plan = run(q, inst, prec, extra | q.FLAG_CHECK_UNITARY)
    plan.sync()
    P1, am1, *_ = plan.probs()
    assert am1 == am0
    assert np.array_equal(P1, P0)


@pytest.mark.parametrize("delta,flagged", [(1e-8, True), (4e-9, False), (-1e-8, True), (-4e-9, False)])
def test_threshold_is_1e8_per_entry(q, delta, flagged):
    inst = W.c1()
    plan = run(q, inst, q.FP64, q.FLAG_CHECK_UNITARY, U=(1.0 + delta) * inst.U)
    if flagged:
        with pytest.raises(q.QpeError) as e:
            plan.sync()
        assert e.value.status == q.ERR_NUMERIC
        with pytest.raises(q.QpeError) as e:
            plan.probs()
        assert e.value.status == q.ERR_NUMERIC
    else:
        plan.sync()
        plan.probs()


@pytest.mark.parametrize("nmat,nmeas,j", [(2, 4, 1), (3, 5, 6)])
def test_paper_analytic_family_is_flagged(q, nmat, nmeas, j):
    inst = W.analytic_instance(nmat, nmeas, j)
    G = inst.U.conj().T @ inst.U
    assert np.abs(G - np.eye(1 << nmat)).max() > 1e-2  # not unitary, by construction
    plan = run(q, inst, q.FP64, q.FLAG_CHECK_UNITARY)
    with pytest.raises(q.QpeError) as e:
        plan.probs()
    assert e.value.status == q.ERR_NUMERIC
    # without the check the eigenvector input still gives the exact phase
    P, am, *_ = run(q, inst, q.FP64, 0).probs()
    assert am == (j << nmeas) >> nmat


def test_nan_is_flagged_by_the_check(q):
    inst = W.c1()
    U = inst.U.copy()
    U[0, 3] = np.nan
    plan = run(q, inst, q.C64_FP32, q.FLAG_CHECK_UNITARY, U=U)
    with pytest.raises(q.QpeError) as e:
        plan.sync()
    assert e.value.status == q.ERR_NUMERIC


@pytest.mark.parametrize("flags", [0, 0x2])
def test_error_word_is_cleared_by_the_next_run(q, flags):
    inst = W.c1()
    plan = q.Plan(inst.nmat, inst.nmeas, q.FP64, flags | q.FLAG_CHECK_UNITARY)
    plan.load(1.001 * inst.U, inst.psi)
    plan.run()
    with pytest.raises(q.QpeError):
        plan.sync()
    plan.load(inst.U, inst.psi)
    plan.run()
    plan.sync()
    P, am, *_ = plan.probs()
    assert am == int(inst.meta["k"][0])
    assert abs(P[am] - 1.0) <= 1e-10


def test_tensor_core_plan_with_check(q):
    inst = W.haar_instance(np.random.default_rng(7), 7, 6)
    plan = run(q, inst, q.C64_TF32X3, q.FLAG_PLAIN | q.FLAG_CHECK_UNITARY)
    P, am, *_ = plan.probs()
    ref = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    assert np.abs(P - ref).max() <= 1e-5
    plan.load(1.001 * inst.U, inst.psi)
    plan.run()
    with pytest.raises(q.QpeError) as e:
        plan.probs()
    assert e.value.status == q.ERR_NUMERIC


def test_batched_flags_only_the_bad_instance(q):
    good = [W.c1(), W.haar_instance(np.random.default_rng(3), 3, 7)]
    bad = W.analytic_instance(2, 6, 2)
    insts = [good[0], bad, good[1]]
    bp = q.BatchedPlan([(i.nmat, i.nmeas) for i in insts], q.FP64, q.FLAG_CHECK_UNITARY)
    for k, inst in enumerate(insts):
        bp.load(k, inst.U, inst.psi)
    bp.run()
    for k in (0, 2):
        P, *_ = bp.probs(k)
        ref = fejer.probabilities(insts[k].phases, insts[k].weights, insts[k].nmeas)
        assert np.abs(P - ref).max() <= 1e-10
    with pytest.raises(q.QpeError) as e:
        bp.probs(1)
    assert e.value.status == q.ERR_NUMERIC
