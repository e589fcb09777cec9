"""Split-precision tensor-core plans (tcgen05 U-application, TF32x3 and
FP16x2) against the FP64 oracle and the closed form."""
import numpy as np
import pytest

from oracle import fejer, gates, readout
from paper_2507_17175_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TF32X3, FP16X2 = 4, 3
# Row tolerance relative to the largest amplitude: tf32 and fp16 splits keep
# ~21-22 significand bits per operand (fp16 after the power-of-two scaling);
# FP32 accumulation over 2d terms and <= 2 tensor-core levels in these shapes.
ROW_TOL = {TF32X3: 5e-6, FP16X2: 5e-6}
PROB_TOL = {TF32X3: 1e-5, FP16X2: 1e-5}
ALL = [TF32X3, FP16X2]
# The bound on the whole histogram's L1 error, sum_y |P(y) - P_FP64(y)|, that
# the split-precision forms must meet against FP64 (the mixed-precision
# acceptance criterion), with the most probable outcome unchanged.
L1_BOUND = 1e-6


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe
    return qpe


@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("nmat,nmeas", [(5, 8), (5, 10), (6, 9), (7, 9), (8, 10)])
def test_tc_rows_after_gates(q, prec, nmat, nmeas):
    """Rows 2^7.. of the state come from the tensor-core GEMM: compare every
    row with the oracle's gate-by-gate state."""
    rng = np.random.default_rng(nmat * 31 + nmeas)
    U = W.haar_unitary(rng, 1 << nmat)
    psi = W.random_state(rng, 1 << nmat, 1)[:, 0]
    psi /= np.linalg.norm(psi)
    plan = q.Plan(nmat, nmeas, prec)
    plan.load(U, psi)
    plan.run_stages(q.STAGE_POWERS, q.STAGE_SWEEP)
    S = plan.state()
    ref = gates.qpe_after_sweeps(U, psi, nmeas)
    assert np.abs(S - ref).max() <= ROW_TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("nmat,nmeas", [(5, 10), (6, 12), (7, 9), (8, 10)])
def test_tc_end_to_end(q, prec, nmat, nmeas):
    rng = np.random.default_rng(nmat * 7 + nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    plan = q.Plan(nmat, nmeas, prec)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, pa, pm = plan.probs()
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    assert np.abs(P - ref).max() <= PROB_TOL[prec]
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * PROB_TOL[prec]:
        assert am == readout.argmax_lowest(ref)


@pytest.mark.parametrize("prec", ALL)
def test_c3_tensor_cores_vs_closed_form(q, prec):
    """Nmat = 12, Nmeas = 20 (32 qubits) with the U-application on the
    tensor cores: the whole histogram against the Fejer closed form (max-abs
    and L1), and the argmax."""
    inst = W.c3()
    plan = q.Plan(inst.nmat, inst.nmeas, prec)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, pa, pm = plan.probs()
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    err = np.abs(P - Q)
    print(f"prec {prec}: max-abs {err.max():.3e} L1 {err.sum():.3e}")
    assert err.max() <= PROB_TOL[prec]
    assert err.sum() <= L1_BOUND
    order = np.argsort(Q)
    assert Q[order[-1]] - Q[order[-2]] > 10 * PROB_TOL[prec]  # no near-tie in this draw
    assert am == order[-1]


@pytest.mark.parametrize("prec", ALL)
def test_batched_split_precision(q, prec):
    """A batched plan under a split precision: instances with Nmat <= 6 run the
    fused complex64 schedule, the others the doubling schedule with the gate
    GEMMs on the tensor cores; every histogram against the oracle."""
    shapes = [(3, 8), (7, 9), (6, 10), (8, 8), (5, 7), (2, 5)]
    rng = np.random.default_rng(prec)
    insts = [W.haar_instance(rng, a, b, superposition=True) for a, b in shapes]
    bp = q.BatchedPlan(shapes, prec, q.FLAG_GRAPH | q.FLAG_SQUARE_TC)
    for i, inst in enumerate(insts):
        bp.load(i, inst.U, inst.psi)
    refs = [gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas) for inst in insts]
    for _ in range(2):
        bp.run()
        for i, (inst, ref) in enumerate(zip(insts, refs)):
            P, am, *_ = bp.probs(i)
            assert np.abs(P - ref).max() <= PROB_TOL[prec], shapes[i]
            assert np.abs(P - ref).sum() <= L1_BOUND, shapes[i]
            top2 = np.sort(ref)[-2:]
            if top2[1] - top2[0] > 10 * PROB_TOL[prec]:
                assert am == readout.argmax_lowest(ref), shapes[i]


@pytest.mark.parametrize("prec", ALL)
def test_c4_split_precision_l1(q, prec):
    """The 512-instance batch (Nmat 3..10, Nmeas 8..18) under each split
    precision, graph-replayed, with tensor-core squaring: every instance's
    whole histogram within L1 1e-6 of its closed form (single Fejer kernel;
    the FP64 floor at Nmeas <= 18 is below 1e-9) and the same most probable
    outcome."""
    insts = W.c4()
    shapes = [(i.nmat, i.nmeas) for i in insts]
    bp = q.BatchedPlan(shapes, prec, q.FLAG_GRAPH | q.FLAG_SQUARE_TC)
    for k, inst in enumerate(insts):
        bp.load(k, inst.U, inst.psi)
    bp.run()
    worst, worst_shape = 0.0, None
    for k, inst in enumerate(insts):
        P, am, *_ = bp.probs(k)
        Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
        l1 = float(np.abs(P - Q).sum())
        if l1 > worst:
            worst, worst_shape = l1, shapes[k]
        order = np.argsort(Q)
        if Q[order[-1]] - Q[order[-2]] > 10 * PROB_TOL[prec]:
            assert am == order[-1], (k, shapes[k])
    print(f"prec {prec}: worst L1 {worst:.3e} at (nmat, nmeas) = {worst_shape}")
    assert worst <= L1_BOUND, (worst, worst_shape)


# ------------------------------------ fused top level on the tensor cores
@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("nmeas", [11, 12, 15, 18, 21])
def test_fused_tensor_core_top_level_vs_oracle(q, prec, nmeas):
    """Nmat = 4 under FP16x2 and TF32x3: the fused schedule with its top level
    (16-point DFT, 128-pencil tiles) as split products on tcgen05, the deep
    levels in complex64 on the CUDA cores. Whole histogram against the gate-by-gate
    oracle (max-abs and the L1 bound), the readout, and the same histogram as
    the complex64 CUDA-core plan within the split's accuracy."""
    rng = np.random.default_rng(400 + nmeas)
    inst = W.haar_instance(rng, 4, nmeas, superposition=True)
    plan = q.Plan(4, nmeas, prec)
    assert plan.query(q.INFO_TC_TOP_LEVEL) == 1
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, pa, pm = plan.probs()
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    err = np.abs(P - ref)
    assert err.max() <= PROB_TOL[prec]
    assert err.sum() <= L1_BOUND
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * PROB_TOL[prec]:
        assert am == readout.argmax_lowest(ref)
    assert abs(pm - readout.phase_weighted_mean(ref)) <= 2e-5
    c64 = q.Plan(4, nmeas, q.C64_FP32)
    c64.load(inst.U, inst.psi)
    c64.run()
    P32, *_ = c64.probs()
    assert np.abs(P - P32).sum() <= L1_BOUND


@pytest.mark.parametrize("prec", ALL)
def test_fused_tensor_core_top_level_eigenvector_and_graph(q, prec):
    """An eigenvector input (single Fejer kernel, a sharp peak), replayed as a
    CUDA graph twice: identical histograms, closed form within the bound."""
    rng = np.random.default_rng(77)
    inst = W.haar_instance(rng, 4, 16)
    plan = q.Plan(4, 16, prec, q.FLAG_GRAPH)
    plan.load(inst.U, inst.psi)
    outs = []
    for _ in range(2):
        plan.run()
        outs.append(plan.probs()[0].copy())
    assert np.array_equal(outs[0], outs[1])
    Q = fejer.probabilities(inst.phases, inst.weights, 16)
    assert np.abs(outs[0] - Q).sum() <= L1_BOUND
    assert int(np.argmax(outs[0])) == int(np.argmax(Q))


def test_fused_tensor_core_top_level_falls_back_below_one_tile(q):
    """Fewer than 128 top-level pencils (Nmeas < 11): the plan keeps the fused
    complex64 top level on the CUDA cores, still within the bound."""
    rng = np.random.default_rng(5)
    inst = W.haar_instance(rng, 4, 9, superposition=True)
    plan = q.Plan(4, 9, FP16X2)
    assert plan.query(q.INFO_TC_TOP_LEVEL) == 0
    plan.load(inst.U, inst.psi)
    plan.run()
    P, *_ = plan.probs()
    assert np.abs(P - gates.qpe_probabilities(inst.U, inst.psi, 9)).sum() <= L1_BOUND


def test_c5_split_precisions_vs_fp64_full_size(q):
    """The 34-qubit workload under FP16x2 and TF32x3 (tensor-core top level)
    against the all-FP64 path on the same GPU: L1 over all 2^30 bins within
    1e-6, the same most probable outcome; and sampled bins against the closed
    form."""
    import torch
    inst = W.c5()
    hs = {}
    for prec in (q.FP64, FP16X2, TF32X3):
        plan = q.Plan(inst.nmat, inst.nmeas, prec)
        plan.load(inst.U, inst.psi)
        plan.run()
        out = torch.empty(inst.N, dtype=torch.float64, device="cuda")
        _, am, _, pm = plan.probs(out)
        hs[prec] = (out, am, pm)
        plan.close()
        del plan
        torch.cuda.empty_cache()
    rng = np.random.default_rng(6)
    ys = rng.integers(0, inst.N, 1 << 14)
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=ys)
    for prec in ALL:
        l1 = float((hs[prec][0] - hs[q.FP64][0]).abs().sum().item())
        print(f"C5 precision {prec} vs FP64: L1 {l1:.3e}")
        assert l1 <= L1_BOUND
        assert hs[prec][1] == hs[q.FP64][1]
        got = hs[prec][0][torch.from_numpy(ys).cuda()].cpu().numpy()
        assert np.abs(got - Q).max() <= PROB_TOL[prec]
