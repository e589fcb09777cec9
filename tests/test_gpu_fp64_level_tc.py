"""QPE_FLAG_LEVEL_TC: the FP64 fused schedule's top level (d = 16, 8-point top
level) with its contraction on the tcgen05 tensor cores by exact digit
products (7 balanced 8-bit digits per operand, the Ozaki scheme) and the
twiddles, DFT, |X|^2 and readout in FP64.

Pins: the oracle's histogram and readout within the FP64 tolerance; the
CUDA-core FP64 plan on the same input within a few units of rounding; the
analytic family's exact phases (delta peaks); sharded plans equal the
unsharded one bit for bit; the full 34-qubit workload against the closed form.
"""
import numpy as np
import pytest

from oracle import fejer, gates, readout
from paper_2507_17175_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U64 = np.finfo(np.float64).eps / 2


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe
    return qpe


def _run(q, inst, flags):
    plan = q.Plan(inst.nmat, inst.nmeas, q.FP64, flags)
    plan.load(inst.U, inst.psi)
    plan.run()
    out = plan.probs()
    on_tc = plan.query(q.INFO_TC_TOP_LEVEL)
    plan.close()
    return out, on_tc


@pytest.mark.parametrize("nmeas", [10, 11, 12, 13, 15, 17])
def test_against_oracle_and_cuda_cores(q, nmeas):
    rng = np.random.default_rng(40 + nmeas)
    inst = W.haar_instance(rng, 4, nmeas, superposition=True)
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    (P, am, pa, pm), on_tc = _run(q, inst, q.FLAG_LEVEL_TC)
    assert on_tc == 1
    assert np.abs(P - ref).max() <= 1e-10
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 1e-9:
        assert am == readout.argmax_lowest(ref)
    assert abs(pm - readout.phase_weighted_mean(ref)) <= 1e-9
    assert abs(P.sum() - ref.sum()) <= 1e-10
    # the CUDA-core FP64 path: both are FP64-accurate, so they agree to a few
    # units of rounding of the largest bin
    (P1, am1, _, pm1), on_tc1 = _run(q, inst, 0)
    assert on_tc1 == 0
    assert np.abs(P - P1).max() <= 64 * U64 * max(P1.max(), 1e-300) * np.sqrt(1 << nmeas)
    assert am == am1 and abs(pm - pm1) <= 1e-12


def test_flag_ignored_outside_its_shape(q):
    """Other target sizes, too few pencils for one tile, or complex64: the
    flag changes nothing (the CUDA-core schedule runs, same histogram)."""
    for nmat, nmeas, prec in [(3, 12, 0), (5, 12, 0), (4, 8, 0), (4, 12, 1)]:
        rng = np.random.default_rng(nmat * 100 + nmeas)
        inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
        plans = []
        for flags in (0, q.FLAG_LEVEL_TC):
            plan = q.Plan(nmat, nmeas, prec, flags)
            plan.load(inst.U, inst.psi)
            plan.run()
            plans.append((plan.probs(), plan.query(q.INFO_TC_TOP_LEVEL)))
            plan.close()
        assert plans[1][1] == 0
        assert np.array_equal(plans[0][0][0], plans[1][0][0])


@pytest.mark.parametrize("j", [0, 5, 15])
def test_analytic_family_exact_phases(q, j):
    """phi_j = j / 16 and psi = x_j: the distribution is a delta at
    y = j 2^(Nmeas - 4) (Sec. 3)."""
    nmeas = 12
    inst = W.analytic_instance(4, nmeas, j)
    (P, am, pa, pm), on_tc = _run(q, inst, q.FLAG_LEVEL_TC)
    assert on_tc == 1
    y0 = j << (nmeas - 4)
    assert am == y0
    assert abs(P[y0] - 1.0) <= 1e-10
    P[y0] = 0.0
    assert np.abs(P).max() <= 1e-10


@pytest.mark.parametrize("world,nmeas", [(2, 12), (4, 14), (8, 13)])
def test_shards_equal_unsharded(q, world, nmeas):
    rng = np.random.default_rng(7 * world + nmeas)
    inst = W.haar_instance(rng, 4, nmeas, superposition=True)
    (Pf, amf, paf, pmf), _ = _run(q, inst, q.FLAG_LEVEL_TC)
    parts, reads = [], []
    for r in range(world):
        sp = q.ShardedPlan(4, nmeas, q.FP64, q.FLAG_LEVEL_TC, r, world)
        assert sp.query(q.INFO_TC_TOP_LEVEL) == 1
        sp.load(inst.U, inst.psi)
        sp.run()
        parts.append(sp.probs()[0].copy())
        reads.append(sp.shard_readout())
        sp.close()
    assert np.array_equal(q.interleave_shards(parts), Pf)
    am, pa, pm, tot = q.merge_shard_readouts(reads)
    assert am == amf and pa == paf and abs(pm - pmf) <= 1e-12


def test_c5_full_size_against_closed_form(q):
    """Nmat = 4, Nmeas = 30 (34 qubits), the benchmark's FP64 workload with the
    flag: sampled bins and the peaks against the Fejer closed form, to the
    input's FP64 floor (as the CUDA-core FP64 path is held to)."""
    import torch
    inst = W.c5(30)
    plan = q.Plan(inst.nmat, inst.nmeas, q.FP64, q.FLAG_LEVEL_TC)
    assert plan.query(q.INFO_TC_TOP_LEVEL) == 1
    plan.load(inst.U, inst.psi)
    plan.run()
    out = torch.empty(inst.N, dtype=torch.float64, device="cuda")
    _, am, pa, pm = plan.probs(out)
    N = inst.N
    rng = np.random.default_rng(5)
    y0 = np.floor(N * inst.phases).astype(np.int64)
    ys = np.concatenate([rng.integers(0, N, 1 << 16), y0 % N, (y0 + 1) % N])
    got = out[torch.from_numpy(ys).cuda()].cpu().numpy()
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=ys)
    tol = max(1e-10, 2 * N * U64 * np.sqrt(inst.d))
    assert np.abs(got - Q).max() <= tol
    cand = np.unique(np.concatenate([(y0 + k) % N for k in (-1, 0, 1, 2)]))
    Qc = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=cand)
    order = np.argsort(Qc)
    if Qc[order[-1]] - Qc[order[-2]] > 10 * tol:
        assert am == cand[order[-1]]
    assert abs(float(out.sum().item()) - 1.0) <= 1e-8
    del out
    plan.close()
    del plan
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,flags,nmeas", [(0, 0x200, 20), (0, 0x202, 20), (1, 0x2, 18), (0, 0x200, 13)])
def test_host_histogram_copied_during_the_run(q, prec, flags, nmeas):
    """qpe_set_host_histogram: after each run the host buffer holds the
    run's histogram bit for bit (the FP64 tensor-core top level copies it in
    eight parts while it computes; other paths copy after the run), across
    graph replays and a changed input; qpe_probs into that buffer returns the
    same readout without copying again."""
    import torch
    rng = np.random.default_rng(nmeas + flags)
    a = W.haar_instance(rng, 4, nmeas, superposition=True)
    b = W.haar_instance(rng, 4, nmeas, superposition=True)
    plan = q.Plan(4, nmeas, prec, flags)
    host = q.host_array(1 << nmeas)
    plan.set_host_histogram(host)
    dev = torch.empty(1 << nmeas, dtype=torch.float64, device="cuda")
    for inst in (a, b, a):
        host[...] = -1.0
        plan.load(inst.U, inst.psi)
        plan.run()
        plan.sync()
        ref = plan.probs(dev)
        assert np.array_equal(host, dev.cpu().numpy())
        got = plan.probs(host)
        assert got[1:] == ref[1:]
    plan.set_host_histogram(None)
    host[...] = -1.0
    plan.run()
    plan.sync()
    assert np.all(host == -1.0)  # no copy once unset
    with pytest.raises(q.QpeError) as e:
        plan.set_host_histogram(np.zeros(1 << nmeas))  # pageable memory
    assert e.value.status == q.ERR_ARG
    plan.close()


def test_host_histogram_of_a_shard(q):
    rng = np.random.default_rng(5)
    inst = W.haar_instance(rng, 4, 14, superposition=True)
    parts = []
    for r in range(2):
        sp = q.ShardedPlan(4, 14, q.FP64, q.FLAG_LEVEL_TC, r, 2)
        host = q.host_array(1 << 13)
        sp.set_host_histogram(host)
        sp.load(inst.U, inst.psi)
        sp.run()
        P = sp.probs()[0]
        assert np.array_equal(host, P)
        parts.append(P.copy())
        sp.close()
    ref = gates.qpe_probabilities(inst.U, inst.psi, 14)
    assert np.abs(q.interleave_shards(parts) - ref).max() <= 1e-10


# ------------------------------------------- the plain schedule's FP64 gates
@pytest.mark.parametrize("nmat,nmeas", [(8, 9), (9, 8), (10, 8)])
def test_plain_gate_rows_on_tensor_cores(q, nmat, nmeas):
    """QPE_FLAG_LEVEL_TC on the plain schedule (d >= 256): the doubling levels of
    at least 128 rows are exact digit products; row m after the gates equals
    the oracle's 2^(-n/2) U^m psi to FP64 accuracy."""
    rng = np.random.default_rng(5 * nmat + nmeas)
    U = W.haar_unitary(rng, 1 << nmat)
    psi = W.random_state(rng, 1 << nmat, 1)[:, 0]
    plan = q.Plan(nmat, nmeas, q.FP64, q.FLAG_LEVEL_TC)
    plan.load(U, psi)
    plan.run_stages(q.STAGE_POWERS, q.STAGE_SWEEP)
    S = plan.state()
    ref = gates.qpe_after_sweeps(U, psi, nmeas)
    tol = 1e-12 * np.abs(psi).max() * (1 << nmat) / np.sqrt(1 << nmeas)
    assert np.abs(S - ref).max() <= tol
    plan.close()


@pytest.mark.parametrize("nmat,nmeas", [(8, 12), (9, 10), (10, 9)])
def test_plain_fp64_gates_against_oracle_and_fp64_units(q, nmat, nmeas):
    rng = np.random.default_rng(17 * nmat + nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    (P, am, pa, pm), _ = _run(q, inst, q.FLAG_LEVEL_TC)
    assert np.abs(P - ref).max() <= 1e-10
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 1e-9:
        assert am == readout.argmax_lowest(ref)
    assert abs(pm - readout.phase_weighted_mean(ref)) <= 1e-9
    (P1, am1, _, pm1), _ = _run(q, inst, 0)
    assert np.abs(P - P1).max() <= 1e-12 and am == am1


def test_c3_fp64_gates_on_tensor_cores_against_closed_form(q):
    """C3 (Nmat = 12, Nmeas = 20, 32 qubits, 64 GiB complex128 state) with the
    doubling GEMMs as digit products (and the squaring on the tensor cores):
    every bin against the closed form to the input's FP64 floor."""
    import torch
    inst = W.c3()
    plan = q.Plan(inst.nmat, inst.nmeas, q.FP64, q.FLAG_LEVEL_TC | q.FLAG_SQUARE_TC)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, pa, pm = plan.probs()
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    tol = max(1e-10, 2 * inst.N * U64 * np.sqrt(inst.d))
    assert np.abs(P - Q).max() <= tol
    order = np.argsort(Q)
    if Q[order[-1]] - Q[order[-2]] > 10 * tol:
        assert am == order[-1]
    assert abs(pm - readout.phase_weighted_mean(Q)) <= 1e-8
    plan.close()
    del plan
    torch.cuda.empty_cache()


# ------------------------------------------- batched plans: gate rounds
BATCH = [(8, 9), (3, 8), (9, 10), (10, 8), (4, 12), (8, 12), (2, 7), (9, 8), (8, 7), (10, 10)]


@pytest.mark.parametrize("flags", [0x200, 0x200 | 0x2, 0x200 | 0x100 | 0x2])
def test_batched_fp64_gate_rounds(q, flags):
    """A batched FP64 plan with QPE_FLAG_LEVEL_TC: every level of at least 128
    rows of the d >= 256 instances is one grouped digit-product round across
    them; (8, 7) stays on the FP64 units and the fused instances are as
    before. Each instance against the oracle, and against the batched plan
    without the flag within a few units of rounding; twice (graph replay)."""
    rng = np.random.default_rng(91)
    insts = [W.haar_instance(rng, a, b, superposition=True) for a, b in BATCH]
    bp = q.BatchedPlan(BATCH, q.FP64, flags)
    ref_plan = q.BatchedPlan(BATCH, q.FP64, flags & ~0x200)
    for i, inst in enumerate(insts):
        bp.load(i, inst.U, inst.psi)
        ref_plan.load(i, inst.U, inst.psi)
    ref_plan.run()
    for rep in range(2):
        bp.run()
        for i, inst in enumerate(insts):
            P, am, pa, pm = bp.probs(i)
            ref = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
            assert np.abs(P - ref).max() <= 1e-10, (i, BATCH[i])
            top2 = np.sort(ref)[-2:]
            if top2[1] - top2[0] > 1e-9:
                assert am == readout.argmax_lowest(ref)
            assert abs(pm - readout.phase_weighted_mean(ref)) <= 1e-9
            P1, am1, _, _ = ref_plan.probs(i)
            assert np.abs(P - P1).max() <= 1e-12 and am == am1, (i, BATCH[i])
