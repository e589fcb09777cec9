"""Batched plans (grouped launches across instances) through the C ABI:
every instance must match its single-instance plan and the oracle."""
import numpy as np
import pytest

from oracle import fejer, gates, readout
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


MIXED = [(3, 8), (1, 1), (6, 12), (2, 7), (4, 13), (7, 6), (5, 10), (3, 3), (8, 5), (6, 16), (2, 14), (4, 1)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("flags", [0, 0x2, 0x8])
def test_mixed_batch_matches_oracle_and_single_plans(q, prec, flags):
    rng = np.random.default_rng(77)
    insts = [W.haar_instance(rng, a, b, superposition=True) for a, b in MIXED]
    bp = q.BatchedPlan(MIXED, prec, flags)
    for i, inst in enumerate(insts):
        bp.load(i, inst.U, inst.psi)
    for rep in range(2):  # second run: graph replay / work lists reused
        bp.run()
        for i, inst in enumerate(insts):
            P, am, pa, pm = bp.probs(i)
            ref = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
            assert np.abs(P - ref).max() <= TOL[prec], (i, MIXED[i])
            top2 = np.sort(ref)[-2:]
            if len(ref) > 1 and top2[1] - top2[0] > 10 * TOL[prec]:
                assert am == readout.argmax_lowest(ref)
            assert abs(pm - readout.phase_weighted_mean(ref)) <= (1e-9 if prec == 0 else 2e-5)
            single = q.Plan(inst.nmat, inst.nmeas, prec, flags & 0x8)
            single.load(inst.U, inst.psi)
            single.run()
            P1, am1, _, _ = single.probs()
            assert np.abs(P - P1).max() <= TOL[prec] and am == am1


def test_batched_keep_state(q):
    rng = np.random.default_rng(5)
    shapes = [(2, 6), (4, 9), (6, 5)]
    insts = [W.haar_instance(rng, a, b, superposition=True) for a, b in shapes]
    bp = q.BatchedPlan(shapes, q.FP64, 0x10)
    for i, inst in enumerate(insts):
        bp.load(i, inst.U, inst.psi)
    bp.run()
    for i, inst in enumerate(insts):
        X = bp.state(i)
        ref = gates.qpe_final_state(inst.U, inst.psi, inst.nmeas)
        assert np.abs(X - ref).max() <= 1e-12


def test_batched_requires_every_instance_loaded(q):
    bp = q.BatchedPlan([(2, 4), (3, 5)], q.C64_FP32)
    rng = np.random.default_rng(1)
    inst = W.haar_instance(rng, 2, 4)
    bp.load(0, inst.U, inst.psi)
    with pytest.raises(q.QpeError) as e:
        bp.run()
    assert e.value.status == q.ERR_STATE


def test_c4_full_batch_vs_fejer(q):
    """The 512-instance workload (Nmat 3..10, Nmeas 8..18) in one batched plan,
    replayed as a CUDA graph; every instance's histogram is checked against
    its single-eigenvector Fejer kernel on sampled outcomes plus its peak."""
    insts = W.c4()
    shapes = [(i.nmat, i.nmeas) for i in insts]
    bp = q.BatchedPlan(shapes, q.C64_FP32, q.FLAG_GRAPH)
    for k, inst in enumerate(insts):
        bp.load(k, inst.U, inst.psi)
    bp.run()
    rng = np.random.default_rng(9)
    worst = 0.0
    for k, inst in enumerate(insts):
        P, am, pa, pm = bp.probs(k)
        ys = rng.integers(0, inst.N, 256)
        y0 = int(np.floor(inst.N * inst.phases[0]))
        ys = np.concatenate([ys, [(y0 + j) % inst.N for j in (-1, 0, 1, 2)]])
        Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=ys)
        worst = max(worst, float(np.abs(P[ys] - Q).max()))
        cand = np.array([(y0 + j) % inst.N for j in (-1, 0, 1, 2)])
        Qc = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=cand)
        order = np.argsort(Qc)
        if Qc[order[-1]] - Qc[order[-2]] > 1e-4:
            assert am == cand[order[-1]], k
        assert abs(P.sum() - 1.0) < 1e-4, k
    assert worst <= 1e-5


def test_precision_study_matches_oracle_readout(q):
    """The Sec. 4.2 study on the GPU path: for small Nmeas its per-eigenvector
    estimates equal the oracle's readout of the same histograms."""
    from paper_2507_17175_gb300 import precision_study as ps
    rows, phases = ps.study_rows([4, 6, 9], q.FP64)
    rng = np.random.default_rng(12345)
    V = W.haar_unitary(rng, 16)
    ph = rng.random(16)
    U = W.unitary_from_eigen(V, ph)
    assert np.array_equal(ph, phases)
    for r in rows:
        n = r["nmeas"]
        em, ew = [], []
        for j in range(16):
            P = gates.qpe_probabilities(U, V[:, j], n)
            em.append(readout.phase_max_norm(P))
            ew.append(readout.phase_weighted_mean(P))
        assert abs(r["err_max_norm"] - float(np.mean(np.abs(np.array(em) - ph)))) < 1e-9
        assert abs(r["err_weighted_mean"] - float(np.mean(np.abs(np.array(ew) - ph)))) < 1e-9


# ------------------------------------------------- squaring tile variants
BIG = [(8, 6), (3, 9), (9, 4), (6, 7), (10, 3), (5, 8)]


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("prec", [0, 1])
def test_forced_square_tiles_match_oracle(q, tile, prec, monkeypatch):
    """Every tile variant of the grouped FP64 squaring gives the same
    histograms (FP64 summation order differs only)."""
    monkeypatch.setenv("QPE_SQUARE_TILE", str(tile))
    rng = np.random.default_rng(tile + prec)
    insts = [W.haar_instance(rng, a, b, superposition=True) for a, b in BIG]
    bp = q.BatchedPlan(BIG, prec, 0x8 if prec else 0)
    assert bp.query(q.INFO_SQUARE_TILE) == tile
    for i, inst in enumerate(insts):
        bp.load(i, inst.U, inst.psi)
    bp.run()
    for i, inst in enumerate(insts):
        P, *_ = bp.probs(i)
        ref = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
        assert np.abs(P - ref).max() <= TOL[prec], (tile, BIG[i])


def test_autotuned_plan(q, monkeypatch):
    monkeypatch.delenv("QPE_SQUARE_TILE", raising=False)
    rng = np.random.default_rng(5)
    insts = [W.haar_instance(rng, a, b, superposition=True) for a, b in BIG]
    bp = q.BatchedPlan(BIG, q.C64_FP32, q.FLAG_AUTOTUNE | q.FLAG_GRAPH)
    assert bp.query(q.INFO_SQUARE_TILE) in (8, 16, 32)
    for i, inst in enumerate(insts):
        bp.load(i, inst.U, inst.psi)
    for _ in range(2):
        bp.run()
        for i, inst in enumerate(insts):
            P, *_ = bp.probs(i)
            ref = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
            assert np.abs(P - ref).max() <= TOL[1]
