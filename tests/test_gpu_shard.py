"""Sharded plans (qpe_plan_shard) through the C ABI.

Rank r of `world` computes the outcomes y = r (mod world) of one problem.
On one GPU the ranks run one after another (their kernels never wait on each
other, so this is the same computation a multi-GPU job performs), and the
interleaved slices must equal the unsharded plan's histogram bit for bit (the
same arithmetic on the same numbers) and the oracle's within the path's
tolerance; the merged readout must equal the unsharded readout. A second test
runs two processes on the GPU that gather over a gloo process group through
host buffers, the exchange a multi-GPU job would do over NCCL.
"""
import os
import socket

import numpy as np
import pytest

from oracle import gates, readout
from paper_2507_17175_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {0: 1e-10, 1: 1e-5, 3: 1e-5}
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEEP = 0x10


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe
    return qpe


@pytest.mark.parametrize("prec,nmat,nmeas,world", [(0, 2, 10, 2), (1, 2, 10, 4), (0, 4, 14, 8), (1, 6, 12, 2),
                                                   (1, 1, 18, 4), (0, 3, 16, 2), (1, 4, 13, 16), (3, 4, 14, 2),
                                                   (3, 4, 13, 4)])
def test_shards_equal_unsharded_plan_and_oracle(q, prec, nmat, nmeas, world):
    rng = np.random.default_rng(1000 * world + 10 * nmat + nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    ref_state = gates.qpe_final_state(inst.U, inst.psi, nmeas)
    ref = gates.probabilities(ref_state)
    full = q.Plan(nmat, nmeas, prec)
    full.load(inst.U, inst.psi)
    full.run()
    Pf, amf, paf, pmf = full.probs()
    parts, reads = [], []
    amp_tol = max(1e-12, 16 * (1 << nmeas) * np.finfo(np.float64).eps / 2) if prec == 0 else 3e-6
    flags = KEEP if prec != 3 else 0  # the tensor-core top level writes the histogram only
    for r in range(world):
        sp = q.ShardedPlan(nmat, nmeas, prec, flags, r, world)
        assert prec != 3 or sp.query(q.INFO_TC_TOP_LEVEL) == 1
        sp.load(inst.U, inst.psi)
        sp.run()
        P, am, pa, pm = sp.probs()
        assert am % world == r
        parts.append(P.copy())
        reads.append(sp.shard_readout())
        if flags & KEEP:
            X = sp.state()  # this rank's rows of the final state, y = r + world j
            assert np.abs(X - ref_state[r::world]).max() <= amp_tol
        sp.close()
    hist = q.interleave_shards(parts)
    assert np.array_equal(hist, Pf)
    assert np.abs(hist - ref).max() <= TOL[prec]
    am, pa, pm, tot = q.merge_shard_readouts(reads)
    assert am == amf and pa == paf
    assert abs(pm - pmf) <= 1e-12
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * TOL[prec]:
        assert am == readout.argmax_lowest(ref)
    assert abs(tot - ref.sum()) <= (1e-10 if prec == 0 else 1e-5)
    if prec == 3:
        assert np.abs(hist - ref).sum() <= 1e-6


def test_c5_complex64_two_shards_full_size(q):
    """The 34-qubit workload split over two ranks: the interleaved halves equal
    the unsharded histogram exactly (all 2^30 bins, compared on the device)."""
    import torch
    inst = W.c5()
    full = q.Plan(inst.nmat, inst.nmeas, q.C64_FP32)
    full.load(inst.U, inst.psi)
    full.run()
    Pf = torch.empty(inst.N, dtype=torch.float64, device="cuda")
    _, amf, _, pmf = full.probs(Pf)
    full.close()
    del full
    torch.cuda.empty_cache()
    parts, reads = [], []
    for r in range(2):
        sp = q.ShardedPlan(inst.nmat, inst.nmeas, q.C64_FP32, 0, r, 2)
        sp.load(inst.U, inst.psi)
        sp.run()
        P = torch.empty(inst.N // 2, dtype=torch.float64, device="cuda")
        sp.probs(P)
        parts.append(P)
        reads.append(sp.shard_readout())
        sp.close()
        del sp
        torch.cuda.empty_cache()
    assert torch.equal(q.interleave_shards(parts), Pf)
    am, _, pm, _ = q.merge_shard_readouts(reads)
    # the complex64 readout sums each thread's bins in FP32 (Kahan); the merge
    # adds the same partials in another order: a few units of 2^-24 apart
    assert am == amf and abs(pm - pmf) <= 1e-7


@pytest.mark.parametrize("prec,nmat,nmeas,world,flags", [(0, 7, 8, 2, 0), (1, 7, 10, 4, 0), (1, 3, 12, 4, 0x8),
                                                         (0, 2, 9, 8, 0x8), (3, 8, 10, 2, 0), (1, 5, 14, 2, 0x8),
                                                         (3, 7, 12, 4, 0), (0, 8, 10, 2, 0x200)])
def test_plain_shards_with_one_exchange(q, prec, nmat, nmeas, world, flags):
    """The plain schedule split over `world` ranks by the low measurement bits
    of the rows: local controlled gates and QFT^-1 passes, one all-to-all of
    N / world^2 rows per pair of ranks (done here by device copies between the
    ranks' buffers), the cross-rank DFT; against the oracle."""
    import torch
    rng = np.random.default_rng(77 * world + 5 * nmat + nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    plans = [q.ShardedPlan(nmat, nmeas, prec, flags, r, world) for r in range(world)]
    for sp in plans:
        sp.load(inst.U, inst.psi)
        sp.run()
    bufs = [sp.buffers() for sp in plans]
    assert all(b[0] is not None for b in bufs)
    nb = bufs[0][0].numel() // world
    assert nb == (inst.N // world // world) * inst.d * (16 if prec == 0 else 8)
    torch.cuda.synchronize()
    for s_ in range(world):
        for r in range(world):
            bufs[s_][1][r * nb:(r + 1) * nb].copy_(bufs[r][0][s_ * nb:(s_ + 1) * nb])
    torch.cuda.synchronize()
    parts, reads = [], []
    for sp in plans:
        sp.finish()
        P, am, _, _ = sp.probs()
        parts.append(P.copy())
        reads.append(sp.shard_readout())
    hist = q.interleave_shards(parts)
    assert np.abs(hist - ref).max() <= TOL[prec]
    if prec == 3:
        assert np.abs(hist - ref).sum() <= 1e-6
    am, pa, pm, tot = q.merge_shard_readouts(reads)
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * TOL[prec]:
        assert am == readout.argmax_lowest(ref)
    assert abs(pm - readout.phase_weighted_mean(ref)) <= (1e-9 if prec == 0 else 2e-5)
    assert abs(tot - ref.sum()) <= (1e-10 if prec == 0 else 1e-5)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q, nmat, nmeas, prec, flags, seed):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2507_17175_gb300 import qpe
    rng = np.random.default_rng(seed)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    plan = qpe.ShardedPlan(nmat, nmeas, prec, flags, rank, world, device="cuda:0")
    plan.load(inst.U, inst.psi)
    plan.run_exchange(dist)  # the plain form's all-to-all goes through host buffers
    hist, am, pa, pm = plan.gather(dist)  # all-gather through host buffers
    out_q.put((rank, hist.numpy(), am, pa, pm))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("prec,nmat,flags", [(0, 3, 0), (1, 3, 0), (1, 7, 0), (0, 3, 0x8)])
def test_two_processes_over_gloo(q, prec, nmat, flags):
    """Two processes share the GPU, each the plan of one rank; the plain form
    exchanges its rows by an all-to-all and both gather the histogram, all
    over a gloo group through host buffers (the kernels of the two ranks never
    wait on each other)."""
    import torch.multiprocessing as mp
    nmeas, seed, world = 12, 17, 2
    ctx = mp.get_context("spawn")
    out_q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out_q, nmat, nmeas, prec, flags, seed))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([out_q.get(timeout=300) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    rng = np.random.default_rng(seed)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    for rank, hist, am, pa, pm in res:
        assert np.abs(hist - ref).max() <= TOL[prec]
        assert am == readout.argmax_lowest(ref)
        assert abs(pm - readout.phase_weighted_mean(ref)) <= (1e-9 if prec == 0 else 2e-5)
    assert np.array_equal(res[0][1], res[1][1])
