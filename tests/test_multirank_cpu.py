"""Multi-rank logic on CPU ranks (gloo, world size 2 and 4, 127.0.0.1).

* bench.py's replica aggregation: the job time is the slowest rank's, the
  throughput counts every rank's runs.
* The library's sharded-plan host path (qpe_plan_shard): each rank holds the
  outcomes y = rank (mod world) compactly, as a sharded plan's qpe_probs
  returns them (here cut from the oracle's histogram, since these ranks have
  no GPU); qpe.gather_shards all-gathers and interleaves the slices and merges
  the ranks' readout partials with the library's qpe_merge_shard_readouts.
* The row-sharded layout of the statevector across ranks (each rank owns the
  rows whose lowest measurement bit equals its rank): local controlled gates
  and a local DFT over the high bits, then one exchange of N/4 rows per rank
  for the cross-rank radix-2 stage, and a gather of the histogram. Emulated
  with numpy on CPU ranks and checked against the oracle's histogram.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _aggregate_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    dist = _init(rank, world, port)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    value, slowest = bench.aggregate(world, 10, local_ms, "cpu")
    q.put((rank, value, slowest))
    dist.destroy_process_group()


def _run(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda t: t[0])


def test_bench_replica_aggregation():
    res = _run(_aggregate_worker, 2)
    for rank, value, slowest in res:
        assert slowest == 150.0
        assert value == pytest.approx(2 * 10 / 0.150)


def _shard_worker(rank, world, port, q, nmat, nmeas, seed):
    import sys
    sys.path.insert(0, ROOT)
    dist = _init(rank, world, port)
    import torch
    from paper_2507_17175_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    N, d = inst.N, inst.d
    # local rows m = rank + 2 m_hi, each 2^(-n/2) U^m psi (controlled gates of its set bits)
    P = [np.array(inst.U)]
    for _ in range(1, nmeas):
        P.append(P[-1] @ P[-1])
    rows = np.empty((N // 2, d), dtype=np.complex128)
    for mh in range(N // 2):
        m = rank + 2 * mh
        v = inst.psi.copy()
        for k in range(nmeas):
            if (m >> k) & 1:
                v = P[k] @ v
        rows[mh] = v / np.sqrt(N)
    # local DFT over the high bits: A_rank[y'] = sum_mh w_(N/2)^(mh y') rows[mh]
    A = np.fft.fft(rows, axis=0)
    # exchange: rank r keeps y' in [r N/4, (r+1) N/4) and needs the other rank's A there
    q4 = N // 4
    mine = slice(rank * q4, (rank + 1) * q4)
    theirs = slice((1 - rank) * q4, (2 - rank) * q4)
    send = torch.from_numpy(np.ascontiguousarray(A[theirs]))
    recv = torch.empty_like(send)
    reqs = [dist.isend(send, 1 - rank), dist.irecv(recv, 1 - rank)]
    for r_ in reqs:
        r_.wait()
    A_other = recv.numpy()
    A0, A1 = (A[mine], A_other) if rank == 0 else (A_other, A[mine])
    yp = np.arange(rank * q4, (rank + 1) * q4)
    w = np.exp(-2j * np.pi * yp / N)[:, None]
    X_lo = (A0 + w * A1) / np.sqrt(N)   # outcomes y'
    X_hi = (A0 - w * A1) / np.sqrt(N)   # outcomes y' + N/2
    P_lo = np.sum(np.abs(X_lo) ** 2, axis=1)
    P_hi = np.sum(np.abs(X_hi) ** 2, axis=1)
    part = torch.from_numpy(np.concatenate([P_lo, P_hi]))
    parts = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(parts, part)
    hist = np.zeros(N)
    for r in range(world):
        p = parts[r].numpy()
        hist[r * q4:(r + 1) * q4] = p[:q4]
        hist[N // 2 + r * q4:N // 2 + (r + 1) * q4] = p[q4:]
    q.put((rank, hist, inst.U, inst.psi))
    dist.destroy_process_group()


@pytest.mark.parametrize("nmat,nmeas", [(2, 6), (3, 9)])
def test_row_sharded_exchange_matches_oracle(nmat, nmeas):
    from oracle import gates
    res = _run(_shard_worker, 2, nmat, nmeas, 31)
    hist0 = res[0][1]
    assert np.array_equal(hist0, res[1][1])
    ref = gates.qpe_probabilities(res[0][2], res[0][3], nmeas)
    assert np.abs(hist0 - ref).max() < 1e-12


def _gather_worker(rank, world, port, q, nmat, nmeas, seed):
    import sys
    sys.path.insert(0, ROOT)
    dist = _init(rank, world, port)
    import torch
    from oracle import gates
    from paper_2507_17175_gb300 import qpe, workloads as W
    rng = np.random.default_rng(seed)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    P = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    N = 1 << nmeas
    local = np.ascontiguousarray(P[rank::world])  # what this rank's plan returns
    ys = np.arange(rank, N, world)
    j = int(np.argmax(local))
    part = qpe.ShardReadout(int(ys[j]), float(local[j]), float(np.sum(local * ys) / N), float(local.sum()),
                            nmeas, rank)
    hist, am, pa, pm = qpe.gather_shards(dist, torch.from_numpy(local), part)
    q.put((rank, hist.numpy(), am, pa, pm, P))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nmat,nmeas", [(2, 3, 9), (4, 2, 10)])
def test_sharded_histogram_gather_and_readout_merge(world, nmat, nmeas):
    from oracle import readout
    res = _run(_gather_worker, world, nmat, nmeas, 7)
    P = res[0][5]
    for rank, hist, am, pa, pm, _ in res:
        assert np.array_equal(hist, P)
        assert am == readout.argmax_lowest(P)
        assert pa == readout.phase_max_norm(P)
        assert abs(pm - readout.phase_weighted_mean(P)) <= 1e-12
