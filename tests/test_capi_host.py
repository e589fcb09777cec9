"""Host-side checks of the C ABI: the library loads, exports every function
include/qpe.h declares, and qpe_plan (host only, no GPU) validates its
arguments and sizes the workspace. No compute call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def q():
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe
    return qpe


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(qpe_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(q):
    names = header_functions()
    assert "qpe_run" in names and "qpe_plan" in names
    lib = ctypes.CDLL(q.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_plan_sizes_workspace(q):
    st, ws, h = q.plan_workspace(6, 16, q.C64_FP32)
    assert st == q.OK
    N, d = 1 << 16, 64
    # default (fused) plan: powers + histogram, no N x d state buffer
    assert N * 8 + 16 * d * d * 16 <= ws < N * d * 8
    st, ws_plain, h2 = q.plan_workspace(6, 16, q.C64_FP32, q.FLAG_PLAIN if hasattr(q, "FLAG_PLAIN") else 0x8)
    assert st == q.OK and ws_plain >= ws + N * d * 8
    q.LIB.qpe_destroy(h2)
    assert q.LIB.qpe_query(h, q.INFO_STATE_BYTES) == N * d * 8
    assert q.LIB.qpe_query(h, q.INFO_FFT_PASSES) == 2
    q.LIB.qpe_destroy(h)
    st, ws64, h = q.plan_workspace(6, 16, q.FP64)
    assert st == q.OK and q.LIB.qpe_query(h, q.INFO_STATE_BYTES) == N * d * 16
    q.LIB.qpe_destroy(h)


@pytest.mark.parametrize("nmat,nmeas,prec,flags,want", [
    (0, 4, 0, 0, "ERR_ARG"),
    (13, 4, 0, 0, "ERR_ARG"),
    (2, 0, 0, 0, "ERR_ARG"),
    (2, 31, 0, 0, "ERR_ARG"),
    (2, 4, 7, 0, "ERR_ARG"),
    (2, 4, -1, 0, "ERR_ARG"),
    (2, 4, 0, 0x400, "ERR_ARG"),
    (9, 8, 1, 0x100, "OK"),   # QPE_FLAG_SQUARE_TC
    (2, 4, 0, 0x200, "OK"),   # QPE_FLAG_LEVEL_TC (ignored outside its shape)
    (2, 4, 0, 0x80, "OK"),    # QPE_FLAG_AUTOTUNE
    (2, 4, 2, 0, "ERR_UNSUPPORTED"),
    (7, 4, 1, 1, "ERR_UNSUPPORTED"),
    (12, 30, 1, 0, "OK"),
    (1, 1, 0, 0, "OK"),
    (6, 16, 1, 0x40, "OK"),   # QPE_FLAG_CHECK_UNITARY
    (7, 10, 3, 0, "OK"),      # QPE_C64_FP16X2
    (4, 10, 3, 0, "OK"),      # FP16x2 with nmat = 4: fused schedule
    (4, 10, 3, 1, "ERR_UNSUPPORTED"),  # split precisions are not gate by gate
    (6, 16, 0, 0x42, "OK"),
])
def test_plan_validation(q, nmat, nmeas, prec, flags, want):
    st, ws, h = q.plan_workspace(nmat, nmeas, prec, flags)
    assert st == getattr(q, want), q.status_string(st)
    if st == q.OK:
        assert ws > 0
        q.LIB.qpe_destroy(h)
    else:
        assert not h.value


def test_null_arguments(q):
    assert q.LIB.qpe_plan(None, None, None) == q.ERR_ARG
    assert q.LIB.qpe_run(None) == q.ERR_ARG
    assert q.LIB.qpe_destroy(None) == q.OK
    assert q.LIB.qpe_query(None, 1) == -1
    assert q.LIB.qpe_last_error(None) == b"null plan"


def test_calls_before_bind_are_state_errors(q):
    st, ws, h = q.plan_workspace(2, 4, q.FP64)
    assert st == q.OK
    assert q.LIB.qpe_run(h) == q.ERR_STATE
    assert q.LIB.qpe_run_stages(h, 1, 4) == q.ERR_STATE
    assert q.LIB.qpe_sync(h) == q.ERR_STATE
    assert q.LIB.qpe_bind(h, None, ws, None) == q.ERR_WORKSPACE
    assert q.LIB.qpe_bind(h, 0x1001, ws, None) == q.ERR_WORKSPACE  # misaligned: rejected before any CUDA call
    assert q.LIB.qpe_bind(h, 0x1000, ws - 1, None) == q.ERR_WORKSPACE  # too small
    assert b"256-byte" in q.LIB.qpe_last_error(h)
    q.LIB.qpe_destroy(h)


def test_status_strings(q):
    for st in range(9):
        assert q.status_string(st).startswith("QPE_")


def test_plan_batched_validation(q):
    st, ws, h = q.plan_batched_workspace([(3, 8), (10, 18), (1, 1), (6, 12)], q.C64_FP32)
    assert st == q.OK and ws > 0
    assert q.LIB.qpe_query(h, q.INFO_INSTANCES) == 4
    q.LIB.qpe_destroy(h)
    # per-instance layout: at least the sum of the single plans' states
    singles = sum(q.plan_workspace(a, b, q.C64_FP32)[1] for a, b in [(3, 8), (10, 18), (1, 1), (6, 12)])
    assert ws >= 0.9 * singles
    assert q.plan_batched_workspace([], q.C64_FP32)[0] == q.ERR_ARG
    assert q.plan_batched_workspace([(0, 4)], q.C64_FP32)[0] == q.ERR_ARG
    assert q.plan_batched_workspace([(2, 4)], q.C64_FP32, q.FLAG_GATE_SWEEP)[0] == q.ERR_UNSUPPORTED
    st, ws, h = q.plan_batched_workspace([(2, 4)], q.C64_FP32, q.FLAG_TIMING)  # coarse stage split
    assert st == q.OK
    q.LIB.qpe_destroy(h)
    # split precisions: any nmat in a batched plan (nmat <= 6 runs fused in complex64); single plans with
    # nmat <= 4 run fused (FP16x2 at nmat = 4 with the top level on the tensor cores), not gate by gate
    st, ws, h = q.plan_batched_workspace([(3, 8), (8, 10)], q.C64_FP16X2, q.FLAG_SQUARE_TC)
    assert st == q.OK and ws > 0
    q.LIB.qpe_destroy(h)
    for prec in (q.C64_FP16X2, q.C64_TF32X3):
        st, ws, h = q.plan_workspace(4, 12, prec, 0)
        assert st == q.OK and q.LIB.qpe_query(h, q.INFO_TC_TOP_LEVEL) == 1
        q.LIB.qpe_destroy(h)
    st, ws, h = q.plan_workspace(3, 8, q.C64_FP16X2, 0)
    assert st == q.OK and q.LIB.qpe_query(h, q.INFO_TC_TOP_LEVEL) == 0
    q.LIB.qpe_destroy(h)
    assert q.plan_workspace(3, 8, q.C64_FP16X2, q.FLAG_GATE_SWEEP)[0] == q.ERR_UNSUPPORTED


def test_fp64_level_tc_plans(q):
    """QPE_FLAG_LEVEL_TC puts the FP64 top level on the tensor cores only for
    nmat = 4 with at least one 128-pencil tile (per rank) and no kept state;
    the table's digit slabs add 128 KiB to the workspace."""
    st, ws0, h = q.plan_workspace(4, 12, q.FP64, 0)
    assert st == q.OK and q.LIB.qpe_query(h, q.INFO_TC_TOP_LEVEL) == 0
    q.LIB.qpe_destroy(h)
    st, ws1, h = q.plan_workspace(4, 12, q.FP64, q.FLAG_LEVEL_TC)
    assert st == q.OK and q.LIB.qpe_query(h, q.INFO_TC_TOP_LEVEL) == 1
    assert q.LIB.qpe_query(h, q.INFO_TOP_LEVEL_BITS) == 3
    q.LIB.qpe_destroy(h)
    assert ws1 - ws0 >= 128 * 1024
    for nmat, nmeas, prec, flags in [(4, 9, 0, 0), (3, 12, 0, 0), (5, 12, 0, 0), (4, 12, 1, 0), (4, 12, 0, 0x10)]:
        st, _, h = q.plan_workspace(nmat, nmeas, prec, flags | q.FLAG_LEVEL_TC)
        assert st == q.OK and q.LIB.qpe_query(h, q.INFO_TC_TOP_LEVEL) == 0, (nmat, nmeas, prec, flags)
        q.LIB.qpe_destroy(h)
    # the plain schedule (d >= 256): the state rows' digit slices of the largest level
    st, w0, h = q.plan_workspace(8, 12, q.FP64, 0)
    q.LIB.qpe_destroy(h)
    st, w1, h = q.plan_workspace(8, 12, q.FP64, q.FLAG_LEVEL_TC)
    q.LIB.qpe_destroy(h)
    assert w1 - w0 >= 7 * (1 << 11) * 512 * 2
    # sharded: decided on the level's whole pencil count, as unsharded (a rank
    # with fewer than 128 pencils runs one partial tile)
    for world in (4, 8, 16):
        st, _, h = q.plan_shard_workspace(4, 12, q.FP64, q.FLAG_LEVEL_TC, 1, world)
        assert st == q.OK and q.LIB.qpe_query(h, q.INFO_TC_TOP_LEVEL) == 1
        q.LIB.qpe_destroy(h)


def test_fp64_level_tc_batched_workspace(q):
    """Batched FP64 plans with QPE_FLAG_LEVEL_TC: every doubling level of at
    least 128 rows of the d >= 256 instances is one grouped digit-product
    round; the rounds share one row-digit buffer sized by the largest round
    (here level 11 of the (8, 12) instance: 7 digit planes of 2^11 rows x 512
    bf16), besides each qualifying instance's squaring digits. Shapes with no
    such level keep the workspace unchanged."""
    shapes = [(8, 12), (9, 10), (3, 8), (10, 7)]
    st, w0, h = q.plan_batched_workspace(shapes, q.FP64, 0)
    assert st == q.OK
    q.LIB.qpe_destroy(h)
    st, w1, h = q.plan_batched_workspace(shapes, q.FP64, q.FLAG_LEVEL_TC)
    assert st == q.OK
    q.LIB.qpe_destroy(h)
    assert w1 - w0 >= 7 * (1 << 11) * 512 * 2
    # the round buffer is shared: far below the sum over every level and instance
    per_level = sum(7 * (1 << j) * 2 * (1 << a) * 2 for a, b in shapes if a >= 8 for j in range(7, b) if b >= 8)
    assert w1 - w0 < per_level + 64 * 2 ** 20
    for small in ([(3, 8), (7, 12)], [(8, 7), (9, 7)]):
        st, a0, h = q.plan_batched_workspace(small, q.FP64, 0)
        q.LIB.qpe_destroy(h)
        st, a1, h = q.plan_batched_workspace(small, q.FP64, q.FLAG_LEVEL_TC)
        q.LIB.qpe_destroy(h)
        assert st == q.OK and a1 == a0, small


def test_bf16x3_is_refused_everywhere(q):
    """bf16 hi/lo splits (~16 bits) cannot keep the histogram's L1 error within
    1e-6 of FP64, so no plan accepts QPE_C64_BF16X3."""
    for nmat, nmeas in ((5, 8), (8, 10), (12, 20), (3, 8)):
        assert q.plan_workspace(nmat, nmeas, q.C64_BF16X3, 0)[0] == q.ERR_UNSUPPORTED
    assert q.plan_batched_workspace([(3, 8), (8, 10)], q.C64_BF16X3, q.FLAG_SQUARE_TC)[0] == q.ERR_UNSUPPORTED
    assert q.plan_batched_workspace([(3, 8)], q.C64_BF16X3)[0] == q.ERR_UNSUPPORTED
    assert q.plan_shard_workspace(4, 12, q.C64_BF16X3, 0, 0, 2)[0] == q.ERR_UNSUPPORTED


# ------------------------------------------------------------ sharded plans
@pytest.mark.parametrize("nmat,nmeas,prec,flags,rank,world,want", [
    (4, 12, 0, 0, 0, 3, "ERR_ARG"),        # world not a power of two
    (4, 12, 0, 0, 2, 2, "ERR_ARG"),        # rank out of range
    (4, 12, 0, 0, -1, 2, "ERR_ARG"),
    (7, 12, 1, 0, 0, 2, "OK"),               # plain schedule, one exchange
    (4, 12, 1, 0x8, 0, 2, "OK"),
    (5, 12, 3, 0, 1, 2, "OK"),               # FP16x2 gate GEMMs on the tensor cores
    (7, 3, 1, 0, 0, 4, "ERR_UNSUPPORTED"),   # plain form needs N >= world^2
    (7, 12, 1, 0x10, 0, 2, "ERR_UNSUPPORTED"),  # the final state stays distributed
    (7, 12, 1, 0x1, 0, 2, "ERR_UNSUPPORTED"),   # not gate by gate
    (5, 12, 2, 0, 0, 2, "ERR_UNSUPPORTED"),  # BF16x3 is refused
    (4, 3, 0, 0, 0, 2, "ERR_UNSUPPORTED"),   # top level with fewer pencils than ranks
    (4, 12, 0, 0, 1, 2, "OK"),
    (2, 20, 1, 0x10, 7, 8, "OK"),
])
def test_plan_shard_validation(q, nmat, nmeas, prec, flags, rank, world, want):
    st, ws, h = q.plan_shard_workspace(nmat, nmeas, prec, flags, rank, world)
    assert st == getattr(q, want), q.status_string(st)
    if st == q.OK:
        q.LIB.qpe_destroy(h)


def test_shard_workspace_shrinks_with_world(q):
    """A rank holds N / world histogram bins and its share of the level buffers."""
    sizes = []
    for world in (1, 2, 4, 8):
        st, ws, h = q.plan_shard_workspace(4, 24, q.FP64, 0, 0, world)
        assert st == q.OK
        sizes.append(ws)
        q.LIB.qpe_destroy(h)
    st, ws1, h = q.plan_workspace(4, 24, q.FP64)
    q.LIB.qpe_destroy(h)
    assert sizes[0] == ws1
    for a, b in zip(sizes, sizes[1:]):
        assert b < a
    assert sizes[3] < sizes[0] / 4


def test_merge_shard_readouts_rule(q):
    """Larger probability wins; an exact tie goes to the lower outcome in any
    order of the parts; sums add; mismatched shapes and NaN are reported."""
    R = q.ShardReadout
    a = R(5, 0.25, 0.1, 0.4, 4, 1)
    b = R(2, 0.25, 0.05, 0.35, 4, 0)
    c = R(9, 0.10, 0.2, 0.25, 4, 2)
    for parts in ([a, b, c], [c, a, b], [b, c, a]):
        am, pa, pm, tot = q.merge_shard_readouts(parts)
        assert am == 2 and pa == 2 / 16
        assert pm == pytest.approx(0.35) and tot == pytest.approx(1.0)
    with pytest.raises(q.QpeError) as e:
        q.merge_shard_readouts([a, R(2, 0.3, 0.0, 0.1, 5, 0)])
    assert e.value.status == q.ERR_SHAPE
    with pytest.raises(q.QpeError) as e:
        q.merge_shard_readouts([a, R(2, float("nan"), 0.0, 0.1, 4, 0)])
    assert e.value.status == q.ERR_NUMERIC


def test_interleave_shards(q):
    P = np.arange(32, dtype=np.float64)
    parts = [P[r::4] for r in range(4)]
    assert np.array_equal(q.interleave_shards(parts), P)


def test_host_alloc_arguments(q):
    """qpe_host_alloc refuses a zero size and a NULL result pointer; freeing
    NULL is fine (the allocation itself needs a GPU and is tested there)."""
    import ctypes
    p = ctypes.c_void_p()
    assert q.LIB.qpe_host_alloc(0, ctypes.byref(p)) == q.ERR_ARG and not p.value
    assert q.LIB.qpe_host_alloc(64, None) == q.ERR_ARG
    assert q.LIB.qpe_host_free(None) == q.OK
