"""The plain histogram's blocked digit reversal (rows of at most 64 bytes),
modelled on the CPU: the tiles cover every outcome y exactly once, each tile
reads its rows as runs of consecutive positions and writes its bins as runs
of consecutive y, for the QFT^-1 pass splits the plans use.

Positions follow the decimation-in-frequency passes: with y's digits
d_0 (lowest, logr[0] bits) .. d_last (highest), the row of y sits at
position p = sum_i d_i 2^(n - logr[0] - .. - logr[i]), y's lowest digit in
p's highest bits."""
import numpy as np
import pytest


def pass_split(n, max_bits=9):
    passes = (n + max_bits - 1) // max_bits
    return [n // passes + (1 if i < n % passes else 0) for i in range(passes)]


def y_to_pos(logr, n, y):
    p, rem, sh = 0, n, 0
    for lr in logr:
        rem -= lr
        p |= ((y >> sh) & ((1 << lr) - 1)) << rem
        sh += lr
    return p


def tiles(logr, n):
    """The kernel's enumeration: per tile, the (y, position) pairs in read
    order (k fastest) and the y in write order (the 32 low values fastest)."""
    lb = logr[-1]
    K = (1 << lb) if lb < 7 else 128
    kc_count = (1 << lb) // K
    ntiles = kc_count << (n - 5 - lb)
    for t in range(ntiles):
        kc, mbits = t % kc_count, t // kc_count
        ybase = mbits << 5
        reads = [(ybase + e // K + ((kc * K + e % K) << (n - lb))) for e in range(32 * K)]
        writes = [(ybase + (e & 31) + ((kc * K + (e >> 5)) << (n - lb))) for e in range(32 * K)]
        yield K, reads, writes


@pytest.mark.parametrize("n", [10, 12, 14, 17, 19, 22])
def test_blocked_digit_reversal_covers_and_runs(n):
    logr = pass_split(n)
    assert len(logr) >= 2 and logr[0] >= 5  # the kernel's condition for the blocked form
    seen = np.zeros(1 << n, dtype=np.int64)
    for K, reads, writes in tiles(logr, n):
        assert sorted(reads) == sorted(writes)
        for y in writes:
            seen[y] += 1
        pos = [y_to_pos(logr, n, y) for y in reads]
        for r in range(32):  # each of the 32 low values: K consecutive positions
            run = pos[r * K:(r + 1) * K]
            assert run == list(range(run[0], run[0] + K))
        for k in range(K):   # each of the K: 32 consecutive bins
            run = writes[k * 32:(k + 1) * 32]
            assert run == list(range(run[0], run[0] + 32))
    assert np.all(seen == 1)


def test_position_map_is_the_pass_order():
    """y_to_pos agrees with digit-reversing a plain radix-2^b index (one pass
    size b): the mixed-radix reversal the QFT^-1 passes leave."""
    n, b = 12, 6
    for y in range(1 << n):
        lo, hi = y & 63, y >> 6
        assert y_to_pos([b, b], n, y) == (lo << 6) | hi
