"""The arithmetic of the FP64-grade squaring on the tensor cores, checked on the
CPU with exact integers (independent of the CUDA code).

The scheme writes every entry x of a row (column) with scale 2^t, |x| < 2^t,
as 2^(t - 55) * sum_{s=1..7} a_s 2^(8 (7 - s)) with balanced integer digits
|a_s| <= 128 (exactly representable in bf16), forms the digit products of
weight u = s + t <= 8 as integer matrix products (exact), and folds
sum_u acc_u 2^(-8 u) 2^(tau + sigma + 2). Checked here:
  * the digits reconstruct every entry to the rounding at 2^(t - 55);
  * every 64-element K-block's sum of one weight stays below 2^23 (the tensor
    cores' FP32 accumulation of integers is then exact);
  * the folded product is within the FP64 product's error bound of
    |A| |B| against an extended-precision reference.
"""
import numpy as np
import pytest

S, BETA = 7, 8


def exponents(m, axis):
    """t with max |m| along `axis` < 2^t (zero lines get a floor)."""
    mx = np.abs(m).max(axis=axis)
    t = np.full(mx.shape, -900, dtype=np.int64)
    nz = mx > 0
    t[nz] = np.floor(np.log2(mx[nz])).astype(np.int64) + 1
    return t


def digits(x, t):
    """Balanced base-2^8 digits (most significant first) of x at scale 2^t."""
    F = np.rint(np.ldexp(x, S * BETA - 1 - t)).astype(np.int64)
    out = np.zeros((S,) + x.shape, dtype=np.int64)
    for s in range(S - 1, 0, -1):
        r = F & 255
        r = np.where(r >= 128, r - 256, r)
        out[s] = r
        F = (F - r) // 256
    out[0] = F
    return out


def embed(P):
    return np.block([[P.real, -P.imag], [P.imag, P.real]])


@pytest.mark.parametrize("d,seed", [(32, 0), (64, 1), (128, 2)])
def test_digits_reconstruct_and_products_are_exact(d, seed):
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2 * d)
    P[3] *= 1e-6  # one row far below the others: its own scale keeps its precision
    E = embed(P)                 # 2d x 2d, rows are the first operand
    B = E[:, :d].T.copy()        # d x 2d, rows = columns of [Re P ; Im P] (second operand, K-major)
    tau = exponents(E, 1)
    sig = exponents(B, 1)
    Ad = digits(E, tau[:, None])
    Bd = digits(B, sig[:, None])
    assert np.abs(Ad).max() <= 128 and np.abs(Bd).max() <= 128  # bf16-exact integers

    # reconstruction: the digits carry x to the rounding at 2^(t - 55)
    w = (2.0 ** (BETA * (S - 1 - np.arange(S))))[:, None, None]
    recon = np.ldexp((Ad * w).sum(0), (tau[:, None] - (S * BETA - 1)))
    assert np.all(np.abs(recon - E) <= np.ldexp(0.5, tau[:, None] - (S * BETA - 1)))

    # per weight and 64-element K-block: exact integer sums below 2^23
    K = 2 * d
    acc = {}
    for u in range(2, S + 2):
        tot = np.zeros((2 * d, d), dtype=np.int64)
        for s in range(1, u):
            t = u - s
            for k0 in range(0, K, 64):
                blk = Ad[s - 1][:, k0:k0 + 64] @ Bd[t - 1][:, k0:k0 + 64].T
                assert np.abs(blk).max() < 2 ** 22, (u, s, k0)
                tot += blk
        # one weight's block sum (all its pairs) is what one accumulator holds
        for k0 in range(0, K, 64):
            wsum = sum(Ad[s - 1][:, k0:k0 + 64] @ Bd[u - s - 1][:, k0:k0 + 64].T for s in range(1, u))
            assert np.abs(wsum).max() < 2 ** 23
        assert np.abs(tot).max() < 2 ** 31  # the int32 sum over K of the drain warps
        acc[u] = tot

    # fold and compare with an extended-precision product
    val = np.zeros((2 * d, d))
    for u in range(2, S + 2):
        val += acc[u].astype(np.float64) * 2.0 ** (-BETA * u)
    C = np.ldexp(val, tau[:, None] + sig[None, :] + 2)
    El = E.astype(np.longdouble)
    Bl = B.astype(np.longdouble)
    ref = El @ Bl.T
    bound = np.abs(E) @ np.abs(B).T
    err = np.abs(C.astype(np.longdouble) - ref)
    # an FP64 GEMM is within about K u |A| |B|; the scheme lands far inside that
    assert np.all(err <= 4 * np.finfo(np.float64).eps * bound + 1e-300)
    # and it reproduces the complex square
    Pc = C[:d] + 1j * C[d:]
    assert np.abs(Pc - P @ P).max() <= 1e-14 * np.abs(P).max() ** 2 * d
