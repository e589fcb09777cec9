"""The arithmetic of the FP64-grade digit products on the tensor cores, checked
on the CPU with exact integers (independent of the CUDA code).

Both operands are written with a power-of-two scale 2^t (|x| < 2^t) as
x = 2^(t - 55) * sum_{s=0..6} a_s 2^(8 (6 - s)) with balanced integer digits
|a_s| <= 128 (exactly representable in bf16); the digit pairs (s, t) of
weight w = s + t <= 6 are formed, each a product of integers.

The squaring (P_(k+1) = P_k^2, K = 2d):
  * the digits reconstruct every entry to the rounding at 2^(t - 55);
  * per weight w the accumulator covers a window of W_w = 8, 4, 4, 2, 2, 2, 2
    K-blocks of 64 (phases 2, 1, 3, 0, 1, 0, 1, every K-block in exactly one
    window), and its sum stays below 2^24: FP32 accumulation of these
    integers is exact;
  * the drain's int64 sums hi = sum_(w<=2) acc_w 2^(8 (2 - w)) and
    lo = sum_(w>=3) acc_w 2^(8 (6 - w)) stay below 2^44 and 2^54, and
    out = 2^(tau + sigma + 2) (hi 2^-32 + lo 2^-64) is within the FP64
    product's error bound of |A| |B| against an extended-precision product;
    a wrong weight shift or a window that skips a K-block fails it.

The FP64 level (d = 16, K = 32 per pencil row, one scale for the table):
  * a weight's sum over K = 32 stays below 2^22, the int32 groups below 2^31,
    hi and lo below 2^36 and 2^46, the drain's fixed point
    V = 2^26 hi + floor(lo / 2^6) below 2^62 (one signed 64-bit integer), and
    V 2^-26 rounded once to FP64 is within 2^-26 + 1 ulp of hi + 2^-32 lo;
  * T against the extended-precision contraction within the FP64 dot
    product's bound, then twiddle, 8-point DFT and |X|^2 against numpy's;
  * a wrong group shift or a sign slip in the table's real embedding fails.
"""
import numpy as np
import pytest

S, BETA = 7, 8
U64 = np.finfo(np.float64).eps / 2
LOG_WIN = [3, 2, 2, 1, 1, 1, 1]
OFF = [2, 1, 3, 0, 1, 0, 1]


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


def windows(w, kblocks, skip=False):
    """The K-blocks of each window of weight w, as the kernel's phase rule
    groups them (start: kb = 0 or (kb + off) mod win = 0; end: (kb + 1 + off)
    mod win = 0 or the last block)."""
    win = 1 << LOG_WIN[w]
    out, cur = [], []
    for kb in range(kblocks):
        if skip and kb == 1:
            continue  # a planted mistake: one K-block never accumulated
        cur.append(kb)
        if (kb + 1 + OFF[w]) % win == 0 or kb + 1 == kblocks:
            out.append(cur)
            cur = []
    return out


def squaring(P, shift_err=False, skip=False):
    d = P.shape[0]
    E = embed(P)                 # 2d x 2d, rows are the first operand
    B = E[:, :d].T.copy()        # d x 2d, rows = columns of [Re P ; Im P] (second operand, K-major)
    tau = exponents(E, 1)
    sig = exponents(B, 1)
    Ad = digits(E, tau[:, None])
    Bd = digits(B, sig[:, None])
    assert np.abs(Ad).max() <= 128 and np.abs(Bd).max() <= 128  # bf16-exact integers
    kblocks = 2 * d // 64
    hi = np.zeros((2 * d, d), dtype=np.int64)
    lo = np.zeros((2 * d, d), dtype=np.int64)
    for w in range(S):
        assert (w + 1) * (1 << LOG_WIN[w]) < 16
        wins = windows(w, kblocks, skip)
        if not skip:
            assert sorted(kb for win in wins for kb in win) == list(range(kblocks))
        for win in wins:
            acc = np.zeros((2 * d, d), dtype=np.int64)
            for kb in win:
                k0 = kb * 64
                for s in range(w + 1):
                    acc += Ad[s][:, k0:k0 + 64] @ Bd[w - s][:, k0:k0 + 64].T
            assert np.abs(acc).max() < 2 ** 24, (w, win)  # exact in the FP32 accumulator
            sh = 8 * ((2 if w <= 2 else 6) - w)
            if shift_err and w == 4:
                sh += 8
            if w <= 2:
                hi += acc << sh
            else:
                lo += acc << sh
    assert np.abs(hi).max() < 2 ** 44 and np.abs(lo).max() < 2 ** 54
    val = hi.astype(np.float64) * 2.0 ** -32 + lo.astype(np.float64) * 2.0 ** -64
    C = np.ldexp(val, tau[:, None] + sig[None, :] + 2)
    return E, B, tau, Ad, C


@pytest.mark.parametrize("d,seed", [(64, 0), (128, 1), (256, 2)])
def test_squaring_digits_windows_and_fold(d, seed):
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2 * d)
    P[3] *= 1e-6  # one row far below the others: its own scale keeps its precision
    E, B, tau, Ad, C = squaring(P)
    # reconstruction: the digits carry x to the rounding at 2^(t - 55)
    w = (2.0 ** (BETA * (S - 1 - np.arange(S))))[:, None, None]
    recon = np.ldexp((Ad * w).sum(0), (tau[:, None] - (S * BETA - 1)))
    assert np.all(np.abs(recon - E) <= np.ldexp(0.5, tau[:, None] - (S * BETA - 1)))
    # an FP64 GEMM is within about K u |A| |B|; the scheme lands far inside that
    ref = E.astype(np.longdouble) @ B.astype(np.longdouble).T
    bound = np.abs(E) @ np.abs(B).T
    assert np.all(np.abs(C.astype(np.longdouble) - ref) <= 4 * np.finfo(np.float64).eps * bound + 1e-300)
    Pc = C[:d] + 1j * C[d:]
    assert np.abs(Pc - P @ P).max() <= 1e-14 * np.abs(P).max() ** 2 * d


@pytest.mark.parametrize("plant", ["shift", "skip"])
def test_squaring_planted_mistakes_fail(plant):
    rng = np.random.default_rng(9)
    d = 64
    P = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2 * d)
    _, _, _, _, C = squaring(P, shift_err=plant == "shift", skip=plant == "skip")
    Pc = C[:d] + 1j * C[d:]
    assert np.abs(Pc - P @ P).max() > 1e-12


def test_extreme_digits_bound():
    """Digits -127 then six -128 (the GPU test's matrix): every window sum of
    the squaring stays below 2^24 even then."""
    from fractions import Fraction
    c = -(127 * Fraction(2) ** 48 + 128 * sum(Fraction(2) ** (8 * j) for j in range(6))) / Fraction(2) ** 55
    d = 256
    P = np.full((d, d), float(c), dtype=np.complex128)
    _, _, _, Ad, C = squaring(P)
    assert np.all(Ad[:, :d, :d] == np.array([-127, -128, -128, -128, -128, -128, -128])[:, None, None])
    assert np.abs(C[:d] - float(c * c * d)).max() <= 4 * U64 * abs(float(c * c * d))


# ---------------------------------------------------------------- FP64 level
def level_T(Z, M, group_err=False, sign_err=False):
    """The level kernel's T[p][m][i] for pencils Z (P x 16 complex) and the
    table M (8 x 16 x 16 complex, T = M Z), modelled step by step."""
    Pn = Z.shape[0]
    A = np.empty((Pn, 32))
    A[:, 0::2], A[:, 1::2] = Z.real, Z.imag                  # k2 = 2 k + c'
    B = np.empty((256, 32))
    for i in range(16):
        for m in range(8):
            for c in range(2):
                n = 16 * i + 2 * m + c
                re, im = M[m, i].real, M[m, i].imag
                if c == 0:
                    B[n, 0::2], B[n, 1::2] = re, (im if sign_err else -im)
                else:
                    B[n, 0::2], B[n, 1::2] = im, re
    emax = np.array([max(int(np.frexp(np.abs(r).max())[1]) + 1022 if np.abs(r).max() > 0 else 0, 0) for r in A])
    tau = np.where(emax == 0, 0, emax - 1022)
    sig = int(exponents(B.reshape(1, -1), 1)[0])
    Ad = digits(A, tau[:, None])
    Bd = digits(B, np.full((256, 1), sig))
    acc = [sum(Ad[s] @ Bd[w - s].T for s in range(w + 1)) for w in range(S)]   # P x 256 each
    assert max(np.abs(a).max() for a in acc) < 2 ** 22
    g0, g1 = acc[0], acc[1] * 256 + acc[2]
    g2, g3 = acc[3] * 256 + acc[4], acc[5] * 256 + acc[6]
    assert max(np.abs(g).max() for g in (g0, g1, g2, g3)) < 2 ** 31
    hi = (g0 << 16) + g1
    lo = (g2 << (8 if group_err else 16)) + g3
    assert np.abs(hi).max() < 2 ** 36 and np.abs(lo).max() < 2 ** 46
    V = (hi << 26) + (lo >> 6)                               # the drain's 62-bit fixed point (floor)
    assert np.abs(V).max() < 2 ** 62
    raw = V.astype(np.float64) * 2.0 ** -26                  # one rounding to nearest even
    exact = hi.astype(np.longdouble) + lo.astype(np.longdouble) * np.longdouble(2.0) ** -32
    assert np.all(np.abs(raw - exact) <= 2.0 ** -26 + U64 * np.abs(exact))
    Tr = np.ldexp(raw, (tau + sig - 30)[:, None]).reshape(Pn, 16, 8, 2)  # [p][i][m][c]
    return (Tr[..., 0] + 1j * Tr[..., 1]).transpose(0, 2, 1)             # [p][m][i]


def _level_inputs(seed):
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((40, 16)) + 1j * rng.standard_normal((40, 16))) * np.exp(rng.uniform(-20, 20, 40))[:, None]
    Z[5] = 0.0
    Z[6] *= 1e-200
    V = np.linalg.qr(rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16)))[0]
    M = np.stack([np.linalg.matrix_power(V, m) for m in range(8)])
    return Z, M


def test_fp64_level_contraction_and_epilogue():
    Z, M = _level_inputs(3)
    T = level_T(Z, M)
    Tref = np.einsum("mik,pk->pmi", M.astype(np.clongdouble), Z.astype(np.clongdouble))
    bound = np.einsum("mik,pk->pmi", np.abs(M), np.abs(Z))
    assert np.all(np.abs(T - Tref) <= 8 * U64 * bound + 1e-300)
    # twiddle, 8-point DFT over m (exp(-2 pi i m y / 8)) and |X|^2 summed over i
    ya = np.arange(40)
    w = np.exp(-2j * np.pi * np.outer(ya, np.arange(8)) / 2 ** 12)
    X = np.fft.fft(T * w[:, :, None], axis=1)
    Xref = np.fft.fft(Tref.astype(np.complex128) * w[:, :, None], axis=1)
    hist, href = (np.abs(X) ** 2).sum(2), (np.abs(Xref) ** 2).sum(2)
    assert np.all(np.abs(hist - href) <= 1e-13 * href.max(axis=1, keepdims=True) + 1e-300)
    assert np.all(hist[5] == 0.0)


@pytest.mark.parametrize("plant", ["group", "sign"])
def test_fp64_level_planted_mistakes_fail(plant):
    Z, M = _level_inputs(4)
    T = level_T(Z, M, group_err=plant == "group", sign_err=plant == "sign")
    Tref = np.einsum("mik,pk->pmi", M, Z)
    assert np.abs(T - Tref).max() > 1e-10 * np.abs(Tref).max()
