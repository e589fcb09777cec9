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
  * a weight's sum over K = 32 stays below 2^22 and reads back exactly
    through the FP32 magic-number addition; the drain's fixed point
    W = floor(E / 2^10), E = sum_w acc_w 2^(8 (6 - w)), equals the exact
    floor and stays below 2^57 + 2;
  * T against the extended-precision contraction within the FP64 dot
    product's bound; the Q61 twiddle products (split at bit 31) below 2^58,
    the integer 8-point DFT below 2^61, and X converted to FP64 (rounded to
    nearest) against numpy's FFT of the exact T within a few units of
    rounding, |X|^2 likewise;
  * a wrong weight shift, a sign slip in the table's real embedding, in the
    twiddle's cross term or in the DFT's rotation fails.
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
MAGIC = 0x4B400000            # bits of 1.5 * 2^23
Q61 = 1 << 61
C_Q61 = 1630477228166597777   # round(2^61 / sqrt(2))


def q61(x):
    """round(x 2^61), halves away from zero, exactly (x a float64)."""
    from fractions import Fraction
    f = Fraction(float(x)) * Q61
    r = int(abs(f) + Fraction(1, 2))
    return r if f >= 0 else -r


def split31(v):
    return v >> 31, v & 0x7FFFFFFF


def tw_fix(wr, wi, qr, qi, plant=None):
    """(wr + i wi)(qr + i qi) 2^-61 as the drain forms it (operands split at
    bit 31, the low x low products dropped, the middle sums floored)."""
    rh, rl = split31(wr)
    ih, il = split31(wi)
    qrh, qrl = split31(qr)
    qih, qil = split31(qi)
    sr = rh * qrl + rl * qrh - ih * qil - il * qih
    si = rh * qil + rl * qih + (ih * qrl if plant != "tw_sign" else -ih * qrl) + il * qrh
    assert abs(sr) < 2 ** 63 and abs(si) < 2 ** 63
    return 2 * (rh * qrh - ih * qih) + (sr >> 30), 2 * (rh * qih + ih * qrh) + (si >> 30)


def rot_fix(x):
    xh, xl = split31(x)
    ch, cl = split31(C_Q61)
    return 2 * xh * ch + ((xh * cl + xl * ch) >> 30)


def dft8_fix(x, plant=None):
    """The drain's 8-point DFT on integers (x: 8 complex as [re, im] pairs)."""
    x = [list(v) for v in x]
    for p in range(4):
        (ur, ui), (vr, vi) = x[p], x[p + 4]
        x[p] = [ur + vr, ui + vi]
        dr, di = ur - vr, ui - vi
        if p == 0:
            x[4] = [dr, di]
        elif p == 1:
            x[5] = [rot_fix(dr + di), rot_fix(di - dr)]
        elif p == 2:
            x[6] = [di, -dr]
        else:
            x[7] = [rot_fix(di - dr), -rot_fix(dr + di)] if plant != "rot" else [rot_fix(dr - di), -rot_fix(dr + di)]
    for g in (0, 4):
        for p in range(2):
            (ur, ui), (vr, vi) = x[g + p], x[g + p + 2]
            x[g + p] = [ur + vr, ui + vi]
            x[g + p + 2] = [ur - vr, ui - vi] if p == 0 else [ui - vi, vr - ur]
    for g in range(0, 8, 2):
        (ur, ui), (vr, vi) = x[g], x[g + 1]
        x[g], x[g + 1] = [ur + vr, ui + vi], [ur - vr, ui - vi]
    x[1], x[4] = x[4], x[1]
    x[3], x[6] = x[6], x[3]
    return x


def fix_to_f64(v, e2):
    """v 2^e2 in FP64: the conversion rounded to nearest (even), the power of
    two exact; below 2^-1022: 0."""
    r = float(np.ldexp(float(v), e2))
    return 0.0 if abs(r) < 2.0 ** -1022 else r


def level_fix(Z, M, ya, N, plant=None):
    """The level kernel for pencils Z (P x 16 complex) and the table M
    (8 x 16 x 16 complex, T = M Z), modelled step by step with exact
    integers: returns T (as the fixed point W carries it) and, per pencil,
    X[y][i] in FP64 and the bins sum_i |X[y][i]|^2."""
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
                    B[n, 0::2], B[n, 1::2] = re, (im if plant == "sign" else -im)
                else:
                    B[n, 0::2], B[n, 1::2] = im, re
    emax = np.array([max(int(np.frexp(np.abs(r).max())[1]) + 1022 if np.abs(r).max() > 0 else 0, 0) for r in A])
    tau = np.where(emax == 0, 0, emax - 1022)
    sig = int(exponents(B.reshape(1, -1), 1)[0])
    Ad = digits(A, tau[:, None])
    Bd = digits(B, np.full((256, 1), sig))
    acc = [sum(Ad[s] @ Bd[w - s].T for s in range(w + 1)) for w in range(S)]   # P x 256 each
    assert max(np.abs(a).max() for a in acc) < 2 ** 22
    # the accumulators read back as ints: FP32 acc + 1.5 2^23, bits - MAGIC
    for a in acc:
        f = a.astype(np.float32) + np.float32(12582912.0)
        assert np.array_equal(f.view(np.int32).astype(np.int64) - MAGIC, a)
    sh = [38, 30, 22, 14, 6]
    if plant == "group":
        sh[3] = 15
    W = ((acc[5] * 256 + acc[6]) >> 10)
    for w in range(5):
        W = W + (acc[w] << sh[w])
    E = sum(acc[w].astype(object) * (1 << (8 * (6 - w))) for w in range(S))
    if plant is None:
        assert np.all(W.astype(object) == E // 1024)        # floor(E / 2^10)
        # the kernel's form: magic bits b = acc + M, the offsets folded into
        # one constant modulo 2^64
        b = [(a + MAGIC).astype(np.uint64) for a in acc]
        low = ((b[5] * 256 + b[6] - 0x8B400000) & 0xFFFFFFFF).astype(np.int64)
        low = np.where(low >= 2 ** 31, low - 2 ** 32, low) >> 10
        kmw = (MAGIC * sum(1 << s_ for s_ in (38, 30, 22, 14, 6))) % 2 ** 64
        assert kmw == 0xE2E2E2E2D0000000
        with np.errstate(over="ignore"):
            Wk = low.astype(np.uint64) - np.uint64(kmw)
            for w_, sh_ in zip(range(5), (38, 30, 22, 14, 6)):
                Wk = Wk + b[w_] * np.uint64(1 << sh_)
        assert np.array_equal(Wk.view(np.int64), W)
    assert np.abs(W).max() < 2 ** 57 + 2
    T = np.ldexp(W.astype(np.float64), (tau + sig - 52)[:, None]).reshape(Pn, 16, 8, 2)
    T = (T[..., 0] + 1j * T[..., 1]).transpose(0, 2, 1)     # [p][m][i] (exact up to FP64 rounding of W)
    Wr = W.reshape(Pn, 16, 8, 2)
    X = np.zeros((Pn, 8, 16), dtype=np.complex128)
    for p in range(Pn):
        tw = np.exp(-2j * np.pi * (np.arange(8) * int(ya[p]) % N) / N)
        q = [(q61(t.real), q61(t.imag)) for t in tw]
        for i in range(16):
            x = [[int(Wr[p, i, m, 0]), int(Wr[p, i, m, 1])] for m in range(8)]
            for m in range(1, 8):
                x[m] = list(tw_fix(x[m][0], x[m][1], *q[m], plant=plant))
                assert max(abs(x[m][0]), abs(x[m][1])) < 2 ** 58
            X8 = dft8_fix(x, plant)
            assert max(max(abs(v[0]), abs(v[1])) for v in X8) < 2 ** 61
            e2 = int(tau[p] + sig - 52)
            for y in range(8):
                X[p, y, i] = complex(fix_to_f64(X8[y][0], e2), fix_to_f64(X8[y][1], e2))
    hist = (X.real ** 2 + X.imag ** 2).sum(2)
    return T, X, hist, np.ldexp(1.0, tau + sig - 52)


def _level_inputs(seed):
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((24, 16)) + 1j * rng.standard_normal((24, 16))) * np.exp(rng.uniform(-20, 20, 24))[:, None]
    Z[5] = 0.0
    Z[6] *= 1e-200
    V = np.linalg.qr(rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16)))[0]
    M = np.stack([np.linalg.matrix_power(V, m) for m in range(8)])
    ya = rng.integers(0, 1 << 12, 24)
    return Z, M, ya, 1 << 15


def _level_ref(Z, M, ya, N):
    Tref = np.einsum("mik,pk->pmi", M.astype(np.clongdouble), Z.astype(np.clongdouble))
    w = np.exp(-2j * np.pi * (np.outer(ya, np.arange(8)) % N) / N)
    Xref = np.fft.fft(Tref.astype(np.complex128) * w[:, :, None], axis=1)
    return Tref, Xref


def test_fp64_level_contraction_and_epilogue():
    Z, M, ya, N = _level_inputs(3)
    T, X, hist, unit = level_fix(Z, M, ya, N)
    Tref, Xref = _level_ref(Z, M, ya, N)
    # the contraction within the FP64 dot product's bound plus the fixed
    # point's floor (one unit of 2^(tau + sigma - 52), 2^-57 of the pencil's
    # bound |T| < 2^(tau + sigma + 5)) and the FP64 rounding of W
    bound = np.einsum("mik,pk->pmi", np.abs(M), np.abs(Z))
    assert np.all(np.abs(T - Tref) <= 8 * U64 * bound + 2 * unit[:, None, None] + 1e-300)
    # twiddle and 8-point DFT in fixed point against numpy's FFT of the exact
    # T: within a few units of rounding of each pencil's largest |X|
    scale = np.abs(Xref).max(axis=(1, 2), keepdims=True)
    assert np.all(np.abs(X - Xref) <= 64 * U64 * scale + 1e-300)
    href = (np.abs(Xref) ** 2).sum(2)
    assert np.all(np.abs(hist - href) <= 256 * U64 * href.max(axis=1, keepdims=True) + 1e-300)
    assert np.all(hist[5] == 0.0)


@pytest.mark.parametrize("plant", ["group", "sign", "tw_sign", "rot"])
def test_fp64_level_planted_mistakes_fail(plant):
    Z, M, ya, N = _level_inputs(4)
    T, X, hist, _ = level_fix(Z, M, ya, N, plant=plant)
    _, Xref = _level_ref(Z, M, ya, N)
    assert np.abs(X - Xref).max() > 1e-10 * np.abs(Xref).max()


def test_producer_digits_from_biased_bytes():
    """The level producer's digits: byte 6 - s of F + B (B = 128 sum 2^(8 s),
    the top digit from bits 48..56) minus 128 equals the balanced digit s of
    F, for |F| <= 2^55 (the ends included); each digit is exact as the float
    (2^23 + d) - (2^23 + 128) and in its bf16 upper half."""
    B = 0x80808080808080
    assert B == 128 * sum(1 << (8 * s) for s in range(S))
    rng = np.random.default_rng(11)
    Fs = [int(v) for v in rng.integers(-(2 ** 55), 2 ** 55, 2000)]
    Fs += [2 ** 55, -(2 ** 55), 0, -1, 1, 127, -128, 128, 2 ** 48 * 128, -(2 ** 48) * 128 - 1]
    for F in Fs:
        U = F + B
        assert 0 <= U < 2 ** 57
        got = [(U >> 48) - 128] + [((U >> (8 * (6 - s))) & 255) - 128 for s in range(1, S)]
        x = np.ldexp(float(F), -55)  # t = 0
        want = digits(np.array([x]), np.array([0]))[:, 0]
        if abs(F) < 2 ** 53:        # x carries F exactly
            assert got == [int(v) for v in want], F
        assert sum(g * 256 ** (6 - s) for s, g in enumerate(got)) == F
        for g in got:
            f = np.float32(np.uint32(0x4B000000 | (g + 128)).view(np.float32)) - np.float32(8388736.0)
            assert f == g and (np.uint32(np.float32(f).view(np.uint32)) & 0xFFFF) == 0
