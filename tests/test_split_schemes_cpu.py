"""The operand splits of the split-precision tensor-core schemes, on the CPU.

x = hi + lo with hi = round(x) and lo = round(x - hi) in the tensor type:
bf16 and tf32 keep 8 and 11 significant bits per part, fp16 11 bits but only
5 exponent bits, which is why FP16x2 scales each state row by a power of two
so that its largest entry lies in [2^14, 2^15) (and U's embedding by 2^14)
before splitting. Checked here: the split's reconstruction error per scheme,
the three-product approximation hi.hi + hi.lo + lo.hi of a product, and that
the scaled fp16 parts stay out of the subnormal range where the unscaled ones
would not.
"""
import numpy as np
import pytest


def round_bits(x, bits):
    """Round float32 values to `bits` significant bits (nearest, ties to even)
    by integer arithmetic on the bit pattern (bf16: 8, tf32: 11)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    drop = 24 - bits
    half = np.uint64(1) << np.uint64(drop - 1)
    lsb = (u >> np.uint64(drop)) & np.uint64(1)
    u = (u + half - np.uint64(1) + lsb) >> np.uint64(drop) << np.uint64(drop)
    return u.astype(np.uint32).view(np.float32)


def split(x, kind):
    x = np.asarray(x, dtype=np.float32)
    if kind == "bf16":
        hi = round_bits(x, 8)
        lo = round_bits(x - hi, 8)
    elif kind == "tf32":
        hi = round_bits(x, 11)
        lo = round_bits(x - hi, 11)
    else:  # fp16 (numpy's IEEE half)
        hi = x.astype(np.float16).astype(np.float32)
        lo = (x - hi).astype(np.float16).astype(np.float32)
    return hi, lo


BITS = {"bf16": 16, "tf32": 22, "fp16": 22}


def test_round_bits_matches_float16_significand():
    # 11 significant bits of a normal float equal IEEE half rounding in range
    x = np.random.default_rng(0).uniform(0.5, 60000, 10000).astype(np.float32)
    assert np.array_equal(round_bits(x, 11), x.astype(np.float16).astype(np.float32))


@pytest.mark.parametrize("kind", ["bf16", "tf32", "fp16"])
def test_split_reconstruction(kind):
    rng = np.random.default_rng(1)
    x = rng.uniform(0.5, 1.0, 20000).astype(np.float32) * np.where(rng.random(20000) < 0.5, -1, 1)
    if kind == "fp16":
        x = x * np.float32(2 ** 14)  # the scaled range FP16x2 works in
    hi, lo = split(x, kind)
    rel = np.abs((hi.astype(np.float64) + lo) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -(BITS[kind] + 1)  # half an ulp of the lo part
    assert rel.max() > 2.0 ** -(BITS[kind] + 6)    # and not more bits than the scheme claims


@pytest.mark.parametrize("kind", ["bf16", "tf32", "fp16"])
def test_three_product_approximation(kind):
    """A real-embedded complex row times U's embedding (K = 2d) by the three
    products, against FP64: relative error at the split's bit count."""
    rng = np.random.default_rng(2)
    d = 256
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)))
    E = np.block([[Q.real, -Q.imag], [Q.imag, Q.real]]).astype(np.float32)
    a = (rng.standard_normal(2 * d) / np.sqrt(2 * d)).astype(np.float32)
    sa = sb = 1.0
    if kind == "fp16":
        e = int(np.floor(np.log2(np.abs(a).max())))
        sa = 2.0 ** (14 - e)   # row max into [2^14, 2^15)
        sb = 2.0 ** 14
    ah, al = split(a * np.float32(sa), kind)
    bh, bl = split(E * np.float32(sb), kind)
    ah, al, bh, bl = (t.astype(np.float64) for t in (ah, al, bh, bl))
    approx = (bh @ ah + bl @ ah + bh @ al) / (sa * sb)
    exact = E.astype(np.float64) @ a.astype(np.float64)
    scale = np.abs(E.astype(np.float64)) @ np.abs(a.astype(np.float64))
    rel = np.abs(approx - exact) / scale
    assert rel.max() <= 4 * 2.0 ** -BITS[kind]


def test_fp16_scaling_keeps_lo_normal():
    """Entries of a normalised 4096-dimensional state are ~1/64: unscaled, the
    fp16 lo part falls below the normal range (2^-14) and loses bits; scaled
    rows keep it normal."""
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(8192) / np.sqrt(8192)).astype(np.float32)
    _, lo_raw = split(a, "fp16")
    tiny = 2.0 ** -14
    assert np.mean((np.abs(lo_raw) < tiny) & (lo_raw != 0)) > 0.5  # mostly subnormal without scaling
    e = int(np.floor(np.log2(np.abs(a).max())))
    _, lo = split(a * np.float32(2.0 ** (14 - e)), "fp16")
    big = np.abs(a) > np.abs(a).max() * 2.0 ** -10  # entries within 10 binades of the row max
    assert np.all((np.abs(lo[big]) >= tiny) | (lo[big] == 0))
