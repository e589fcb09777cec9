"""QPE_FLAG_SQUARE_TC: U^(2^k) squarings on the tcgen05 tensor cores with
FP64-grade accuracy (balanced 8-bit digits with power-of-two row / column
scales, exact integer accumulation of 28 bf16 digit products).

Pins: the powers against the FP64 CUDA-core squaring and numpy's
matrix_power; exact results for a signed permutation matrix (every product
is exact in FP64, so the emulation must reproduce it bit for bit); the
histograms against the oracle and the closed form; a NaN reported.
"""
import numpy as np
import pytest

from oracle import fejer, gates
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


def powers(q, U, nmeas, flags, prec=0):
    nmat = int(np.log2(U.shape[0]))
    plan = q.Plan(nmat, nmeas, prec, flags | q.FLAG_PLAIN)
    plan.load(U, np.eye(U.shape[0], dtype=np.complex128)[:, 0])
    plan.run_stages(q.STAGE_POWERS, q.STAGE_POWERS)
    return [plan.power(k) for k in range(nmeas)]


@pytest.mark.parametrize("nmat,nmeas", [(8, 7), (9, 6), (10, 5)])
def test_powers_match_fp64_squaring(q, nmat, nmeas):
    rng = np.random.default_rng(nmat)
    U = W.haar_unitary(rng, 1 << nmat)
    tc = powers(q, U, nmeas, q.FLAG_SQUARE_TC)
    fp = powers(q, U, nmeas, 0)
    ref = U.copy()
    d = 1 << nmat
    for k in range(nmeas):
        # both sides round each squaring at ~sqrt(d) u relative to |A||B|; errors double per step
        tol = (2.0 ** k) * 64 * np.sqrt(d) * U64
        assert np.abs(tc[k] - fp[k]).max() <= tol, k
        assert np.abs(tc[k] - ref).max() <= tol, k
        ref = ref @ ref


def test_signed_permutation_is_exact(q):
    """Entries in {0, +-1, +-i}: every product and sum is exact, so the digit
    products must reproduce the FP64 squares bit for bit."""
    rng = np.random.default_rng(3)
    d = 256
    perm = rng.permutation(d)
    phase = np.array([1, -1, 1j, -1j])[rng.integers(0, 4, d)]
    U = np.zeros((d, d), dtype=np.complex128)
    U[np.arange(d), perm] = phase
    tc = powers(q, U, 6, q.FLAG_SQUARE_TC)
    ref = U.copy()
    for k in range(6):
        assert np.array_equal(tc[k], ref), k
        ref = ref @ ref


@pytest.mark.parametrize("nmat", [8, 10, 12])
def test_extreme_digits_accumulate_exactly(q, nmat):
    """Every entry c = -(127 2^48 + 128 sum_(j<6) 2^(8j)) 2^-55 (in [0.5, 1), so
    its row and column scale is 2^0), whose balanced base-256 digits are -127
    then six times -128: the digit products are +2^14 (16256 or 16129 with a
    leading digit) and the integer sums of the accumulation windows reach the
    largest value the windows allow (up to 14 * 2^20, against 2^24). The square
    of c J (J all ones) is c^2 d J; the formed digit pairs miss it only by the
    pairs dropped below 2^-53. One unit lost in a window sum of weight w moves
    the result by 2^(-8 w - 14 - nmat) of itself: above the tolerance of 4 ulps
    for the weights w <= 3 (window sums up to 12 * 2^20); the lower weights
    lie below FP64 resolution."""
    from fractions import Fraction
    d = 1 << nmat
    c = -(127 * Fraction(2) ** 48 + 128 * sum(Fraction(2) ** (8 * j) for j in range(6))) / Fraction(2) ** 55
    assert float(c) == c and 0.5 <= -c < 1  # exact in FP64
    U = np.full((d, d), float(c), dtype=np.complex128)
    tc = powers(q, U, 2, q.FLAG_SQUARE_TC)
    exact = float(c * c * d)
    assert np.all(tc[1].imag == 0.0)
    assert np.abs(tc[1].real - exact).max() <= 4 * U64 * abs(exact)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_end_to_end_against_oracle(q, prec, tol):
    rng = np.random.default_rng(11)
    inst = W.haar_instance(rng, 8, 9, superposition=True)
    plan = q.Plan(8, 9, prec, q.FLAG_SQUARE_TC)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, *_ = plan.probs()
    ref = gates.qpe_probabilities(inst.U, inst.psi, 9)
    assert np.abs(P - ref).max() <= tol


@pytest.mark.parametrize("prec", [1, 3])
def test_c3_with_tensor_core_squaring(q, prec):
    """Nmat = 12, Nmeas = 20 (32 qubits), squarings on the tensor cores, gates
    in complex64 on the CUDA cores or as FP16x2 products on the tensor cores:
    the whole histogram against the Fejer closed form (max-abs, and for the
    split precision the L1 bound 1e-6)."""
    inst = W.c3()
    plan = q.Plan(inst.nmat, inst.nmeas, prec, q.FLAG_SQUARE_TC | q.FLAG_TIMING)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, *_ = plan.probs()
    st = plan.stage_times()
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    err = np.abs(P - Q)
    print(f"prec {prec}: squaring {st[0]:.1f} ms, max-abs {err.max():.3e} L1 {err.sum():.3e}")
    assert err.max() <= 1e-5
    if prec == 3:
        assert err.sum() <= 1e-6
    assert am == int(np.argmax(Q))


def test_nan_is_reported(q):
    inst = W.haar_instance(np.random.default_rng(2), 8, 4)
    U = inst.U.copy()
    U[5, 7] = np.nan
    plan = q.Plan(8, 4, q.C64_FP32, q.FLAG_SQUARE_TC)
    plan.load(U, inst.psi)
    plan.run()
    with pytest.raises(q.QpeError) as e:
        plan.probs()
    assert e.value.status == q.ERR_NUMERIC


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_mix_with_tensor_core_squaring(q, prec):
    """Instances with d >= 256 square on the tensor cores, the others in the
    grouped FP64 launches, in one plan."""
    shapes = [(8, 7), (3, 9), (9, 5), (6, 8), (10, 4), (2, 6)]
    rng = np.random.default_rng(21 + prec)
    insts = [W.haar_instance(rng, a, b, superposition=True) for a, b in shapes]
    bp = q.BatchedPlan(shapes, prec, q.FLAG_SQUARE_TC | q.FLAG_GRAPH)
    for i, inst in enumerate(insts):
        bp.load(i, inst.U, inst.psi)
    for _ in range(2):
        bp.run()
        for i, inst in enumerate(insts):
            P, *_ = bp.probs(i)
            ref = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
            assert np.abs(P - ref).max() <= (1e-10 if prec == 0 else 1e-5), shapes[i]
