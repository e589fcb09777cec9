"""Pins of the CPU oracle against things other than itself.

Each pin checks the oracle against a library routine, a closed form proven
from the paper's definitions, brute force on tiny inputs, or the paper's own
exact-phase claim (Sec. 3). ``test_planted_mistakes`` then plants plausible
mistakes in the oracle (a flipped sign, a transposed operand, a wrong bit, a
dropped normalisation, ...) and checks that at least one pin fails for each.
"""
import os

import numpy as np
import pytest

from oracle import circuit_matrix, fejer, gates, readout
from paper_2507_17175_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- pin checks
# Each returns the worst error it saw; the tests assert on it and the
# planted-mistake test asserts that it grows.

def pin_qft_vs_numpy_fft(ns=range(1, 8)):
    """QFT^-1 gate sequence == numpy.fft.fft(., axis=0, norm="ortho"), the
    matrix exp(-2 pi i m y / N) / sqrt(N)."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for n in ns:
        S = W.random_state(rng, 1 << n, 3)
        ref = np.fft.fft(S, axis=0, norm="ortho")
        gates.qft_inverse(S)
        worst = max(worst, float(np.abs(S - ref).max()))
    return worst


def pin_full_matrix(cases=((1, 1), (2, 2), (3, 1), (2, 3), (4, 2), (3, 3), (6, 2), (5, 3))):
    """Gate-by-gate final state == whole-circuit matrix applied to |0> psi
    (<= 8 qubits), random unitary U and random normalised psi."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for n, nmat in cases:
        d = 1 << nmat
        U = W.haar_unitary(rng, d)
        psi = W.random_state(rng, d, 1)[:, 0]
        psi /= np.linalg.norm(psi)
        a = gates.qpe_final_state(U, psi, n)
        b = circuit_matrix.qpe_final_state(U, psi, n)
        worst = max(worst, float(np.abs(a - b).max()))
    return worst


def pin_exact_phase_c1():
    """C1: phases k_j / 64 exactly representable in 6 bits, psi = V[:,0]:
    probability 1 at y = k_0, every other bin 0 (Sec. 3)."""
    inst = W.c1()
    P = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
    target = np.zeros_like(P)
    target[int(inst.meta["k"][0])] = 1.0
    return float(np.abs(P - target).max())


def pin_fejer_vs_gates(n=9, nmat=3, seed=5):
    """Gate-by-gate histogram == sum_j |c_j|^2 F_n(phi_j - y/N) for a
    superposition input with non-representable phases."""
    rng = np.random.default_rng(seed)
    inst = W.haar_instance(rng, nmat, n, superposition=True)
    P = gates.qpe_probabilities(inst.U, inst.psi, n)
    Q = fejer.probabilities(inst.phases, inst.weights, n)
    return float(np.abs(P - Q).max())


def pin_fejer_closed_vs_sum():
    """Closed form sin^2(pi N d)/(N^2 sin^2(pi d)) == |N^-1 sum_m e^{2 pi i m d}|^2
    term by term."""
    worst = 0.0
    rng = np.random.default_rng(3)
    for n in (1, 3, 6, 10):
        N = 1 << n
        for delta in list(rng.random(5)) + [0.0, 1.0 / N, 0.5, 3.0 / N + 1e-9]:
            a = fejer.fejer(n, np.array([N * delta]))[0]
            b = fejer.fejer_bruteforce(n, delta)
            worst = max(worst, abs(a - b))
    return worst


def pin_norm(n=7, nmat=2):
    """sum_y P(y) == ||psi||^2 for an unnormalised psi (every gate is unitary)."""
    rng = np.random.default_rng(13)
    U = W.haar_unitary(rng, 1 << nmat)
    psi = 1.7 * W.random_state(rng, 1 << nmat, 1)[:, 0]
    P = gates.qpe_probabilities(U, psi, n)
    return abs(float(P.sum()) - float(np.vdot(psi, psi).real))


def pin_powers(n=9, nmat=3):
    """Repeated squaring == numpy.linalg.matrix_power(U, 2^k), and
    == repetition of U 2^k times."""
    rng = np.random.default_rng(17)
    U = W.haar_unitary(rng, 1 << nmat)
    sq = gates.powers_by_squaring(U, n)
    rep = gates.powers_by_repetition(U, n)
    worst = 0.0
    for k in range(n):
        ref = np.linalg.matrix_power(U, 1 << k)
        worst = max(worst, float(np.abs(sq[k] - ref).max()), float(np.abs(rep[k] - ref).max()))
    return worst


def pin_rows_after_sweeps(n=6, nmat=2):
    """After the Hadamard layer and all controlled gates, row m equals
    2^(-n/2) U^m psi (brute force: U applied m times)."""
    rng = np.random.default_rng(19)
    U = W.haar_unitary(rng, 1 << nmat)
    psi = W.random_state(rng, 1 << nmat, 1)[:, 0]
    S = gates.qpe_after_sweeps(U, psi, n)
    worst = 0.0
    v = psi.copy()
    for m in range(1 << n):
        worst = max(worst, float(np.abs(S[m] - v / np.sqrt(1 << n)).max()))
        v = U @ v
    return worst


def pin_eigen_rows(n=8, nmat=3):
    """For psi = v_j (an eigenvector), row m after the sweeps is exactly
    exp(2 pi i m phi_j) v_j / sqrt(N)."""
    rng = np.random.default_rng(23)
    inst = W.haar_instance(rng, nmat, n)
    S = gates.qpe_after_sweeps(inst.U, inst.psi, n)
    m = np.arange(1 << n)[:, None]
    ref = np.exp(2j * np.pi * m * inst.phases[0]) * inst.psi[None, :] / np.sqrt(1 << n)
    return float(np.abs(S - ref).max())


def pin_paper_exact_cases():
    """The analytic family of Sec. 3 (phases j / 2^Nmat, eigenvector x_j as
    input) read against tests/golden/paper_exact_phases.txt."""
    worst = 0.0
    with open(os.path.join(GOLDEN, "paper_exact_phases.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            nmat, nmeas, j, y, p = line.split()
            inst = W.analytic_instance(int(nmat), int(nmeas), int(j))
            P = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
            tgt = np.zeros_like(P)
            tgt[int(y)] = float(p)
            worst = max(worst, float(np.abs(P - tgt).max()))
    return worst


PINS = {
    "qft_vs_numpy_fft": (pin_qft_vs_numpy_fft, 1e-12),
    "full_matrix": (pin_full_matrix, 1e-12),
    "exact_phase_c1": (pin_exact_phase_c1, 1e-12),
    "fejer_vs_gates": (pin_fejer_vs_gates, 1e-12),
    "fejer_closed_vs_sum": (pin_fejer_closed_vs_sum, 1e-12),
    "norm": (pin_norm, 1e-12),
    "powers": (pin_powers, 1e-12),
    "rows_after_sweeps": (pin_rows_after_sweeps, 1e-12),
    "eigen_rows": (pin_eigen_rows, 1e-12),
    "paper_exact_cases": (pin_paper_exact_cases, 1e-10),
}


@pytest.mark.parametrize("name", sorted(PINS))
def test_pin(name):
    fn, tol = PINS[name]
    err = fn()
    assert err <= tol, f"{name}: error {err:.3e} > {tol:.1e}"


# ----------------------------------------------------------- further checks

def test_c2_fejer_full_size():
    """C2 at full size (22 qubits): gate-by-gate histogram vs the Fejer closed
    form, to the FP64 floor of a 64 x 64 constructed unitary."""
    inst = W.c2()
    P = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    assert np.abs(P - Q).max() < 1e-10
    assert readout.argmax_lowest(P) == readout.argmax_lowest(Q)
    # U^(2^15) multiplies the rounding-level non-unitarity of the constructed
    # U by ~2^15, so the norm holds to ~N u rather than u.
    assert abs(P.sum() - 1.0) < 1e-10


def test_fejer_exact_integer_limit():
    """F_n = 1 at delta integer, 0 at the other multiples of 1/N."""
    n = 5
    N = 1 << n
    x = np.arange(-2 * N, 2 * N + 1, dtype=np.float64)
    F = fejer.fejer(n, x)
    want = np.where(np.mod(x, N) == 0, 1.0, 0.0)
    assert np.abs(F - want).max() < 1e-15


def test_readout_estimators():
    P = np.array([0.1, 0.3, 0.3, 0.2, 0.1])
    assert readout.argmax_lowest(P) == 1  # tie -> lowest index
    P = np.zeros(8)
    P[2] = 0.5
    P[6] = 0.5
    assert readout.phase_weighted_mean(P) == pytest.approx((2 + 6) / 2 / 8)
    assert readout.circular_distance(0.95, 0.05) == pytest.approx(0.1)
    Q = np.zeros(16)
    Q[15] = 0.5
    Q[1] = 0.5
    assert readout.circular_distance(readout.phase_circular_mean(Q), 0.0) < 1e-12


def test_c5_closed_form_invariant_under_coefficient_phases():
    """C5's distribution depends on |c_j|^2 only: redraw the phases of c_j and
    the gate-by-gate histogram is unchanged (reduced Nmeas)."""
    inst = W.c5(nmeas=8)
    V = inst.meta["V"]
    c = V.conj().T @ inst.psi
    rng = np.random.default_rng(99)
    psi2 = V @ (np.abs(c) * np.exp(2j * np.pi * rng.random(c.shape[0])))
    P1 = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
    P2 = gates.qpe_probabilities(inst.U, psi2, inst.nmeas)
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    assert np.abs(P1 - P2).max() < 1e-12
    assert np.abs(P1 - Q).max() < 1e-12


# ------------------------------------------------------- planted mistakes

def _bad_qft_sign(S):
    n = S.shape[0].bit_length() - 1
    for g in reversed(gates.qft_gate_list(n)):
        if g[0] == "h":
            gates.hadamard(S, g[1])
        elif g[0] == "cp":
            gates.controlled_phase(S, g[1], g[2], +g[3])  # sign not negated
        else:
            gates.swap(S, g[1], g[2])


def _bad_qft_no_swaps(S):
    n = S.shape[0].bit_length() - 1
    for g in reversed(gates.qft_gate_list(n)):
        if g[0] == "h":
            gates.hadamard(S, g[1])
        elif g[0] == "cp":
            gates.controlled_phase(S, g[1], g[2], -g[3])


def _bad_qft_swaps_last(S):
    n = S.shape[0].bit_length() - 1
    gl = list(reversed(gates.qft_gate_list(n)))
    for g in [g for g in gl if g[0] != "swap"] + [g for g in gl if g[0] == "swap"]:
        if g[0] == "h":
            gates.hadamard(S, g[1])
        elif g[0] == "cp":
            gates.controlled_phase(S, g[1], g[2], -g[3])
        else:
            gates.swap(S, g[1], g[2])


def _bad_controlled_transposed(S, bit, M):
    v = gates._pair_view(S, bit)
    v[:, 1] = v[:, 1] @ M  # M^T instead of M applied


def _bad_controlled_wrong_bit(S, bit, M):
    n = S.shape[0].bit_length() - 1
    v = gates._pair_view(S, n - 1 - bit)
    v[:, 1] = v[:, 1] @ M.T


def _bad_squaring(U, n):
    P = [np.array(U, dtype=np.complex128)]
    for _ in range(1, n):
        P.append(P[-1] @ U)  # U^(k+1) instead of U^(2^k)
    return P


def _bad_hadamard_scale(S, bit):
    gates.apply_single(S, bit, np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128))


def _bad_probabilities_abs(fs):
    return np.sum(np.abs(fs), axis=1)


def _bad_phase_sign(S, bit_a, bit_b, theta):
    N = S.shape[0]
    m = np.arange(N)
    sel = ((m >> bit_a) & 1).astype(bool) | ((m >> bit_b) & 1).astype(bool)  # OR not AND
    S[sel] *= np.exp(1j * theta)


_orig_fejer = fejer.fejer


def _bad_fejer_no_N2(n, x):
    return _orig_fejer(n, x) * float(1 << n) ** 2 / float(1 << n)


def _bad_fejer_sign(n, x):
    return _orig_fejer(n, -np.asarray(x) + 1.0)


MUTANTS = {
    "qft_sign": (gates, "qft_inverse", _bad_qft_sign),
    "qft_no_swaps": (gates, "qft_inverse", _bad_qft_no_swaps),
    "qft_swaps_last": (gates, "qft_inverse", _bad_qft_swaps_last),
    "controlled_transposed": (gates, "controlled_unitary", _bad_controlled_transposed),
    "controlled_wrong_bit": (gates, "controlled_unitary", _bad_controlled_wrong_bit),
    "squaring": (gates, "powers_by_squaring", _bad_squaring),
    "hadamard_scale": (gates, "hadamard", _bad_hadamard_scale),
    "probabilities_abs": (gates, "probabilities", _bad_probabilities_abs),
    "phase_or": (gates, "controlled_phase", _bad_phase_sign),
    "fejer_no_N2": (fejer, "fejer", _bad_fejer_no_N2),
    "fejer_sign": (fejer, "fejer", _bad_fejer_sign),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes(name, monkeypatch):
    """Each planted mistake must make at least one pin fail."""
    mod, attr, bad = MUTANTS[name]
    monkeypatch.setattr(mod, attr, bad)
    failed = []
    for pname, (fn, tol) in PINS.items():
        try:
            err = fn()
        except Exception:  # a crash also counts as caught
            failed.append(pname)
            continue
        if not (err <= tol):
            failed.append(pname)
    assert failed, f"planted mistake {name} was caught by no pin"
