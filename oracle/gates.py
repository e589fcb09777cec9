"""Gate-by-gate FP64 statevector simulation of QPE (Sec. 2, Fig. 1).

The state of Nmeas + Nmat qubits is held as an (N, d) complex128 array S with
N = 2^Nmeas rows (measurement register, row index m) and d = 2^Nmat columns
(target register). Every gate of Fig. 1 is applied on its own, in circuit
order, with no fusion: the Hadamard layer, one controlled-U^(2^k) per
measurement qubit, then the inverse quantum Fourier transform written out as
its textbook gate sequence (Hadamards, controlled phase rotations, swaps).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

_H = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0)


def _pair_view(S: np.ndarray, bit: int) -> np.ndarray:
    """View S (N, d) as (N / 2^(bit+1), 2, 2^bit, d): axis 1 is measurement
    bit ``bit``."""
    N, d = S.shape
    return S.reshape(N >> (bit + 1), 2, 1 << bit, d)


def apply_single(S: np.ndarray, bit: int, G: np.ndarray) -> None:
    """Apply the 2x2 gate G to measurement qubit ``bit`` in place."""
    v = _pair_view(S, bit)
    a = v[:, 0].copy()
    b = v[:, 1].copy()
    v[:, 0] = G[0, 0] * a + G[0, 1] * b
    v[:, 1] = G[1, 0] * a + G[1, 1] * b


def hadamard(S: np.ndarray, bit: int) -> None:
    """H on measurement qubit ``bit`` (Fig. 1, first column)."""
    apply_single(S, bit, _H)


def controlled_unitary(S: np.ndarray, bit: int, M: np.ndarray) -> None:
    """Controlled-M with measurement qubit ``bit`` as control and the target
    register as target (Fig. 1, the U^(2^k) boxes): every row whose bit is 1
    becomes M times that row (the row read as a column vector)."""
    v = _pair_view(S, bit)
    v[:, 1] = v[:, 1] @ M.T


def controlled_phase(S: np.ndarray, bit_a: int, bit_b: int, theta: float) -> None:
    """Multiply the amplitudes whose measurement bits a and b are both 1 by
    exp(i theta) (the controlled rotation of the QFT circuit; symmetric in its
    two qubits)."""
    N = S.shape[0]
    m = np.arange(N)
    sel = ((m >> bit_a) & 1).astype(bool) & ((m >> bit_b) & 1).astype(bool)
    S[sel] *= np.exp(1j * theta)


def swap(S: np.ndarray, bit_a: int, bit_b: int) -> None:
    """SWAP of measurement qubits a and b: row m moves to the row with those
    two bits exchanged."""
    N = S.shape[0]
    m = np.arange(N)
    ba = (m >> bit_a) & 1
    bb = (m >> bit_b) & 1
    partner = m ^ ((ba ^ bb) << bit_a) ^ ((ba ^ bb) << bit_b)
    S[:] = S[partner]


def qft_gate_list(n: int) -> list[tuple]:
    """The textbook QFT circuit on n qubits as a gate list.

    Qubits are named q_1 .. q_n with q_1 the most significant bit of m (bit
    n-1). For j = 1..n: H on q_j, then for k = 2..n-j+1 the rotation
    R_k = diag(1, exp(2 pi i / 2^k)) on q_j controlled by q_{j+k-1}; finally
    q_i and q_{n+1-i} are swapped. Entries are ("h", bit), ("cp", bit_a,
    bit_b, theta) or ("swap", bit_a, bit_b).
    """
    gates: list[tuple] = []
    bit = lambda j: n - j  # noqa: E731  (q_j -> bit index)
    for j in range(1, n + 1):
        gates.append(("h", bit(j)))
        for k in range(2, n - j + 2):
            gates.append(("cp", bit(j + k - 1), bit(j), 2.0 * np.pi / (1 << k)))
    for i in range(1, n // 2 + 1):
        gates.append(("swap", bit(i), bit(n + 1 - i)))
    return gates


def qft_inverse(S: np.ndarray) -> None:
    """Apply QFT^-1 on the measurement register gate by gate (Fig. 1, the
    QFT^-1 box): the adjoint of ``qft_gate_list``, i.e. the same gates in
    reverse order with every rotation angle negated (H and SWAP are their own
    inverses)."""
    n = S.shape[0].bit_length() - 1
    for g in reversed(qft_gate_list(n)):
        if g[0] == "h":
            hadamard(S, g[1])
        elif g[0] == "cp":
            controlled_phase(S, g[1], g[2], -g[3])
        else:
            swap(S, g[1], g[2])


def powers_by_squaring(U: np.ndarray, n: int) -> list[np.ndarray]:
    """P_k = U^(2^k) for k = 0..n-1 by repeated squaring, P_{k+1} = P_k P_k
    (the controlled gates of Fig. 1 need U^(2^k); squaring is how this
    emulator builds them)."""
    P = [np.array(U, dtype=np.complex128)]
    for _ in range(1, n):
        P.append(P[-1] @ P[-1])
    return P


def powers_by_repetition(U: np.ndarray, n: int) -> list[np.ndarray]:
    """P_k = U^(2^k) built by multiplying U into the identity 2^k times, the
    construction the paper's cost argument implies (Sec. 4.1: the number of
    controlled-U operations doubles with each measurement qubit). Exponential
    cost; for small n only."""
    d = U.shape[0]
    P = []
    acc = np.eye(d, dtype=np.complex128)
    applied = 0
    for k in range(n):
        while applied < (1 << k):
            acc = U @ acc
            applied += 1
        P.append(acc.copy())
    return P


def initial_state(psi: np.ndarray, n: int) -> np.ndarray:
    """|0...0>_meas (x) psi as an (2^n, d) array (Fig. 1, left edge)."""
    d = psi.shape[0]
    S = np.zeros((1 << n, d), dtype=np.complex128)
    S[0] = psi
    return S


def hadamard_layer(S: np.ndarray) -> None:
    """H on every measurement qubit (Fig. 1)."""
    n = S.shape[0].bit_length() - 1
    for b in range(n):
        hadamard(S, b)


def controlled_sweeps(S: np.ndarray, powers: list[np.ndarray]) -> None:
    """Controlled-U^(2^k) for k = 0..n-1, control = measurement qubit k (Fig. 1,
    top wire controls U^(2^0))."""
    for k, P in enumerate(powers):
        controlled_unitary(S, k, P)


def qpe_after_sweeps(U: np.ndarray, psi: np.ndarray, n: int, powers=None) -> np.ndarray:
    """State after the Hadamard layer and all controlled-U^(2^k) gates."""
    if powers is None:
        powers = powers_by_squaring(U, n)
    S = initial_state(np.asarray(psi, dtype=np.complex128), n)
    hadamard_layer(S)
    controlled_sweeps(S, powers)
    return S


def qpe_final_state(U: np.ndarray, psi: np.ndarray, n: int, powers=None) -> np.ndarray:
    """Final state of the QPE circuit of Fig. 1 before measurement, (2^n, d),
    row y = measurement outcome y (the statevector the paper's emulator writes
    out, Sec. 3)."""
    S = qpe_after_sweeps(U, psi, n, powers)
    qft_inverse(S)
    return S


def probabilities(final_state: np.ndarray) -> np.ndarray:
    """Measurement distribution of the measurement register: P(y) = sum over
    the target register of |amplitude(y, t)|^2 (Sec. 3, the norms of the
    final statevector)."""
    return np.sum(final_state.real ** 2 + final_state.imag ** 2, axis=1)


def qpe_probabilities(U: np.ndarray, psi: np.ndarray, n: int, powers=None) -> np.ndarray:
    return probabilities(qpe_final_state(U, psi, n, powers))
