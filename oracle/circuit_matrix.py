"""The whole QPE circuit (Fig. 1) as one explicit square matrix.

For Nmeas + Nmat <= 8 qubits, every gate is written out as a full
2^(Nmeas+Nmat) matrix built from its definition (Kronecker products and block
diagonals), the matrices are multiplied in circuit order, and the product is
applied to |0>_meas (x) psi. Nothing here reuses the gate-by-gate code: the
inverse QFT comes from its defining matrix, not from the H / phase / swap
sequence, and U^(2^k) is U multiplied 2^k times, not squared.

Flat index = m * 2^Nmat + t; measurement qubit k is bit k of m.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

MAX_QUBITS = 8


def _check(n: int, nmat: int) -> None:
    if n + nmat > MAX_QUBITS:
        raise ValueError(f"full circuit matrix limited to {MAX_QUBITS} qubits, got {n + nmat}")


def hadamard_matrix(n: int, nmat: int, k: int) -> np.ndarray:
    """H on measurement qubit k: I_(2^(n-1-k)) (x) H (x) I_(2^k) (x) I_d."""
    H = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0)
    return np.kron(np.kron(np.kron(np.eye(1 << (n - 1 - k)), H), np.eye(1 << k)), np.eye(1 << nmat))


def controlled_matrix(n: int, nmat: int, k: int, M: np.ndarray) -> np.ndarray:
    """Controlled-M, control = measurement qubit k: block diagonal over m with
    block M where bit k of m is 1 and the identity elsewhere."""
    d = 1 << nmat
    N = 1 << n
    out = np.zeros((N * d, N * d), dtype=np.complex128)
    for m in range(N):
        blk = M if (m >> k) & 1 else np.eye(d)
        out[m * d:(m + 1) * d, m * d:(m + 1) * d] = blk
    return out


def inverse_qft_matrix(n: int, nmat: int) -> np.ndarray:
    """QFT^-1 on the measurement register from its definition,
    F^dagger[y, m] = 2^(-n/2) exp(-2 pi i m y / 2^n), tensored with I_d."""
    N = 1 << n
    y = np.arange(N)[:, None]
    m = np.arange(N)[None, :]
    F = np.exp(-2j * np.pi * ((m * y) % N) / N) / np.sqrt(N)
    return np.kron(F, np.eye(1 << nmat))


def power_by_repetition(U: np.ndarray, e: int) -> np.ndarray:
    """U^e as e explicit multiplications."""
    out = np.eye(U.shape[0], dtype=np.complex128)
    for _ in range(e):
        out = out @ U
    return out


def qpe_circuit_matrix(U: np.ndarray, n: int) -> np.ndarray:
    """Product of all gates of Fig. 1 in circuit order:
    QFT^-1 . CU_(n-1) ... CU_0 . H_(n-1) ... H_0."""
    nmat = U.shape[0].bit_length() - 1
    _check(n, nmat)
    dim = (1 << n) << nmat
    C = np.eye(dim, dtype=np.complex128)
    for k in range(n):
        C = hadamard_matrix(n, nmat, k) @ C
    for k in range(n):
        C = controlled_matrix(n, nmat, k, power_by_repetition(U, 1 << k)) @ C
    C = inverse_qft_matrix(n, nmat) @ C
    return C


def qpe_final_state(U: np.ndarray, psi: np.ndarray, n: int) -> np.ndarray:
    """Circuit matrix applied to |0>_meas (x) psi, returned as (2^n, d)."""
    d = U.shape[0]
    v = np.zeros(((1 << n) * d,), dtype=np.complex128)
    v[:d] = psi
    return (qpe_circuit_matrix(U, n) @ v).reshape(1 << n, d)
