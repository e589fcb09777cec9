"""The reassociation behind the fused schedule, on the CPU.

With m = m_b + L m_a (m_b the low r bits, L = 2^r) and y = y_a + N_a y_b
(N_a = N / L),

    X[y] = sum_{m_b} w_L^(m_b y_b) w_N^(m_b y_a) U^(m_b) Z[y_a],
    Z[y_a] = sum_{m_a} w_{N_a}^(m_a y_a) (U^L)^(m_a) psi,

and Z is the same transform for U^L on n - r qubits, so the levels recurse.
Checked here in FP64 numpy against the direct sum X[y] = sum_m w_N^(m y)
U^m psi and against the oracle's gate-by-gate histogram, for level widths
that do and do not divide n.
"""
import numpy as np
import pytest

from oracle import gates
from paper_2507_17175_gb300 import workloads as W


def levels(U, psi, n, r):
    """X[y] for y < 2^n (rows of a 2^n x d array) by the level recursion."""
    d = U.shape[0]
    if n == 0:
        return psi[None, :].copy()
    rb = min(r, n)
    L, N = 1 << rb, 1 << n
    Na = N // L
    Z = levels(np.linalg.matrix_power(U, L), psi, n - rb, r)  # Na x d
    M = [np.linalg.matrix_power(U, mb) for mb in range(L)]     # the level's table U^(m_b)
    X = np.zeros((N, d), dtype=np.complex128)
    for ya in range(Na):
        T = np.array([np.exp(-2j * np.pi * mb * ya / N) * (M[mb] @ Z[ya]) for mb in range(L)])
        for yb in range(L):
            w = np.exp(-2j * np.pi * np.arange(L) * yb / L)
            X[ya + Na * yb] = w @ T
    return X


def direct(U, psi, n):
    N = 1 << n
    rows = [psi]
    for _ in range(N - 1):
        rows.append(U @ rows[-1])
    S = np.array(rows)  # S[m] = U^m psi
    F = np.exp(-2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N)
    return F @ S


@pytest.mark.parametrize("nmat,n,r", [(2, 6, 2), (2, 7, 3), (3, 5, 5), (1, 8, 3), (3, 6, 4)])
def test_level_recursion_equals_direct_transform(nmat, n, r):
    rng = np.random.default_rng(nmat * 100 + n * 10 + r)
    inst = W.haar_instance(rng, nmat, n, superposition=True)
    X = levels(inst.U, inst.psi, n, r)
    Xd = direct(inst.U, inst.psi, n)
    assert np.abs(X - Xd).max() <= 1e-11 * np.abs(Xd).max()
    # and its histogram is the circuit's (QFT^-1 normalisation 2^-n on the amplitudes' sum)
    P = (np.abs(X) ** 2).sum(axis=1) / float(1 << (2 * n))
    ref = gates.qpe_probabilities(inst.U, inst.psi, n)
    assert np.abs(P - ref).max() <= 1e-12


def test_wrong_twiddle_is_caught():
    """Dropping the inter-level twiddle w_N^(m_b y_a) breaks the identity."""
    rng = np.random.default_rng(7)
    inst = W.haar_instance(rng, 2, 6, superposition=True)
    U, psi, n, r = inst.U, inst.psi, 6, 2
    L, N = 1 << r, 1 << n
    Na = N // L
    Z = levels(np.linalg.matrix_power(U, L), psi, n - r, r)
    X = np.zeros((N, U.shape[0]), dtype=np.complex128)
    for ya in range(Na):
        T = np.array([np.linalg.matrix_power(U, mb) @ Z[ya] for mb in range(L)])  # no twiddle
        for yb in range(L):
            X[ya + Na * yb] = np.exp(-2j * np.pi * np.arange(L) * yb / L) @ T
    assert np.abs(X - direct(U, psi, n)).max() > 1e-3
