"""Closed forms of the QPE measurement distribution.

For psi = sum_j c_j v_j with v_j orthonormal eigenvectors of U, U v_j =
exp(2 pi i phi_j) v_j (Sec. 2), the state after the controlled gates has rows
2^(-n/2) U^m psi, and after QFT^-1 the amplitude at outcome y is
sum_j c_j a_n(phi_j - y/N) v_j with

    a_n(delta) = N^-1 sum_{m<N} exp(2 pi i m delta),   N = 2^n.

Orthonormality of the v_j removes the cross terms, so

    P(y) = sum_j |c_j|^2 F_n(phi_j - y/N),
    F_n(delta) = |a_n(delta)|^2 = sin^2(pi N delta) / (N^2 sin^2(pi delta)),

with F_n = 1 at integer delta (the Fejer kernel). For an exactly
representable phase phi = k/N this is probability 1 at y = k, the paper's
exact-estimation case (Sec. 3).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def fejer(n: int, x: np.ndarray) -> np.ndarray:
    """F_n evaluated at delta = x / N, taking x = N * delta directly so that
    the caller can form N phi - y without rounding (N phi is exact in binary
    floating point and so is its difference with an integer of similar size).

    F_n(x / N) = sin^2(pi x) / (N^2 sin^2(pi x / N)); at integer x that is a
    multiple of N the quotient is replaced by its limit 1.
    """
    N = float(1 << n)
    x = np.asarray(x, dtype=np.float64)
    # reduce x modulo N into (-N/2, N/2]: F_n has period N in x
    xr = x - N * np.round(x / N)
    num = np.sin(np.pi * xr) ** 2
    den = (N * np.sin(np.pi * xr / N)) ** 2
    out = np.empty_like(xr)
    small = np.abs(xr) < 1e-300
    out[small] = 1.0
    with np.errstate(invalid="ignore", divide="ignore"):
        out[~small] = num[~small] / den[~small]
    return out


def fejer_bruteforce(n: int, delta: float) -> float:
    """|N^-1 sum_{m<N} exp(2 pi i m delta)|^2 summed term by term (small n)."""
    N = 1 << n
    m = np.arange(N)
    return float(np.abs(np.exp(2j * np.pi * m * delta).sum() / N) ** 2)


def probabilities(phases: np.ndarray, weights: np.ndarray, n: int,
                  y: np.ndarray | None = None) -> np.ndarray:
    """P(y) = sum_j w_j F_n(phi_j - y/N) for the outcomes ``y`` (all 2^n by
    default); w_j = |c_j|^2."""
    N = 1 << n
    if y is None:
        y = np.arange(N, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    out = np.zeros(y.shape, dtype=np.float64)
    for phi, w in zip(np.asarray(phases, dtype=np.float64), np.asarray(weights, dtype=np.float64)):
        if w == 0.0:
            continue
        out += w * fejer(n, N * phi - y.astype(np.float64))
    return out
