"""Phase readout from the measurement distribution (Sec. 3 and Sec. 4.2).

Two estimators are defined in the paper's precision study:

* maximum norm: the single outcome y with the largest probability, phase
  y / 2^n (ties resolved to the lowest y);
* weighted average: sum_y P(y) y / 2^n, weights the squared norms.

Errors are compared as plain absolute differences (as in Sec. 4.2) and, for
phases near the 0/1 wrap, as circular distances.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def argmax_lowest(P: np.ndarray) -> int:
    """Index of the maximum of P; the lowest index among exact ties
    (numpy.argmax returns the first occurrence)."""
    return int(np.argmax(P))


def phase_max_norm(P: np.ndarray) -> float:
    N = P.shape[0]
    return argmax_lowest(P) / N


def phase_weighted_mean(P: np.ndarray) -> float:
    N = P.shape[0]
    y = np.arange(N, dtype=np.float64)
    return float(np.sum(P * y) / N)


def phase_circular_mean(P: np.ndarray) -> float:
    """arg(sum_y P(y) exp(2 pi i y / N)) / (2 pi), mapped into [0, 1)."""
    N = P.shape[0]
    z = np.sum(P * np.exp(2j * np.pi * np.arange(N) / N))
    return float(np.mod(np.angle(z) / (2.0 * np.pi), 1.0))


def circular_distance(a: float, b: float) -> float:
    d = abs(a - b) % 1.0
    return min(d, 1.0 - d)
