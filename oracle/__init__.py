"""Plain FP64 CPU oracle for the QPE circuit (test infrastructure).

This package is the checker, not the product. Only the test suite, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it. The CUDA library never calls it, and it imports nothing from the
CUDA path; both consume the same seeded inputs from
``paper_2507_17175_gb300.workloads``.

Modules (each function cites the passage of the paper it follows):

* ``gates``          gate-by-gate statevector simulation of the circuit in
                     Fig. 1 (Hadamard layer, controlled-U^(2^k), inverse QFT
                     built from H / controlled-phase / swap gates, measurement).
* ``circuit_matrix`` the whole circuit as one explicit 2^(Nmeas+Nmat) square
                     matrix, for up to 8 qubits.
* ``fejer``          closed forms of the measurement distribution for inputs
                     whose eigen-decomposition is known.
* ``readout``        the two phase estimators of Sec. 4.2 (maximum norm and
                     weighted average) and the circular distance used to
                     compare phases.

Conventions (the readings the paper leaves open, fixed the same way on both
sides of the parity tests):

* measurement qubit k (k = 0 is the top wire of Fig. 1) is bit k of the
  measurement index m and controls U^(2^k);
* the flat state index is m * 2^Nmat + t (measurement register = high bits);
* QFT^-1 is the matrix F^dagger[y, m] = 2^(-n/2) exp(-2 pi i m y / 2^n),
  including the final swaps, so an eigenphase phi peaks at y = 2^n phi.

Every function here is pinned by the ``-m "not gpu"`` tests against something
other than itself (library routines, closed forms, brute force, the paper's
exact-phase claim); none is "parity unpinned".
"""
from . import gates, circuit_matrix, fejer, readout  # noqa: F401
