"""Seeded synthetic QPE inputs: the unitary U, the input state psi, and the
eigen-data they were built from.

This module only draws inputs. It holds none of the QPE method's arithmetic
(no powers of U, no controlled gates, no Fourier transform, no readout), so
both the CUDA path and the CPU oracle can consume what it produces without
sharing any of the method's code.

The paper validates on two problem families (Sec. 3): an analytically
tractable U with phases j/2^Nmat, and a seeded random unitary (seed 12345)
with reference eigenphases from SciPy. The random family is reproduced here
as U = V diag(exp(2 pi i phi)) V^dagger with V Haar-random (phase-fixed QR of
a complex Gaussian matrix, Mezzadri 2007), so the eigenphases are known by
construction instead of by an eigensolver.

Five named workloads:

  c1  Nmat=2,  Nmeas=6,  phases k_j/64 (exactly representable), psi = V[:,0]
  c2  Nmat=6,  Nmeas=16, phases ~ U[0,1), psi = V[:,0]
  c3  Nmat=12, Nmeas=20, phases ~ U[0,1), psi = V[:,0]
  c4  512 instances, Nmat in {3..10}, Nmeas in {8..18}, psi = V[:,0]
  c5  Nmat=4,  Nmeas=30, psi = sum_j c_j V[:,j], |c_j|^2 ~ Dirichlet(1),
      arg c_j ~ U[0, 2 pi)

All draws use numpy's PCG64 generator seeded with 12345 (the paper's seed);
c4 spawns one child SeedSequence per instance.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED = 12345


@dataclass
class Instance:
    """One QPE problem: U (d x d, complex128, row-major), psi (d,), and the
    eigen-data used to build them (phases phi_j and weights |c_j|^2 of psi in
    the eigenbasis)."""

    name: str
    nmat: int
    nmeas: int
    U: np.ndarray
    psi: np.ndarray
    phases: np.ndarray
    weights: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return 1 << self.nmat

    @property
    def N(self) -> int:
        return 1 << self.nmeas


def haar_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-random d x d unitary: QR of a complex Gaussian, with the phases of
    R's diagonal moved into Q (Mezzadri 2007) so the distribution is exactly
    Haar."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    diag = np.diagonal(r)
    return q * (diag / np.abs(diag))[None, :]


def unitary_from_eigen(V: np.ndarray, phases: np.ndarray) -> np.ndarray:
    """U = V diag(exp(2 pi i phi)) V^dagger, eigenphases phi in [0, 1)."""
    lam = np.exp(2j * np.pi * np.asarray(phases, dtype=np.float64))
    return (V * lam[None, :]) @ V.conj().T


def haar_instance(rng: np.random.Generator, nmat: int, nmeas: int, name: str = "haar",
                  phases: np.ndarray | None = None, superposition: bool = False) -> Instance:
    """A Haar-eigenbasis instance. psi is V[:,0] unless ``superposition``, in
    which case psi = V c with |c|^2 ~ Dirichlet(1,...,1) and uniform phases."""
    d = 1 << nmat
    V = haar_unitary(rng, d)
    if phases is None:
        phases = rng.random(d)
    phases = np.asarray(phases, dtype=np.float64)
    U = unitary_from_eigen(V, phases)
    if superposition:
        w = rng.dirichlet(np.ones(d))
        theta = rng.random(d) * 2.0 * np.pi
        c = np.sqrt(w) * np.exp(1j * theta)
        psi = V @ c
        weights = w
    else:
        psi = V[:, 0].copy()
        weights = np.zeros(d)
        weights[0] = 1.0
    return Instance(name, nmat, nmeas, np.ascontiguousarray(U), np.ascontiguousarray(psi),
                    phases, weights, {"V": V})


def c1() -> Instance:
    """Nmat=2, Nmeas=6: phases k_j/64 with distinct seeded k_j, psi = V[:,0].
    The exact answer is probability 1 at index k_0."""
    rng = np.random.default_rng(SEED)
    V = haar_unitary(rng, 4)
    k = rng.choice(64, 4, replace=False)
    phases = k / 64.0
    inst = Instance("c1", 2, 6, np.ascontiguousarray(unitary_from_eigen(V, phases)),
                    np.ascontiguousarray(V[:, 0].copy()), phases,
                    np.array([1.0, 0.0, 0.0, 0.0]), {"V": V, "k": k})
    return inst


def c2() -> Instance:
    """Nmat=6, Nmeas=16: 64 x 64 Haar eigenbasis, phases ~ U[0,1)."""
    return haar_instance(np.random.default_rng(SEED), 6, 16, "c2")


def c3() -> Instance:
    """Nmat=12, Nmeas=20: 4096 x 4096 Haar eigenbasis, phases ~ U[0,1)."""
    return haar_instance(np.random.default_rng(SEED), 12, 20, "c3")


def c4_shapes(count: int = 512) -> list[tuple[int, int]]:
    """(Nmat, Nmeas) of the batched workload's instances, without building U."""
    out = []
    for s in np.random.SeedSequence(SEED).spawn(count):
        rng = np.random.default_rng(s)
        nmat = int(rng.integers(3, 11))
        nmeas = int(rng.integers(8, 19))
        out.append((nmat, nmeas))
    return out


def c4(count: int = 512) -> list[Instance]:
    """512 independent instances, Nmat uniform in {3..10}, Nmeas in {8..18}."""
    out = []
    for i, s in enumerate(np.random.SeedSequence(SEED).spawn(count)):
        rng = np.random.default_rng(s)
        nmat = int(rng.integers(3, 11))
        nmeas = int(rng.integers(8, 19))
        out.append(haar_instance(rng, nmat, nmeas, f"c4[{i}]"))
    return out


def c5(nmeas: int = 30) -> Instance:
    """Nmat=4, Nmeas=30 (34 qubits): psi a Dirichlet-weighted superposition of
    all 16 eigenvectors. ``nmeas`` may be lowered for reduced-size checks; the
    draw does not depend on it."""
    return haar_instance(np.random.default_rng(SEED), 4, nmeas, "c5", superposition=True)


def by_name(name: str) -> Instance:
    return {"c1": c1, "c2": c2, "c3": c3, "c5": c5}[name]()


def analytic_instance(nmat: int, nmeas: int, j: int) -> Instance:
    """The paper's analytically tractable family (Sec. 3): phi_j = j / 2^Nmat,
    eigenvector x_j with ones in components k <= j, normalised (0-based j, so
    the norm is sqrt(j+1)), P = (x_0 ... x_{d-1}), U = P Lambda P^{-1}.

    P's columns are not orthogonal, so U is not unitary; it is still a valid
    input when psi is one of its eigenvectors x_j, which is what this returns.
    """
    d = 1 << nmat
    phases = np.arange(d) / float(d)
    P = np.zeros((d, d), dtype=np.complex128)
    for col in range(d):
        P[: col + 1, col] = 1.0 / np.sqrt(col + 1.0)
    lam = np.exp(2j * np.pi * phases)
    U = (P * lam[None, :]) @ np.linalg.inv(P)
    psi = P[:, j].copy()
    w = np.zeros(d)
    w[j] = 1.0
    return Instance(f"analytic[{nmat},{nmeas},{j}]", nmat, nmeas, np.ascontiguousarray(U),
                    psi, phases, w, {"P": P})


def random_state(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """A complex Gaussian rows x cols array (for unit tests of single steps)."""
    return (rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))) / np.sqrt(2.0)
