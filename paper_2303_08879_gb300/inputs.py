"""Seeded synthetic Gaussian-circuit workloads.

This module only draws random circuit parameters and propagates a Gaussian
state through textbook linear optics (single-mode squeezing, displacement, a
Haar-random interferometer and per-mode pure loss) in the real quadrature
picture.  It holds none of the Fock-recurrence method: the map from the
quadrature covariance to the Bargmann triple (A, b, c) and everything after it
live in the library (product path) and, independently, in ``oracle/``.

Conventions
-----------
* Quadrature ordering (x_1..x_M, p_1..p_M), hbar = 1, vacuum covariance I/2.
* Squeezing r on mode j: x_j -> e^{-r} x_j, p_j -> e^{r} p_j.
* Displacement alpha: <x> = sqrt(2) Re(alpha), <p> = sqrt(2) Im(alpha).
* Interferometer U acts as the symplectic [[Re U, -Im U], [Im U, Re U]].
* Loss eta: V -> eta V + (1 - eta)/2 I per mode, mean -> sqrt(eta) mean.
* Circuit order: squeeze -> displace -> interferometer -> loss (Fig. 1 of the
  paper shows squeezed vacua sent through an interferometer before detection).

Every random draw comes from ``numpy.random.Generator(PCG64(...))`` seeded by
(workload id, circuit index), so both sides of a parity test see identical
inputs.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "GaussianCircuit", "haar_unitary", "make_circuit", "workload",
    "WORKLOADS", "rng_for",
]


@dataclasses.dataclass
class GaussianCircuit:
    """One synthetic noisy Gaussian circuit and the state it prepares."""
    M: int
    r: np.ndarray          # squeezing per mode
    alpha: np.ndarray      # complex displacement per mode
    U: np.ndarray          # M x M unitary
    eta: np.ndarray        # transmissivity per mode
    V: np.ndarray          # 2M x 2M real quadrature covariance (x.., p..)
    mean: np.ndarray       # 2M real quadrature mean
    cutoffs: tuple         # photon-number cutoff per mode (k < C)
    detected: tuple        # True for PNR-detected modes


def rng_for(workload_id: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(workload_id), int(index)]))


def haar_unitary(M: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random unitary: QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri, Notices AMS 54 (2007) 592)."""
    Z = (rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def propagate(M, r, alpha, U, eta):
    """Quadrature covariance and mean after squeeze, displace, U, loss."""
    V = np.diag(np.concatenate([np.exp(-2.0 * r), np.exp(2.0 * r)])) / 2.0
    mean = np.sqrt(2.0) * np.concatenate([alpha.real, alpha.imag])
    S = np.block([[U.real, -U.imag], [U.imag, U.real]])
    V = S @ V @ S.T
    mean = S @ mean
    x = np.sqrt(np.concatenate([eta, eta]))
    V = x[:, None] * V * x[None, :] + np.diag(np.concatenate([1 - eta, 1 - eta])) / 2.0
    mean = x * mean
    V = 0.5 * (V + V.T)
    return V, mean


def make_circuit(M, rng, *, r_range, eta_range, alpha_var=0.0,
                 cutoffs, detected=None, identity_interferometer=False):
    r = rng.uniform(r_range[0], r_range[1], size=M)
    U = np.eye(M, dtype=complex) if identity_interferometer else haar_unitary(M, rng)
    eta = rng.uniform(eta_range[0], eta_range[1], size=M)
    if alpha_var > 0:
        s = np.sqrt(alpha_var / 2.0)
        alpha = rng.normal(scale=s, size=M) + 1j * rng.normal(scale=s, size=M)
    else:
        alpha = np.zeros(M, dtype=complex)
    V, mean = propagate(M, r, alpha, U, eta)
    det = tuple([True] * M) if detected is None else tuple(bool(v) for v in detected)
    return GaussianCircuit(M, r, alpha, U, eta, V, mean, tuple(int(c) for c in cutoffs), det)


# ---------------------------------------------------------------------------
# The synthetic workloads (shapes and distributions of the paper's
# GBS / conditional-state settings); tests take the first few circuits of one.
# ---------------------------------------------------------------------------

def _gbs_m2_c10(i, rng):
    return make_circuit(2, rng, r_range=(0.0, 1.0), eta_range=(0.5, 1.0), cutoffs=(10, 10))


def _cond_m3(i, rng):
    c0 = int(rng.integers(10, 21)); c1 = int(rng.integers(10, 21)); cu = int(rng.integers(20, 31))
    return make_circuit(3, rng, r_range=(0.0, 1.2), eta_range=(0.7, 1.0), alpha_var=0.5,
                        cutoffs=(c0, c1, cu), detected=(True, True, False))


def _gbs_m8_c6(i, rng):
    return make_circuit(8, rng, r_range=(0.3, 1.0), eta_range=(0.6, 1.0), cutoffs=(6,) * 8)


def _gbs_m12_c5(i, rng):
    return make_circuit(12, rng, r_range=(0.2, 0.8), eta_range=(0.8, 1.0), cutoffs=(5,) * 12)


WORKLOADS = {
    # name: (seed stream of the workload, number of circuits, maker)
    "gbs_m2_c10": (1, 1, _gbs_m2_c10),
    "cond_m3_batch64": (2, 64, _cond_m3),
    "gbs_m8_c6_batch16": (3, 16, _gbs_m8_c6),
    "gbs_m12_c5": (5, 1, _gbs_m12_c5),
}


def workload(name: str, n: int | None = None, start: int = 0):
    """Return the list of circuits of a named workload (first ``n`` only)."""
    wid, count, maker = WORKLOADS[name]
    n = count if n is None else n
    return [maker(i, rng_for(wid, i)) for i in range(start, start + n)]


def random_symmetric(D, rng, scale=0.2, with_b=True, b_scale=0.3):
    """A generic complex symmetric A and vector b (no physical meaning): used
    only to exercise the recurrence on arbitrary inputs."""
    X = (rng.normal(size=(D, D)) + 1j * rng.normal(size=(D, D))) * scale
    A = X + X.T
    b = (rng.normal(size=D) + 1j * rng.normal(size=D)) * b_scale if with_b else np.zeros(D, complex)
    return A, b
