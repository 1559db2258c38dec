"""Gaussian state -> Bargmann triple (A, b, c).  TEST INFRASTRUCTURE ONLY.

Follows Sec. 2.1, eqs. (A_rho) and (b_rho), and the vacuum amplitude of
Sec. 2.2:

    A = P_M sigma_- sigma_+^{-1},   b = P_M sigma_+^{-1} mu,
    c = exp(-mu^dagger sigma_+^{-1} mu / 2) / sqrt(det sigma_+),
    sigma_pm = sigma +- I/2,  P_M = [[0, I], [I, 0]],

with sigma, mu the complex covariance and mean in the (a_1..a_M, a^dag_1..
a^dag_M) basis.  Readings (the paper leaves these implicit):
  * hbar = 1, so vacuum has real quadrature covariance I/2 and complex
    covariance I/2 (sigma_+ = I for vacuum, c = 1);
  * the bar on mu in the vacuum formula is the same complex mean mu;
  * the block order is then interleaved per mode, and each mode's pair is
    ordered so that lattice index 2j is the row m and 2j+1 the column n of
    <m|rho|n> (a coherent state gives G_{01} = e^{-|alpha|^2} conj(alpha)).
"""
from __future__ import annotations

import numpy as np


def quadrature_to_complex(V, mean):
    """(x.., p..) real covariance/mean -> complex sigma, mu in the (a.., a^dag..)
    basis, with a = (x + i p)/sqrt(2)."""
    M = V.shape[0] // 2
    I = np.eye(M)
    W = np.block([[I, 1j * I], [I, -1j * I]]) / np.sqrt(2.0)
    return W @ V @ W.conj().T, W @ mean


def gaussian_to_triple(V, mean):
    """Return (A, b, c) in the interleaved lattice order of the library."""
    V = np.asarray(V, dtype=float)
    mean = np.asarray(mean, dtype=float)
    M = V.shape[0] // 2
    sigma, mu = quadrature_to_complex(V, mean)
    I2 = np.eye(2 * M)
    sp = sigma + I2 / 2.0
    sm = sigma - I2 / 2.0
    Z = np.zeros((M, M))
    P = np.block([[Z, np.eye(M)], [np.eye(M), Z]])
    spi = np.linalg.inv(sp)
    A = P @ sm @ spi
    b = P @ spi @ mu
    c = np.exp(-0.5 * (mu.conj() @ spi @ mu)) / np.sqrt(np.linalg.det(sp))
    # lattice index 2j <- a^dag_j (block index M + j), 2j+1 <- a_j (block index j)
    perm = [v for j in range(M) for v in (M + j, j)]
    return A[np.ix_(perm, perm)], b[perm], complex(c)


def pure_triple(V, mean):
    """(A_psi, b_psi, psi_0) of a pure Gaussian state.  Its density triple has
    no coupling between ket and bra indices (A_rho = A_psi (+) conj(A_psi),
    Sec. 2.1); with the pair order above the ket index m of <m|rho|n> is the
    even lattice index, so A_psi and b_psi are the even-even block and even
    entries, and psi_0 = sqrt(rho_0) (Sec. 2.2, global phase dropped)."""
    A, b, c = gaussian_to_triple(V, mean)
    if np.max(np.abs(A[0::2, 1::2])) > 1e-9 * max(1.0, np.max(np.abs(A))):
        raise ValueError("state is not pure")
    return A[0::2, 0::2].copy(), b[0::2].copy(), complex(np.sqrt(c.real))
