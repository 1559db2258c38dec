"""Closed-form amplitude derivatives and the vector-Jacobian product.
TEST INFRASTRUCTURE ONLY.

Sec. 2.5 computes the downstream gradient with respect to the conjugate of a
parameter xi in {b_m, A_mn} by the chain rule, eqs. (dL_dB), (dL_dA):

    dL/dxi* = sum_k dL/dG_k* (dG_k/dxi)*,

because G_k is holomorphic in A and b.  With PyTorch's convention for a real
loss (grad z = dL/dRe z + i dL/dIm z = 2 dL/dz*) the same sum reads
grad xi = sum_k gbar_k conj(dG_k/dxi).

The local derivatives follow from the generating function
c exp(z^T A z/2 + b^T z) of the amplitudes (the same object the recurrence of
eq. (recrel) computes coefficient by coefficient):

    dG_k/db_m  = sqrt(k_m) G_{k - 1_m}
    dG_k/dA_mn = 1/2 sqrt(k_m (k_n - delta_mn)) G_{k - 1_m - 1_n}
    dG_k/dc    = G_k / c

where A enters only through its symmetric part (A + A^T)/2, so each entry
A_mn is an independent input and the gradient with respect to A is symmetric.
These act on a full lattice array (the output of ``full_lattice``).
"""
from __future__ import annotations

import numpy as np


def _shift(G, idx_list):
    """Array H with H[k] = G[k - sum of 1_i for i in idx_list] (0 if negative)."""
    H = G
    for i in idx_list:
        pad = [(0, 0)] * G.ndim
        pad[i] = (1, 0)
        sl = [slice(None)] * G.ndim
        sl[i] = slice(0, G.shape[i])
        H = np.pad(H, pad)[tuple(sl)]
    return H


def _kgrid(shape, i):
    sh = [1] * len(shape)
    sh[i] = shape[i]
    return np.arange(shape[i], dtype=float).reshape(sh)


def dG_db(G, m):
    return np.sqrt(_kgrid(G.shape, m)) * _shift(G, [m])


def dG_dA(G, m, n):
    km = _kgrid(G.shape, m)
    kn = _kgrid(G.shape, n) - (1.0 if m == n else 0.0)
    fac = 0.5 * np.sqrt(np.clip(km * kn, 0.0, None))
    return fac * _shift(G, [m, n])


def vjp(G, gbar, c):
    """(grad_A, grad_b, grad_c) for upstream gbar (same shape as G)."""
    D = G.ndim
    gA = np.zeros((D, D), np.complex128)
    gb = np.zeros(D, np.complex128)
    for m in range(D):
        gb[m] = np.sum(gbar * np.conj(dG_db(G, m)))
        for n in range(D):
            gA[m, n] = np.sum(gbar * np.conj(dG_dA(G, m, n)))
    gc = np.sum(gbar * np.conj(G / c))
    return gA, gb, gc


def jvp(G, c, dA, db, dc):
    """Directional derivative of every amplitude along (dA, db, dc)."""
    D = G.ndim
    out = G * (dc / c)
    for m in range(D):
        out = out + db[m] * dG_db(G, m)
        for n in range(D):
            out = out + dA[m, n] * dG_dA(G, m, n)
    return out
