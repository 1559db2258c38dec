"""Brute-force loop hafnian.  TEST INFRASTRUCTURE ONLY.

An independent definition of the Fock amplitudes used to pin the recurrence:
the amplitudes of Sec. 2.1 are the scaled Taylor coefficients of the
generating function c exp(z^T A z / 2 + b^T z),

    G_k = sqrt(k!) [z^k] c exp(z^T A z / 2 + b^T z) = c lhaf(A_(k)) / sqrt(k!),

where A_(k) repeats row/column i of A k_i times and carries b_i on its
diagonal (the loops).  The loop hafnian is the sum over all partitions of
the rows into pairs {p, q} (weight A_pq) and singletons {p} (weight b_p),
the object behind the GBS probability formulas the paper compares against
in Sec. 4.2.  Cost grows like the telephone numbers: tiny inputs only.
"""
from __future__ import annotations

from functools import lru_cache
from math import factorial, sqrt

import numpy as np


def loop_hafnian(X):
    """lhaf of a symmetric n x n matrix whose diagonal holds the loop weights."""
    X = np.asarray(X, dtype=np.complex128)
    n = X.shape[0]

    @lru_cache(maxsize=None)
    def rec(mask):
        if mask == 0:
            return 1.0 + 0.0j
        p = (mask & -mask).bit_length() - 1       # lowest remaining row
        rest = mask & ~(1 << p)
        total = X[p, p] * rec(rest)                # p is a singleton (loop)
        m = rest
        while m:
            q = (m & -m).bit_length() - 1
            m &= m - 1
            total += X[p, q] * rec(rest & ~(1 << q))   # p paired with q
        return total

    return rec((1 << n) - 1)


def amplitude(A, b, c, k):
    """G_k = c lhaf(A_(k)) / sqrt(prod k_i!) for a lattice index k."""
    A = np.asarray(A, dtype=np.complex128)
    As = 0.5 * (A + A.T)
    b = np.asarray(b, dtype=np.complex128)
    idx = [i for i, ki in enumerate(k) for _ in range(int(ki))]
    X = As[np.ix_(idx, idx)].copy() if idx else np.zeros((0, 0), np.complex128)
    for p, i in enumerate(idx):
        X[p, p] = b[i]
    norm = 1.0
    for ki in k:
        norm *= factorial(int(ki))
    return c * loop_hafnian(X) / sqrt(norm)
