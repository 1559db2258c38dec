"""Algorithmic work of the walks, for the roofline figures of the benchmark.

Flops are 8 per complex term of eq. (recrel) (four real multiply-adds per
complex product); the real 1/sqrt(P_w + 1) scalings are not counted.  The
terms of a written amplitude are those of its pivot P (Algorithm 1, Sec.
3.1.3): one per lattice index l with P_l >= 1 (the term sqrt(P_l) A_wl
G_{P - 1_l}), plus the b_w G_P term when b != 0.  Every amplitude a pivot
writes has the pivot's terms, so a walk's count is
sum over pivots of (amplitudes written) x (terms).

Pivots of the all-detected walk (modes with C_j >= 2; see fk_shape.h):
  AP(K) e + 1_{2K}: modes < K zero, e_K <= C_K - 2.  Terms
      1 + [e_K >= 1] + 2 #{m > K : e_m >= 1}  (+1 with b).
      Writes: DIAG[e + 1_K]; T2(K)[e] if e_K <= C_K - 3; P1010/P1001(K, m)[e]
      for each m > K with e_m <= C_m - 2.
  DP d (b != 0 only): d_0 <= C_0 - 2.  Terms 2 #{q : d_q >= 1} + 1.
      Writes: T1K(0)[d]; T1B(0)[d] if d_0 <= C_0 - 3; T1K(q), T1B(q)[d] for
      q >= 1 with d_q <= C_q - 2.
The sums factorise over the modes (the constraints are per mode), so they
are evaluated in closed form instead of enumerating the ~1e8 pivots of the
12-mode workload.
"""
from __future__ import annotations

import numpy as np


def _prod(xs):
    p = 1
    for x in xs:
        p *= int(x)
    return p


def _sum_product(n, f0, g0, f, g):
    """sum over the grid prod_i range(n_i) of (f0 + sum_i f_i(x_i)) (g0 + sum_i g_i(x_i)).

    f, g: lists of integer arrays, f[i][x] for x < n[i]."""
    N = _prod(n)
    F = [int(np.sum(fi)) for fi in f]
    G = [int(np.sum(gi)) for gi in g]
    total = f0 * g0 * N
    for i in range(len(n)):
        rest = N // int(n[i])
        total += f0 * G[i] * rest + g0 * F[i] * rest
        total += int(np.sum(np.asarray(f[i], np.int64) * np.asarray(g[i], np.int64))) * rest
    for i in range(len(n)):
        for j in range(len(n)):
            if i != j:
                total += F[i] * G[j] * (N // (int(n[i]) * int(n[j])))
    return total


def diag_terms_writes(cutoffs, has_b=False):
    """(sum over written amplitudes of their complex terms, amplitudes written)
    for the all-detected walk of one circuit (the vacuum seed excluded)."""
    C = [int(c) for c in cutoffs if int(c) >= 2]
    M = len(C)
    terms = writes = 0
    for K in range(M):
        n = [C[K] - 1] + C[K + 1:]
        xK = np.arange(C[K] - 1)
        # terms: 1 (+1 with b) + [e_K >= 1] + 2 sum_m [e_m >= 1]
        f = [(xK >= 1).astype(np.int64)] + [2 * (np.arange(c) >= 1).astype(np.int64) for c in C[K + 1:]]
        # writes: 1 + [e_K <= C_K - 3] + 2 sum_m [e_m <= C_m - 2]
        g = [(xK <= C[K] - 3).astype(np.int64)] + [2 * (np.arange(c) <= c - 2).astype(np.int64)
                                                   for c in C[K + 1:]]
        f0 = 1 + (1 if has_b else 0)
        terms += _sum_product(n, f0, 1, f, g)
        writes += _sum_product(n, 1, 1, [np.zeros_like(fi) for fi in f], g)
    if has_b and M > 0:
        n = [C[0] - 1] + C[1:]
        f = [2 * (np.arange(x) >= 1).astype(np.int64) for x in n]
        g = [(np.arange(C[0] - 1) <= C[0] - 3).astype(np.int64)] + \
            [2 * (np.arange(c) <= c - 2).astype(np.int64) for c in C[1:]]
        terms += _sum_product(n, 1, 1, f, g)
        writes += _sum_product(n, 1, 1, [np.zeros_like(fi) for fi in f], g)
    return terms, writes


def diag_flops(cutoffs, has_b=False):
    """Algorithmic FP64 flops of one circuit's all-detected forward walk."""
    return 8 * diag_terms_writes(cutoffs, has_b)[0]


def cond_terms(cutoffs, detected):
    """Sum of complex terms over the amplitudes of the conditional walk
    (Algorithm 2, Sec. 3.2) of one circuit with b != 0 and one or more
    undetected modes.

    Step 1 (detected part zero): eq. (recrel) over the undetected sub-lattice,
    each u != 0 from u - 1_w (w = its first nonzero index): 1 + #{l : P_l >= 1}
    terms.  Step 2: every detected position y != 0 of the Algorithm-1
    structure (with the offset_1 amplitudes, which the undetected reads need)
    and every u: the detected pivot's terms (b included) plus one per nonzero
    undetected index of u (the read (u - 1_l, P_y))."""
    det = [int(c) for c, d in zip(cutoffs, detected) if d]
    und = [int(c) for c, d in zip(cutoffs, detected) if not d and int(c) >= 2]
    dims = [c for c in und for _ in (0, 1)]
    if dims:
        grid = np.stack(np.meshgrid(*[np.arange(x) for x in dims], indexing="ij"), -1).reshape(-1, len(dims))
    else:
        grid = np.zeros((1, 0), np.int64)
    U2 = grid.shape[0]
    nz_u = (grid >= 1).sum(axis=1)
    step1 = 0
    for u in grid[1:]:
        w = int(np.nonzero(u)[0][0])
        P = u.copy()
        P[w] -= 1
        step1 += 1 + int((P >= 1).sum())
    det_terms, det_writes = diag_terms_writes(det, has_b=True)
    step2 = U2 * det_terms + det_writes * int(nz_u.sum())
    return step1 + step2


def cond_flops(cutoffs, detected):
    return 8 * cond_terms(cutoffs, detected)


def cond_amplitudes(cutoffs, detected):
    """Amplitudes the conditional walk of one circuit stores (b != 0): the
    u-block of every position of the detected Algorithm-1 structure with its
    offset_1 amplitudes, the vacuum position included (U2 (1 + writes))."""
    det = [int(c) for c, d in zip(cutoffs, detected) if d]
    und = [int(c) for c, d in zip(cutoffs, detected) if not d and int(c) >= 2]
    U2 = _prod(c * c for c in und)
    return U2 * (1 + diag_terms_writes(det, has_b=True)[1])

