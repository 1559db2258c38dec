"""CPU oracle for the Fock-amplitude recurrence of arXiv 2303.08879.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library
(``paper_2303_08879_gb300``) and never imports it.

Contents
  triple        -- Gaussian (sigma, mu) -> Bargmann triple (A, b, c),
                   eqs. (A_rho), (b_rho) and the vacuum amplitude of Sec. 2.2.
  full_lattice  -- O1: eq. (recrel) over every index of a box (plain
                   definition of the density matrix), with a forward-mode
                   tangent (eqs. recrel_dB, recrel_dA of Sec. 2.5).
  Walk          -- O2: Algorithms 1 and 2 written naively as a memoised walk.
  hafnian       -- brute-force loop hafnian (an independent definition used
                   only to pin O1).
  gradients     -- closed-form derivatives of the amplitudes and the
                   vector-Jacobian product of Sec. 2.5, eqs. (dL_dB), (dL_dA).

Every function's docstring cites the passage of the paper it follows.
Parity status: every function here is pinned by tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .triple import gaussian_to_triple  # noqa: F401
from . import hafnian, gradients  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fock_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, no fast-math, FP contraction off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.or_full_lattice.argtypes = [I, P, P, P, P, P, P, P, P, P]
            lib.or_full_lattice.restype = I
            lib.or_walk_new.argtypes = [I, P, P, P, P, P, P, P, P]
            lib.or_walk_new.restype = P
            lib.or_walk_free.argtypes = [P]
            lib.or_walk_free.restype = None
            lib.or_walk_amplitude.argtypes = [P, P, P, P]
            lib.or_walk_amplitude.restype = I
            lib.or_walk_prob.argtypes = [P, P, P, P]
            lib.or_walk_prob.restype = I
            lib.or_walk_all_probs.argtypes = [P, P, P]
            lib.or_walk_all_probs.restype = I
            lib.or_walk_all_conditional.argtypes = [P, P, P]
            lib.or_walk_all_conditional.restype = I
            lib.or_walk_stats.argtypes = [P, P]
            lib.or_walk_stats.restype = None
            lib.or_walk_level_hist.argtypes = [P, P, I]
            lib.or_walk_level_hist.restype = None
            _lib = lib
    return _lib


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def full_lattice(A, b, c, dims, tangent=None):
    """O1: every amplitude G_k for 0 <= k < dims by eq. (recrel), Sec. 2.1-2.2.

    dims has one entry per lattice index (D entries; a density matrix of M
    modes with cutoffs C uses dims = (C_1, C_1, C_2, C_2, ...)).  Returns the
    array of shape dims, and its tangent along ``tangent = (dA, db, dc)``
    (eqs. recrel_dA, recrel_dB of Sec. 2.5) when given.
    """
    lib = _load()
    A = _c128(A); b = _c128(b)
    D = len(dims)
    assert A.shape == (D, D) and b.shape == (D,)
    cc = _c128([c])
    G = np.zeros(tuple(dims), np.complex128)
    if tangent is not None:
        dA, db, dc = _c128(tangent[0]), _c128(tangent[1]), _c128([tangent[2]])
        Gd = np.zeros_like(G)
    else:
        dA = db = dc = Gd = None
    dd = np.asarray(dims, dtype=np.int32)
    rc = lib.or_full_lattice(D, _ptr(dd), _ptr(A), _ptr(b), _ptr(cc), _ptr(dA), _ptr(db),
                             _ptr(dc), _ptr(G), _ptr(Gd))
    if rc != 0:
        raise RuntimeError(f"or_full_lattice failed ({rc})")
    return (G, Gd) if tangent is not None else G


def dm_dims(cutoffs):
    return tuple(int(c) for c in cutoffs for _ in (0, 1))


def full_dm_probs(A, b, c, cutoffs):
    """p(n) = G_{n1 n1 n2 n2 ...} from the full density matrix (Sec. 3.1)."""
    G = full_lattice(A, b, c, dm_dims(cutoffs))
    M = len(cutoffs)
    out = np.zeros(tuple(cutoffs), np.complex128)
    for n in np.ndindex(*cutoffs):
        out[n] = G[tuple(v for a in n for v in (a, a))]
    return out


def full_dm_conditional(A, b, c, cutoffs, detected):
    """Diagonal blocks of the full density matrix (Sec. 3.2): rho[pattern][ket][bra]."""
    G = full_lattice(A, b, c, dm_dims(cutoffs))
    M = len(cutoffs)
    det = [j for j in range(M) if detected[j]]
    und = [j for j in range(M) if not detected[j]]
    NU = int(np.prod([cutoffs[j] for j in und])) if und else 1
    NP = int(np.prod([cutoffs[j] for j in det])) if det else 1
    out = np.zeros((NP, NU, NU), np.complex128)
    for p, n in enumerate(np.ndindex(*[cutoffs[j] for j in det])):
        for kk, ket in enumerate(np.ndindex(*[cutoffs[j] for j in und])):
            for bb, bra in enumerate(np.ndindex(*[cutoffs[j] for j in und])):
                x = [0] * (2 * M)
                for a, j in enumerate(det):
                    x[2 * j] = x[2 * j + 1] = n[a]
                for a, j in enumerate(und):
                    x[2 * j] = ket[a]
                    x[2 * j + 1] = bra[a]
                out[p, kk, bb] = G[tuple(x)]
    return out


class Walk:
    """O2: naive Algorithm 1 / Algorithm 2 (Sec. 3.1.3, 3.2) as a memoised walk.

    Each amplitude is written from the pivot that Algorithm 1 applies to it
    (diagonal pivots for offset_1 types, off-diagonal pivots diag + 1_{2K-1}
    anchored at the first nonzero mode for the rest); undetected modes keep
    their full (ket, bra) indices (Algorithm 2).  ``tangent = (dA, db, dc)``
    carries the forward-mode derivative of eqs. (recrel_dB), (recrel_dA)
    along one direction through the same walk.
    """

    def __init__(self, A, b, c, cutoffs, detected=None, tangent=None):
        self._lib = _load()
        self.M = len(cutoffs)
        self.cutoffs = tuple(int(x) for x in cutoffs)
        D = 2 * self.M
        self._A = _c128(A); self._b = _c128(b); self._c = _c128([c])
        assert self._A.shape == (D, D) and self._b.shape == (D,)
        self._cut = np.asarray(self.cutoffs, np.int32)
        self._det = None if detected is None else np.asarray([1 if v else 0 for v in detected], np.uint8)
        self.detected = tuple([True] * self.M) if detected is None else tuple(bool(v) for v in detected)
        if tangent is not None:
            self._dA, self._db, self._dc = _c128(tangent[0]), _c128(tangent[1]), _c128([tangent[2]])
        else:
            self._dA = self._db = self._dc = None
        self._h = self._lib.or_walk_new(self.M, _ptr(self._cut), _ptr(self._det), _ptr(self._A),
                                        _ptr(self._b), _ptr(self._c), _ptr(self._dA), _ptr(self._db),
                                        _ptr(self._dc))
        if not self._h:
            raise RuntimeError("or_walk_new failed")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.or_walk_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def amplitude(self, x):
        x = np.asarray(x, np.int32)
        g = np.zeros(1, np.complex128); t = np.zeros(1, np.complex128)
        rc = self._lib.or_walk_amplitude(self._h, _ptr(x), _ptr(g), _ptr(t))
        if rc:
            raise RuntimeError(f"walk failed ({rc}) at {x.tolist()}")
        return g[0], t[0]

    def prob(self, n):
        n = np.asarray(n, np.int32)
        g = np.zeros(1, np.complex128); t = np.zeros(1, np.complex128)
        rc = self._lib.or_walk_prob(self._h, _ptr(n), _ptr(g), _ptr(t))
        if rc:
            raise RuntimeError(f"walk failed ({rc}) at pattern {n.tolist()}")
        return g[0], t[0]

    def all_probs(self, with_tangent=False):
        out = np.zeros(self.cutoffs, np.complex128)
        od = np.zeros_like(out) if with_tangent else None
        rc = self._lib.or_walk_all_probs(self._h, _ptr(out), _ptr(od))
        if rc:
            raise RuntimeError(f"walk failed ({rc})")
        return (out, od) if with_tangent else out

    def all_conditional(self, with_tangent=False):
        det = [j for j in range(self.M) if self.detected[j]]
        und = [j for j in range(self.M) if not self.detected[j]]
        NP = int(np.prod([self.cutoffs[j] for j in det])) if det else 1
        NU = int(np.prod([self.cutoffs[j] for j in und])) if und else 1
        out = np.zeros((NP, NU, NU), np.complex128)
        od = np.zeros_like(out) if with_tangent else None
        rc = self._lib.or_walk_all_conditional(self._h, _ptr(out), _ptr(od))
        if rc:
            raise RuntimeError(f"walk failed ({rc})")
        return (out, od) if with_tangent else out

    def level_hist(self, nlev):
        """[nlev, 6] counts of stored amplitudes per level and type (diag,
        offset_1 ket, offset_1 bra, offset_2, offset_1010, offset_1001); level
        s holds total weight 2s (2s+1 for offset_1)."""
        h = np.zeros(6 * nlev, np.int64)
        self._lib.or_walk_level_hist(self._h, _ptr(h), nlev)
        return h.reshape(nlev, 6)

    def stats(self):
        s = np.zeros(9, np.int64)
        self._lib.or_walk_stats(self._h, _ptr(s))
        keys = ["diag", "off1_ket", "off1_bra", "off2", "off1010", "off1001",
                "pivots", "stored", "undetected_block"]
        return dict(zip(keys, (int(v) for v in s)))
