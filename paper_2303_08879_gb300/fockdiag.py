"""Thin Python binding of the C ABI (include/fockdiag.h).

Argument marshalling only: every step of the walk runs in libfockdiag.so.
PyTorch provides device memory, streams and the autograd hook; no fallback
exists -- a missing or unloadable library raises ``FockError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# FOCKDIAG_LIB selects another build of the same ABI (the debug-checks
# library libfockdiag_debug.so)
LIB_PATH = os.environ.get("FOCKDIAG_LIB") or os.path.join(_HERE, "libfockdiag.so")

FK_OK = 0
FK_ETIMEOUT = 6
FK_ENONFINITE = 7
FK_EBZERO = 8
FK_OP_DIAG, FK_OP_DIAG_VJP, FK_OP_COND, FK_OP_COND_VJP = 1, 2, 3, 4
FK_FLAG_B_ZERO = 1
FK_FLAG_RECOMPUTE = 2
FK_FLAG_ENGINE_FP64 = 0x10
FK_FLAG_ENGINE_TENSOR = 0x20
FK_FLAG_CHECK_FINITE = 0x40

# every symbol the header declares
EXPORTS = [
    "fk_status_string", "fk_version", "fk_gaussian_to_triple", "fk_workspace_size",
    "fock_diag_probs", "fock_diag_probs_batched", "fock_diag_probs_vjp",
    "fock_diag_probs_vjp_batched", "fk_workspace_status", "fk_selftest_wait_timeout",
    "fk_describe_diag_schedule", "fk_measure_fp64_fma_rate", "fock_diag_probs_static",
    "fk_conditional_workspace_size", "fock_conditional_dm", "fock_conditional_dm_batched",
    "fock_conditional_dm_vjp", "fock_conditional_dm_vjp_batched",
    "fk_circuit_triple", "fk_circuit_triple_batched", "fk_mlp_sizes", "fk_mlp_load", "fk_mlp_forward", "fk_mlp_backward", "fk_mlp_train_step",
    "fk_herald_scores", "fk_diag_set_tuning", "fk_diag_set_engine", "fk_diag_set_vjp_split_event",
    "fk_global_size", "fk_global_pattern_index", "fk_global_workspace_size",
    "fock_diag_probs_global_batched", "fock_diag_probs_global_vjp_batched",
    "fk_describe_global_schedule", "fock_diag_probs_stop_batched", "fock_diag_probs_stop_vjp_batched",
    "fk_gaussian_to_pure_triple", "fk_pure_workspace_size", "fock_pure_amplitudes_batched",
    "fock_pure_amplitudes_vjp_batched", "fk_diag_tuning_flags",
    "fk_multi_workspace_size", "fock_diag_probs_multi_batched", "fock_diag_probs_multi_vjp_batched",
    "fk_tc_gemm_bf16", "fk_debug_checks", "fk_workspace_debug", "fk_debug_set_trace",
]


class FockError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = _status_text(status)
        super().__init__(f"{where}: {msg} (status {status})" if where else msg)


_lock = threading.Lock()
_lib = None


def _status_text(st):
    try:
        return lib().fk_status_string(int(st)).decode()
    except Exception:
        return f"status {st}"


def lib():
    """Load libfockdiag.so (raises FockError if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise FockError(-1, f"{LIB_PATH} is not built (run paper_2303_08879_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, U, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t
        L.fk_status_string.argtypes = [I]
        L.fk_status_string.restype = ctypes.c_char_p
        L.fk_version.restype = I
        L.fk_gaussian_to_triple.argtypes = [I, P, P, P, P, P]
        L.fk_workspace_size.argtypes = [I, P, P, I, I, U, ctypes.POINTER(Z)]
        L.fock_diag_probs.argtypes = [P, P, P, I, P, P, P, Z, P]
        L.fock_diag_probs_batched.argtypes = [I, P, P, P, I, P, P, U, P, Z, P]
        L.fock_diag_probs_vjp.argtypes = [P, P, P, I, P, P, P, P, P, P, Z, P]
        L.fock_diag_probs_vjp_batched.argtypes = [I, P, P, P, I, P, P, P, P, P, U, P, Z, P]
        L.fk_workspace_status.argtypes = [P, P, ctypes.POINTER(I)]
        L.fk_selftest_wait_timeout.argtypes = [P, Z, ctypes.c_ulonglong, P]
        L.fk_debug_checks.restype = I
        L.fk_workspace_debug.argtypes = [P, P, P]
        L.fk_debug_set_trace.argtypes = [P, I]
        L.fk_describe_diag_schedule.argtypes = [I, P, U, P, I]
        L.fk_measure_fp64_fma_rate.argtypes = [P, Z, ctypes.POINTER(ctypes.c_double), P]
        L.fock_diag_probs_static.argtypes = [I, P, P, P, I, P, P, U, P, ctypes.POINTER(I)]
        L.fk_global_size.argtypes = [I, I, ctypes.POINTER(ctypes.c_int64)]
        L.fk_global_pattern_index.argtypes = [I, I, P, ctypes.POINTER(ctypes.c_int64)]
        L.fk_global_workspace_size.argtypes = [I, I, I, I, U, ctypes.POINTER(Z)]
        L.fock_diag_probs_global_batched.argtypes = [I, P, P, P, I, I, P, U, P, Z, P]
        L.fock_diag_probs_global_vjp_batched.argtypes = [I, P, P, P, I, I, P, P, P, P, U, P, Z, P]
        L.fk_describe_global_schedule.argtypes = [I, I, U, P, I]
        Dbl = ctypes.c_double
        L.fock_diag_probs_stop_batched.argtypes = [I, P, P, P, I, P, Dbl, P, P, U, P, Z, P]
        L.fock_diag_probs_stop_vjp_batched.argtypes = [I, P, P, P, I, P, Dbl, P, P, P, P, U, P, Z, P]
        L.fk_gaussian_to_pure_triple.argtypes = [I, P, P, P, P, P]
        L.fk_pure_workspace_size.argtypes = [I, I, P, I, U, ctypes.POINTER(Z)]
        L.fock_pure_amplitudes_batched.argtypes = [I, P, P, P, I, P, P, U, P, Z, P]
        L.fock_pure_amplitudes_vjp_batched.argtypes = [I, P, P, P, I, P, P, P, P, P, U, P, Z, P]
        L.fk_diag_set_tuning.argtypes = [I, I, I]
        L.fk_diag_set_engine.argtypes = [I]
        L.fk_diag_tuning_flags.argtypes = [I, I, I, I, ctypes.POINTER(ctypes.c_uint)]
        L.fk_multi_workspace_size.argtypes = [I, I, P, I, U, ctypes.POINTER(Z), P]
        L.fk_tc_gemm_bf16.argtypes = [I, I, I, P, P, P, P, I, P, P]
        L.fock_diag_probs_multi_batched.argtypes = [I, P, P, P, I, P, P, U, P, Z, P]
        L.fock_diag_probs_multi_vjp_batched.argtypes = [I, P, P, P, I, P, P, P, P, P, U, P, Z, P]
        L.fk_diag_set_vjp_split_event.argtypes = [P]
        L.fk_herald_scores.argtypes = [I, P, P, I, P, ctypes.c_double, P, P, P, P]
        L.fk_circuit_triple.argtypes = [I, P, ctypes.c_double, P, P, P, P, P, P]
        L.fk_circuit_triple_batched.argtypes = [I, I, P, ctypes.c_double, P, P, P, P, P, P, I]
        L.fk_conditional_workspace_size.argtypes = [I, I, P, P, I, U, ctypes.POINTER(Z), P]
        L.fock_conditional_dm.argtypes = [P, P, P, I, P, P, P, P, Z, P]
        L.fock_conditional_dm_batched.argtypes = [I, P, P, P, I, P, P, P, U, P, Z, P]
        L.fock_conditional_dm_vjp.argtypes = [P, P, P, I, P, P, P, P, P, P, P, Z, P]
        L.fock_conditional_dm_vjp_batched.argtypes = [I, P, P, P, I, P, P, P, P, P, P, U, P, Z, P]
        for name in EXPORTS:           # fail here, not at first use, if one is missing
            getattr(L, name)
        _lib = L
        return L


def _check(st, where):
    if st != FK_OK:
        raise FockError(st, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _cut(cutoffs):
    return (ctypes.c_int * len(cutoffs))(*[int(c) for c in cutoffs])


def _need_cuda_c128(name, t):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a CUDA complex128 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


# ----------------------------------------------------------------- host side
def fk_gaussian_to_triple(V, mean):
    """Bargmann triple (A, b, c) of a Gaussian state (numpy in, numpy out)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    M = V.shape[0] // 2
    A = np.zeros((2 * M, 2 * M), np.complex128)
    b = np.zeros(2 * M, np.complex128)
    c = np.zeros(1, np.complex128)
    st = lib().fk_gaussian_to_triple(M, V.ctypes.data, mean.ctypes.data, A.ctypes.data,
                                     b.ctypes.data, c.ctypes.data)
    _check(st, "fk_gaussian_to_triple")
    return A, b, complex(c[0])


def fk_circuit_triple(theta, eta, M=3, jacobian=False):
    """(A, b, c[, dA, db, dc]) of the parameterised circuit (numpy, host)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    D = 2 * M
    P = M * M + 2 * M
    assert th.shape == (P,)
    A = np.zeros((D, D), np.complex128); b = np.zeros(D, np.complex128)
    c = np.zeros(1, np.complex128)
    if jacobian:
        dA = np.zeros((P, D, D), np.complex128); db = np.zeros((P, D), np.complex128)
        dc = np.zeros(P, np.complex128)
        ptrs = (dA.ctypes.data, db.ctypes.data, dc.ctypes.data)
    else:
        ptrs = (None, None, None)
    st = lib().fk_circuit_triple(M, th.ctypes.data, float(eta), A.ctypes.data, b.ctypes.data,
                                 c.ctypes.data, *ptrs)
    _check(st, "fk_circuit_triple")
    if jacobian:
        return A, b, complex(c[0]), dA, db, dc
    return A, b, complex(c[0])


def fk_circuit_triple_batched(theta, eta, M=3, jacobian=False, threads=0):
    """Stacked (A, b, c[, dA, db, dc]) for parameter rows theta [n, M^2 + 2M]."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    n, P = th.shape
    D = 2 * M
    assert P == M * M + 2 * M
    A = np.zeros((n, D, D), np.complex128); b = np.zeros((n, D), np.complex128)
    c = np.zeros(n, np.complex128)
    if jacobian:
        dA = np.zeros((n, P, D, D), np.complex128); db = np.zeros((n, P, D), np.complex128)
        dc = np.zeros((n, P), np.complex128)
        ptrs = (dA.ctypes.data, db.ctypes.data, dc.ctypes.data)
    else:
        ptrs = (None, None, None)
    st = lib().fk_circuit_triple_batched(n, M, th.ctypes.data, float(eta), A.ctypes.data,
                                         b.ctypes.data, c.ctypes.data, *ptrs, int(threads))
    _check(st, "fk_circuit_triple_batched")
    return (A, b, c, dA, db, dc) if jacobian else (A, b, c)


def fk_workspace_size(M, cutoffs, batch=1, op=FK_OP_DIAG, flags=0, detected_mask=None):
    n = ctypes.c_size_t(0)
    mask = None
    if detected_mask is not None:
        mask = (ctypes.c_ubyte * M)(*[1 if v else 0 for v in detected_mask])
    st = lib().fk_workspace_size(M, _cut(cutoffs), mask, batch, op, flags, ctypes.byref(n))
    _check(st, "fk_workspace_size")
    return int(n.value)


def fk_describe_diag_schedule(M, cutoffs, flags=0):
    L = sum(max(int(c) - 1, 0) for c in cutoffs)
    n = 3 + 6 * (L + 1)
    out = np.zeros(n, np.int64)
    st = lib().fk_describe_diag_schedule(M, _cut(cutoffs), flags, out.ctypes.data, n)
    _check(st, "fk_describe_diag_schedule")
    lev = int(out[2])
    rows = out[3:3 + 6 * lev].reshape(lev, 6)
    return {"stored": int(out[0]), "pivots": int(out[1]), "levels": lev,
            "per_level": rows}


def workspace(nbytes, device=None):
    """A 256-byte aligned device workspace (torch allocations are)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8,
                       device=device or torch.device("cuda"))


# --------------------------------------------------------------- device side
def fock_diag_probs_batched(A, b, c, cutoffs, probs=None, flags=0, ws=None, stream=None,
                            for_vjp=True):
    """p(n) for a batch of circuits of one shape (Algorithm 1).

    A [B, D, D], b [B, D], c [B] complex128 CUDA tensors.  Returns
    (probs [B, *cutoffs], ws); ``ws`` keeps the walk for a following VJP.
    """
    for n, t in (("A", A), ("b", b), ("c", c)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], len(cutoffs)
    if A.shape != (B, 2 * M, 2 * M) or b.shape != (B, 2 * M) or c.shape != (B,):
        raise ValueError("shapes must be A[B,2M,2M], b[B,2M], c[B]")
    if probs is None:
        probs = torch.empty((B,) + tuple(int(x) for x in cutoffs), dtype=torch.complex128,
                            device=A.device)
    _need_cuda_c128("probs", probs)
    need = fk_workspace_size(M, cutoffs, B, FK_OP_DIAG_VJP if for_vjp else FK_OP_DIAG, flags)
    if ws is None:
        ws = workspace(need, A.device)
    st = lib().fock_diag_probs_batched(B, _ptr(A), _ptr(b), _ptr(c), M, _cut(cutoffs), _ptr(probs),
                                       flags, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_diag_probs_batched")
    return probs, ws


def fock_diag_probs(A, b, c, cutoffs, probs=None, ws=None, stream=None):
    """Single-circuit form: A [D, D], b [D], c [] -> probs [*cutoffs]."""
    p, ws = fock_diag_probs_batched(A.unsqueeze(0), b.unsqueeze(0), c.reshape(1), cutoffs,
                                    None if probs is None else probs.unsqueeze(0), 0, ws, stream)
    return p[0], ws


def fock_diag_probs_vjp_batched(A, b, c, cutoffs, grad_probs, ws, flags=0, stream=None,
                                out=None):
    """(grad_A, grad_b, grad_c) of a batch (PyTorch complex-gradient convention)."""
    for n, t in (("A", A), ("b", b), ("c", c), ("grad_probs", grad_probs)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], len(cutoffs)
    if out is None:
        gA = torch.empty_like(A); gb = torch.empty_like(b); gc = torch.empty_like(c)
    else:
        gA, gb, gc = out
    need = fk_workspace_size(M, cutoffs, B, FK_OP_DIAG_VJP, flags)
    if ws is None:
        ws = workspace(need, A.device)
        flags |= FK_FLAG_RECOMPUTE
    st = lib().fock_diag_probs_vjp_batched(B, _ptr(A), _ptr(b), _ptr(c), M, _cut(cutoffs),
                                           _ptr(grad_probs), _ptr(gA), _ptr(gb), _ptr(gc), flags,
                                           _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_diag_probs_vjp_batched")
    return gA, gb, gc


# ------------------------------------------- per-circuit cutoffs, one launch
def _multi_cut(cutoffs):
    cut = np.ascontiguousarray(np.asarray(cutoffs, dtype=np.int32))
    if cut.ndim != 2:
        raise ValueError("cutoffs must be [batch][M]")
    return cut, cut.shape[0], cut.shape[1]


def fk_multi_workspace_size(cutoffs, op=FK_OP_DIAG_VJP, flags=0):
    """(bytes, out_offsets[B + 1]) of a launch whose circuits have their own cutoffs."""
    cut, B, M = _multi_cut(cutoffs)
    n = ctypes.c_size_t(0)
    offs = np.zeros(B + 1, np.int64)
    _check(lib().fk_multi_workspace_size(B, M, cut.ctypes.data, op, flags, ctypes.byref(n),
                                         offs.ctypes.data), "fk_multi_workspace_size")
    return int(n.value), offs


def multi_blocks(probs, cutoffs):
    """Per-circuit views [*cutoffs[i]] of the packed output."""
    cut, B, M = _multi_cut(cutoffs)
    out, off = [], 0
    for i in range(B):
        n = int(np.prod(cut[i]))
        out.append(probs[off:off + n].view(*(int(x) for x in cut[i])))
        off += n
    return out


def fock_diag_probs_multi_batched(A, b, c, cutoffs, probs=None, flags=0, ws=None, stream=None,
                                  for_vjp=True):
    """p(n) of a batch whose circuits have different cutoffs (cutoffs [B][M];
    unused modes of a circuit get cutoff 1), in one launch.  Returns
    (probs packed [sum_i prod C_i], offsets [B + 1], ws)."""
    for n, t in (("A", A), ("b", b), ("c", c)):
        _need_cuda_c128(n, t)
    cut, B, M = _multi_cut(cutoffs)
    if A.shape != (B, 2 * M, 2 * M) or b.shape != (B, 2 * M) or c.shape != (B,):
        raise ValueError("shapes must be A[B,2M,2M], b[B,2M], c[B]")
    need, offs = fk_multi_workspace_size(cut, FK_OP_DIAG_VJP if for_vjp else FK_OP_DIAG, flags)
    if probs is None:
        probs = torch.empty(int(offs[-1]), dtype=torch.complex128, device=A.device)
    _need_cuda_c128("probs", probs)
    if ws is None:
        ws = workspace(need, A.device)
    st = lib().fock_diag_probs_multi_batched(B, _ptr(A), _ptr(b), _ptr(c), M, cut.ctypes.data, _ptr(probs),
                                             flags, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_diag_probs_multi_batched")
    return probs, offs, ws


def fock_diag_probs_multi_vjp_batched(A, b, c, cutoffs, grad_probs, ws, flags=0, stream=None, out=None):
    """(grad_A, grad_b, grad_c) of a per-circuit-cutoff batch; grad_probs packed
    like the forward's output.  ws = the forward's workspace, or None to
    recompute the forward."""
    for n, t in (("A", A), ("b", b), ("c", c), ("grad_probs", grad_probs)):
        _need_cuda_c128(n, t)
    cut, B, M = _multi_cut(cutoffs)
    if out is None:
        gA = torch.empty_like(A); gb = torch.empty_like(b); gc = torch.empty_like(c)
    else:
        gA, gb, gc = out
    if ws is None:
        ws = workspace(fk_multi_workspace_size(cut, FK_OP_DIAG_VJP, flags)[0], A.device)
        flags |= FK_FLAG_RECOMPUTE
    st = lib().fock_diag_probs_multi_vjp_batched(B, _ptr(A), _ptr(b), _ptr(c), M, cut.ctypes.data,
                                                 _ptr(grad_probs), _ptr(gA), _ptr(gb), _ptr(gc), flags,
                                                 _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_diag_probs_multi_vjp_batched")
    return gA, gb, gc


# ------------------------------------------------------- pure state vector
def fk_gaussian_to_pure_triple(V, mean):
    """(A_psi [M, M], b_psi [M], psi_0) of a pure Gaussian state (host)."""
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
    mean = np.ascontiguousarray(np.asarray(mean, dtype=np.float64))
    M = V.shape[0] // 2
    A = np.zeros((M, M), np.complex128); b = np.zeros(M, np.complex128); c = np.zeros(1, np.complex128)
    st = lib().fk_gaussian_to_pure_triple(M, V.ctypes.data, mean.ctypes.data, A.ctypes.data,
                                          b.ctypes.data, c.ctypes.data)
    _check(st, "fk_gaussian_to_pure_triple")
    return A, b, complex(c[0])


def fk_pure_workspace_size(cutoffs, batch=1, op=FK_OP_DIAG_VJP, flags=0):
    n = ctypes.c_size_t(0)
    _check(lib().fk_pure_workspace_size(int(batch), len(cutoffs), _cut(cutoffs), int(op), int(flags),
                                        ctypes.byref(n)), "fk_pure_workspace_size")
    return int(n.value)


def fock_pure_amplitudes_batched(A, b, c, cutoffs, psi=None, flags=0, ws=None, stream=None):
    """State vectors psi [B, *cutoffs] of pure states (A [B, M, M], b [B, M],
    c [B]).  Returns (psi, ws); ws keeps the walk for a following VJP."""
    for n, t in (("A", A), ("b", b), ("c", c)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], len(cutoffs)
    if A.shape != (B, M, M) or b.shape != (B, M) or c.shape != (B,):
        raise ValueError("shapes must be A[B,M,M], b[B,M], c[B]")
    if psi is None:
        psi = torch.empty((B,) + tuple(int(x) for x in cutoffs), dtype=torch.complex128, device=A.device)
    if ws is None:
        ws = workspace(fk_pure_workspace_size(cutoffs, B, FK_OP_DIAG_VJP, flags), A.device)
    st = lib().fock_pure_amplitudes_batched(B, _ptr(A), _ptr(b), _ptr(c), M, _cut(cutoffs), _ptr(psi),
                                            flags, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_pure_amplitudes_batched")
    return psi, ws


def fock_pure_amplitudes_vjp_batched(A, b, c, cutoffs, grad_psi, ws, flags=0, stream=None):
    for n, t in (("A", A), ("b", b), ("c", c), ("grad_psi", grad_psi)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], len(cutoffs)
    gA = torch.empty_like(A); gb = torch.empty_like(b); gc = torch.empty_like(c)
    if ws is None:
        ws = workspace(fk_pure_workspace_size(cutoffs, B, FK_OP_DIAG_VJP, flags), A.device)
        flags |= FK_FLAG_RECOMPUTE
    st = lib().fock_pure_amplitudes_vjp_batched(B, _ptr(A), _ptr(b), _ptr(c), M, _cut(cutoffs),
                                                _ptr(grad_psi), _ptr(gA), _ptr(gb), _ptr(gc), flags,
                                                _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_pure_amplitudes_vjp_batched")
    return gA, gb, gc


# ------------------------------------------------------------- early stop
def fock_diag_probs_stop_batched(A, b, c, cutoffs, eps, probs=None, flags=0, ws=None, stream=None):
    """Algorithm 1 with the probability-sum stop of Sec. 2.3: per circuit, the
    pivots stop once the probabilities with at most n photons sum to >= 1 - eps.
    Returns (probs [B, *cutoffs] with zeros above the stop, levels [B] = photon
    numbers completed, ws)."""
    for n, t in (("A", A), ("b", b), ("c", c)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], len(cutoffs)
    if A.shape != (B, 2 * M, 2 * M) or b.shape != (B, 2 * M) or c.shape != (B,):
        raise ValueError("shapes must be A[B,2M,2M], b[B,2M], c[B]")
    if probs is None:
        probs = torch.empty((B,) + tuple(int(x) for x in cutoffs), dtype=torch.complex128,
                            device=A.device)
    levels = torch.zeros(B, dtype=torch.int32, device=A.device)
    if ws is None:
        ws = workspace(fk_workspace_size(M, cutoffs, B, FK_OP_DIAG_VJP, flags), A.device)
    st = lib().fock_diag_probs_stop_batched(B, _ptr(A), _ptr(b), _ptr(c), M, _cut(cutoffs),
                                            float(eps), _ptr(probs), _ptr(levels), flags,
                                            _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_diag_probs_stop_batched")
    return probs, levels, ws


def fock_diag_probs_stop_vjp_batched(A, b, c, cutoffs, eps, grad_probs, ws, flags=0, stream=None):
    for n, t in (("A", A), ("b", b), ("c", c), ("grad_probs", grad_probs)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], len(cutoffs)
    gA = torch.empty_like(A); gb = torch.empty_like(b); gc = torch.empty_like(c)
    if ws is None:
        ws = workspace(fk_workspace_size(M, cutoffs, B, FK_OP_DIAG_VJP, flags), A.device)
        flags |= FK_FLAG_RECOMPUTE
    st = lib().fock_diag_probs_stop_vjp_batched(B, _ptr(A), _ptr(b), _ptr(c), M, _cut(cutoffs),
                                                float(eps), _ptr(grad_probs), _ptr(gA), _ptr(gb),
                                                _ptr(gc), flags, _ptr(ws), ws.numel(),
                                                _stream(stream))
    _check(st, "fock_diag_probs_stop_vjp_batched")
    return gA, gb, gc


# ------------------------------------------------------ global photon cutoff
def fk_global_size(M, n_max):
    """Patterns with n_1 + ... + n_M < n_max (outputs per circuit)."""
    n = ctypes.c_int64(0)
    _check(lib().fk_global_size(int(M), int(n_max), ctypes.byref(n)), "fk_global_size")
    return int(n.value)


def fk_global_pattern_index(M, n_max, pattern):
    """Position of a pattern in the level-major output (-1 if outside)."""
    arr = (ctypes.c_int * M)(*[int(v) for v in pattern])
    n = ctypes.c_int64(0)
    _check(lib().fk_global_pattern_index(int(M), int(n_max), arr, ctypes.byref(n)),
           "fk_global_pattern_index")
    return int(n.value)


def fk_global_workspace_size(M, n_max, batch=1, op=FK_OP_DIAG_VJP, flags=0):
    n = ctypes.c_size_t(0)
    _check(lib().fk_global_workspace_size(int(batch), int(M), int(n_max), int(op), int(flags),
                                          ctypes.byref(n)), "fk_global_workspace_size")
    return int(n.value)


def fk_describe_global_schedule(M, n_max, flags=0):
    out = np.zeros(3, np.int64)
    _check(lib().fk_describe_global_schedule(int(M), int(n_max), int(flags), out.ctypes.data, 3),
           "fk_describe_global_schedule")
    return {"allocated": int(out[0]), "pivots": int(out[1]), "outputs": int(out[2])}


def fock_diag_probs_global_batched(A, b, c, n_max, probs=None, flags=0, ws=None, stream=None,
                                   for_vjp=True):
    """p(n) for every pattern with fewer than n_max photons (global cutoff),
    packed level-major [B, fk_global_size(M, n_max)].  Returns (probs, ws)."""
    for n, t in (("A", A), ("b", b), ("c", c)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], A.shape[1] // 2
    if A.shape != (B, 2 * M, 2 * M) or b.shape != (B, 2 * M) or c.shape != (B,):
        raise ValueError("shapes must be A[B,2M,2M], b[B,2M], c[B]")
    if probs is None:
        probs = torch.empty((B, fk_global_size(M, n_max)), dtype=torch.complex128, device=A.device)
    _need_cuda_c128("probs", probs)
    need = fk_global_workspace_size(M, n_max, B, FK_OP_DIAG_VJP if for_vjp else FK_OP_DIAG, flags)
    if ws is None:
        ws = workspace(need, A.device)
    st = lib().fock_diag_probs_global_batched(B, _ptr(A), _ptr(b), _ptr(c), M, int(n_max),
                                              _ptr(probs), flags, _ptr(ws), ws.numel(),
                                              _stream(stream))
    _check(st, "fock_diag_probs_global_batched")
    return probs, ws


def fock_diag_probs_global_vjp_batched(A, b, c, n_max, grad_probs, ws, flags=0, stream=None,
                                       out=None):
    for n, t in (("A", A), ("b", b), ("c", c), ("grad_probs", grad_probs)):
        _need_cuda_c128(n, t)
    B, M = A.shape[0], A.shape[1] // 2
    if out is None:
        gA = torch.empty_like(A); gb = torch.empty_like(b); gc = torch.empty_like(c)
    else:
        gA, gb, gc = out
    if ws is None:
        ws = workspace(fk_global_workspace_size(M, n_max, B, FK_OP_DIAG_VJP, flags), A.device)
        flags |= FK_FLAG_RECOMPUTE
    st = lib().fock_diag_probs_global_vjp_batched(B, _ptr(A), _ptr(b), _ptr(c), M, int(n_max),
                                                  _ptr(grad_probs), _ptr(gA), _ptr(gb), _ptr(gc),
                                                  flags, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_diag_probs_global_vjp_batched")
    return gA, gb, gc


def fk_workspace_status(ws, stream=None):
    v = ctypes.c_int(0)
    st = lib().fk_workspace_status(_ptr(ws), _stream(stream), ctypes.byref(v))
    _check(st, "fk_workspace_status")
    return int(v.value)


def fk_debug_checks():
    """True for the debug-checks build (libfockdiag_debug.so)."""
    return bool(lib().fk_debug_checks())


def fk_workspace_debug(ws, stream=None):
    """Access-violation record of the debug-checks build: (count, source
    line of the first, its index, box start, box end)."""
    out = (ctypes.c_longlong * 5)()
    _check(lib().fk_workspace_debug(_ptr(ws), _stream(stream), out), "fk_workspace_debug")
    return tuple(int(v) for v in out)


def fk_debug_set_trace(buf):
    """Register a zeroed device int64 tensor of 1 + 2 n words for per-level
    timestamps (debug-checks build); None unregisters it."""
    if buf is None:
        _check(lib().fk_debug_set_trace(None, 0), "fk_debug_set_trace")
        return
    _check(lib().fk_debug_set_trace(_ptr(buf), (buf.numel() - 1) // 2), "fk_debug_set_trace")


def check_workspace(ws, stream=None, where="device"):
    st = fk_workspace_status(ws, stream)
    if st != FK_OK:
        raise FockError(st, where)


def fk_selftest_wait_timeout(ws, timeout_ns, stream=None):
    st = lib().fk_selftest_wait_timeout(_ptr(ws), ws.numel(), int(timeout_ns), _stream(stream))
    _check(st, "fk_selftest_wait_timeout")


def fk_measure_fp64_fma_rate(device=None, stream=None):
    """FP64 FMA throughput of the device in TFLOP/s (roofline denominator)."""
    ws = workspace(256, device)
    v = ctypes.c_double(0.0)
    st = lib().fk_measure_fp64_fma_rate(_ptr(ws), ws.numel(), ctypes.byref(v), _stream(stream))
    _check(st, "fk_measure_fp64_fma_rate")
    return float(v.value)


# ------------------------------------------------------ conditional states
def _cond_args(cutoffs, mask):
    cut = np.ascontiguousarray(np.asarray(cutoffs, dtype=np.int32))
    if cut.ndim == 1:
        cut = cut[None, :]
    B, M = cut.shape
    msk = (ctypes.c_ubyte * M)(*[1 if v else 0 for v in mask])
    return cut, B, M, msk


def fk_conditional_workspace_size(cutoffs, mask, op=FK_OP_COND_VJP, flags=0):
    """(workspace bytes, rho offsets [B + 1]) for circuits cutoffs[B][M]."""
    cut, B, M, msk = _cond_args(cutoffs, mask)
    n = ctypes.c_size_t(0)
    offs = np.zeros(B + 1, np.int64)
    st = lib().fk_conditional_workspace_size(B, M, cut.ctypes.data, msk, op, flags,
                                             ctypes.byref(n), offs.ctypes.data)
    _check(st, "fk_conditional_workspace_size")
    return int(n.value), offs


def conditional_blocks(rho, cutoffs, mask):
    """Split the packed output into per-circuit [patterns, ket, bra] views."""
    cut, B, M, _ = _cond_args(cutoffs, mask)
    out, off = [], 0
    for i in range(B):
        npat = int(np.prod([cut[i, j] for j in range(M) if mask[j]]))
        nu = int(np.prod([cut[i, j] for j in range(M) if not mask[j]]))
        out.append(rho[off:off + npat * nu * nu].view(npat, nu, nu))
        off += npat * nu * nu
    return out


def fock_conditional_dm_batched(A, b, c, cutoffs, mask, rho=None, flags=0, ws=None, stream=None,
                                for_vjp=True):
    """Conditional states (Algorithm 2) of a batch; cutoffs[B][M] may differ
    per circuit.  Returns (rho packed, offsets, ws)."""
    for n, t in (("A", A), ("b", b), ("c", c)):
        _need_cuda_c128(n, t)
    cut, B, M, msk = _cond_args(cutoffs, mask)
    if A.shape != (B, 2 * M, 2 * M) or b.shape != (B, 2 * M) or c.shape != (B,):
        raise ValueError("shapes must be A[B,2M,2M], b[B,2M], c[B]")
    need, offs = fk_conditional_workspace_size(cut, mask, FK_OP_COND_VJP if for_vjp else FK_OP_COND,
                                               flags)
    if rho is None:
        rho = torch.empty(int(offs[-1]), dtype=torch.complex128, device=A.device)
    _need_cuda_c128("rho", rho)
    if ws is None:
        ws = workspace(need, A.device)
    st = lib().fock_conditional_dm_batched(B, _ptr(A), _ptr(b), _ptr(c), M, cut.ctypes.data, msk,
                                           _ptr(rho), flags, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_conditional_dm_batched")
    return rho, offs, ws


def fock_conditional_dm_vjp_batched(A, b, c, cutoffs, mask, grad_rho, ws, flags=0, stream=None,
                                    out=None):
    for n, t in (("A", A), ("b", b), ("c", c), ("grad_rho", grad_rho)):
        _need_cuda_c128(n, t)
    cut, B, M, msk = _cond_args(cutoffs, mask)
    if out is None:
        gA = torch.empty_like(A); gb = torch.empty_like(b); gc = torch.empty_like(c)
    else:
        gA, gb, gc = out
    need, _ = fk_conditional_workspace_size(cut, mask, FK_OP_COND_VJP, flags)
    if ws is None:
        ws = workspace(need, A.device)
        flags |= FK_FLAG_RECOMPUTE
    st = lib().fock_conditional_dm_vjp_batched(B, _ptr(A), _ptr(b), _ptr(c), M, cut.ctypes.data,
                                               msk, _ptr(grad_rho), _ptr(gA), _ptr(gb), _ptr(gc),
                                               flags, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fock_conditional_dm_vjp_batched")
    return gA, gb, gc


def fk_diag_set_tuning(tpb=0, ch=0, blocks_per_sm=0):
    _check(lib().fk_diag_set_tuning(int(tpb), int(ch), int(blocks_per_sm)), "fk_diag_set_tuning")


FK_ENGINE_FP64, FK_ENGINE_TENSOR, FK_ENGINE_AUTO = 0, 1, 2


def fk_diag_set_engine(engine):
    """Process-default product engine of the all-detected walk (FK_ENGINE_FP64,
    FK_ENGINE_TENSOR: exact base-256 digit products on the fp16 tensor cores,
    or FK_ENGINE_AUTO, the default: tensor for up to 8 kept modes)."""
    _check(lib().fk_diag_set_engine(int(engine)), "fk_diag_set_engine")


def fk_diag_tuning_flags(engine=FK_ENGINE_AUTO, tpb=0, ch=0, blocks_per_sm=0):
    """Flag bits that select engine and tile shape for one call (OR them into
    `flags`); they take precedence over the process defaults."""
    out = ctypes.c_uint(0)
    _check(lib().fk_diag_tuning_flags(int(engine), int(tpb), int(ch), int(blocks_per_sm),
                                      ctypes.byref(out)), "fk_diag_tuning_flags")
    return int(out.value)


def fk_diag_set_vjp_split_event(event=None):
    """Measurement hook: record `event` (a torch.cuda.Event) between the two
    launches of every following tensor-engine VJP; None switches it off.
    The event must outlive the hook."""
    handle = None if event is None else ctypes.c_void_p(event.cuda_event)
    _check(lib().fk_diag_set_vjp_split_event(handle), "fk_diag_set_vjp_split_event")
