"""Autotuner for the product engine and tile shape of the all-detected walk.

For one workload (shape of the batch, b = 0 or not) it times the tensor-core
engine and every compiled FP64 tile shape (pivots per tile x output rows per
register chunk) with a few caps on resident blocks per SM, forward + VJP,
with CUDA events, and sets the fastest with ``fk_diag_set_engine`` and
``fk_diag_set_tuning``.  Both engines meet the same accuracy bar.  Results
are cached in a JSON file keyed by (modes, cutoffs, batch, flags, device
name) so later runs reuse them.
"""
from __future__ import annotations

import json
import os

import torch

from . import fockdiag as fd

# (engine, pivots per tile, rows per chunk, blocks-per-SM cap); the tensor
# engine has one tile shape (128 pivots) and ignores the chunk size.
TENSOR, FP64 = "tensor", "fp64"
CANDIDATES = [(TENSOR, 128, 4, 0),
              (FP64, 128, 8, 0), (FP64, 128, 4, 0), (FP64, 64, 8, 0), (FP64, 64, 4, 0), (FP64, 256, 8, 0),
              (FP64, 128, 8, 2), (FP64, 128, 4, 3), (FP64, 64, 8, 4)]


def apply(cand):
    """Set engine and tile shape of a candidate."""
    engine, tpb, ch, cap = cand
    fd.fk_diag_set_engine(fd.FK_ENGINE_TENSOR if engine == TENSOR else fd.FK_ENGINE_FP64)
    fd.fk_diag_set_tuning(tpb, ch, cap)


def _name(cand):
    return "%s/%d/%d/%d" % cand


def _parse(name):
    e, t, c, b = name.split("/")
    return (e, int(t), int(c), int(b))


def _key(cutoffs, batch, flags):
    name = torch.cuda.get_device_name()
    return f"diag|C={','.join(str(int(c)) for c in cutoffs)}|B={batch}|flags={flags}|{name}"


def _load(path):
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def tune_diag(A, b, c, cutoffs, grad_probs, flags=0, steps=2, cache_path=None,
              candidates=CANDIDATES):
    """Pick and set the fastest engine and tile shape for this batch; returns
    (best candidate, {candidate: ms per forward + VJP})."""
    cache = _load(cache_path)
    key = _key(cutoffs, A.shape[0], flags)
    if key in cache:
        best = _parse(cache[key]["best"])
        apply(best)
        return best, cache[key]["ms"]
    M = len(cutoffs)
    B = A.shape[0]
    times = {}
    probs = torch.empty((B,) + tuple(cutoffs), dtype=torch.complex128, device=A.device)
    gA, gb, gc = torch.empty_like(A), torch.empty_like(b), torch.empty_like(c)
    for cand in candidates:
        try:
            apply(cand)
            ws = fd.workspace(fd.fk_workspace_size(M, cutoffs, B, fd.FK_OP_DIAG_VJP, flags), A.device)
        except fd.FockError:
            continue
        run = lambda: (fd.fock_diag_probs_batched(A, b, c, cutoffs, probs=probs, flags=flags, ws=ws),
                       fd.fock_diag_probs_vjp_batched(A, b, c, cutoffs, grad_probs, ws, flags=flags,
                                                      out=(gA, gb, gc)))
        run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            run()
        e1.record()
        torch.cuda.synchronize()
        fd.check_workspace(ws, where="autotune")
        times[_name(cand)] = e0.elapsed_time(e1) / steps
        del ws
    best_s = min(times, key=times.get)
    best = _parse(best_s)
    apply(best)
    if cache_path:
        cache[key] = {"best": best_s, "ms": times}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best, times
