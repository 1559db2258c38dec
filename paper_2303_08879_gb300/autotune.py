"""Autotuner for the tile shape of the all-detected walk.

For one workload (shape of the batch, b = 0 or not) it times every compiled
tile shape (pivots per tile x output rows per register chunk) and a few caps
on resident blocks per SM, forward + VJP, with CUDA events, and sets the
fastest with ``fk_diag_set_tuning``.  Results are cached in a JSON file keyed
by (modes, cutoffs, batch, flags, device name) so later runs reuse them.
"""
from __future__ import annotations

import json
import os

import torch

from . import fockdiag as fd

CANDIDATES = [(128, 8, 0), (128, 4, 0), (64, 8, 0), (64, 4, 0), (256, 8, 0),
              (128, 8, 2), (128, 4, 3), (64, 8, 4)]


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
    """Pick and set the fastest tile shape for this batch; returns
    (best candidate, {candidate: ms per forward + VJP})."""
    cache = _load(cache_path)
    key = _key(cutoffs, A.shape[0], flags)
    if key in cache:
        best = tuple(cache[key]["best"])
        fd.fk_diag_set_tuning(*best)
        return best, cache[key]["ms"]
    M = len(cutoffs)
    B = A.shape[0]
    times = {}
    probs = torch.empty((B,) + tuple(cutoffs), dtype=torch.complex128, device=A.device)
    gA, gb, gc = torch.empty_like(A), torch.empty_like(b), torch.empty_like(c)
    for cand in candidates:
        try:
            fd.fk_diag_set_tuning(*cand)
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
        times["%d/%d/%d" % cand] = e0.elapsed_time(e1) / steps
        del ws
    best_s = min(times, key=times.get)
    best = tuple(int(v) for v in best_s.split("/"))
    fd.fk_diag_set_tuning(*best)
    if cache_path:
        cache[key] = {"best": list(best), "ms": times}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best, times
