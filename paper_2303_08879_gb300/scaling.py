"""Storage and time of the all-detected walk as functions of the cutoff: the
quantities of Fig. 8 (stored amplitudes against pivots applied, with and
without the buffer of Sec. 3.1.4) and Fig. 10 (memory and time against a
common cutoff C at M = 4), counted from the walk's schedule and timed on the
device kernels.

Counting (b = 0, Algorithm 1 with the canonical pivots of Sec. 3.1.3): the
pivots of level s (digit sum s) are the AP(K) pivots e (modes < K zero,
e_K <= C_K - 2).  Each writes one diagonal value, T2(K)[e] when
e_K <= C_K - 3 and the pair P1010/P1001(K,m)[e] for every m > K with
e_m <= C_m - 2.  Every off-diagonal value is read by exactly one pivot, one
level later (Sec. 3.1.4), so with the buffer strategy the values written at
level s can be dropped once level s + 1 is done.

    python -m paper_2303_08879_gb300.scaling [--time]
"""
from __future__ import annotations

import itertools
import json
import math
import sys

import numpy as np


def level_counts(cutoffs):
    """Per pivot level s: (pivots, diagonal writes, off-diagonal writes)."""
    C = [int(c) for c in cutoffs if c >= 2]
    M = len(C)
    L = sum(c - 1 for c in C)
    piv = np.zeros(L + 1, np.int64)
    dia = np.zeros(L + 1, np.int64)
    off = np.zeros(L + 1, np.int64)
    for K in range(M):
        ranges = [range(C[K] - 1)] + [range(C[m]) for m in range(K + 1, M)]
        grid = np.array(list(itertools.product(*ranges)), dtype=np.int64).reshape(-1, M - K)
        s = grid.sum(axis=1)
        eK = grid[:, 0]
        n_off = (eK <= C[K] - 3).astype(np.int64)
        for j, m in enumerate(range(K + 1, M), start=1):
            n_off += 2 * (grid[:, j] <= C[m] - 2)
        np.add.at(piv, s, 1)
        np.add.at(dia, s, 1)
        np.add.at(off, s, n_off)
    return piv, dia, off


def buffer_curve(cutoffs):
    """Fig. 8 per level: pivots applied so far, amplitudes stored without a
    buffer and with the buffer strategy (after each level)."""
    piv, dia, off = level_counts(cutoffs)
    applied = np.cumsum(piv)
    no_buffer = 1 + np.cumsum(dia + off)          # + the vacuum amplitude
    diag_done = 1 + np.cumsum(dia)
    with_buffer = diag_done + off                  # level s's off-diagonals await level s + 1
    # while level s runs, the inputs of level s - 1 are still held
    peak_during = diag_done + off + np.concatenate([[0], off[:-1]])
    return {"pivots": applied, "no_buffer": no_buffer, "buffer": with_buffer,
            "buffer_peak_during": peak_during}


def slope(x, y):
    """Least-squares slope of log y against log x over the upper half of x."""
    x = np.asarray(x, float); y = np.asarray(y, float)
    h = len(x) // 2
    return float(np.polyfit(np.log(x[h:]), np.log(y[h:]), 1)[0])


def space_table(M, cs):
    """Fig. 10a: amplitudes for a common cutoff C: state vector C^M, naive
    density matrix C^(2M), Algorithm 1 without / with buffer."""
    rows = []
    for C in cs:
        bc = buffer_curve((C,) * M)
        rows.append({"C": C, "state_vector": C ** M, "naive_dm": C ** (2 * M),
                     "algorithm1": int(bc["no_buffer"][-1]),
                     "algorithm1_buffer_peak": int(bc["buffer_peak_during"].max()),
                     "pivots": int(bc["pivots"][-1])})
    return rows


def time_table(M, cs, batch=64, reps=5, seed=0):
    """Fig. 10b on the device: forward and forward + VJP time per circuit of a
    batch of random GBS circuits, and the workspace per circuit."""
    import torch
    from . import fockdiag as fd
    from . import inputs
    rows = []
    for C in cs:
        rng = np.random.default_rng(seed + C)
        circs = [inputs.make_circuit(M, rng, r_range=(0.3, 1.0), eta_range=(0.6, 1.0),
                                     cutoffs=(C,) * M) for _ in range(batch)]
        trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
        A = torch.from_numpy(np.stack([t[0] for t in trip])).cuda()
        b = torch.from_numpy(np.stack([t[1] for t in trip])).cuda()
        c = torch.from_numpy(np.array([t[2] for t in trip], np.complex128)).cuda()
        cut = (C,) * M
        flags = fd.FK_FLAG_B_ZERO
        p, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags)
        w = torch.ones_like(p)
        out = tuple(torch.empty_like(x) for x in (A, b, c))
        fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags, out=out)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fwd = vjp = 0.0
        for _ in range(reps):
            ev[0].record()
            fd.fock_diag_probs_batched(A, b, c, cut, probs=p, flags=flags, ws=ws)
            ev[1].record()
            fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags, out=out)
            ev[2].record()
            torch.cuda.synchronize()
            fwd += ev[0].elapsed_time(ev[1]); vjp += ev[1].elapsed_time(ev[2])
        fd.check_workspace(ws)
        rows.append({"C": C, "batch": batch, "forward_ms_per_circuit": fwd / reps / batch,
                     "vjp_ms_per_circuit": vjp / reps / batch,
                     "workspace_bytes_per_circuit": ws.numel() // batch})
        del p, ws, w
        torch.cuda.empty_cache()
    return rows


def main(argv):
    out = {}
    bc = buffer_curve((10,) * 4)
    out["fig8_M4_C10"] = {k: v.tolist() for k, v in bc.items()}
    cs = [4, 5, 6, 7, 8, 10, 12, 14, 16]
    sp = space_table(4, cs)
    out["fig10_space_M4"] = sp
    out["fig10_space_slopes"] = {k: slope(cs, [r[k] for r in sp])
                                 for k in ("state_vector", "naive_dm", "algorithm1",
                                           "algorithm1_buffer_peak", "pivots")}
    if "--time" in argv:
        from . import fockdiag as fd
        for engine, name in ((fd.FK_ENGINE_FP64, "fp64"), (fd.FK_ENGINE_TENSOR, "tensor")):
            fd.fk_diag_set_engine(engine)
            tt = time_table(4, cs)
            out[f"fig10_time_M4_{name}"] = tt
            out[f"fig10_time_slopes_{name}"] = {
                k: slope(cs, [r[k] for r in tt])
                for k in ("forward_ms_per_circuit", "vjp_ms_per_circuit", "workspace_bytes_per_circuit")}
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1:])
