"""Walks run on the debug-checks build of the library (libfockdiag_debug.so,
selected through FOCKDIAG_LIB), one process of their own.  Run by
tests/test_debug_checks_gpu.py; prints one JSON object on stdout.

Every all-detected entry point (one shape, several shapes, global cutoff,
early stop) runs forward + VJP on both product engines, and the conditional
walk (Algorithm 2) forward + VJP, with every access checked against its
storage box; the one-shape and conditional results are compared with the CPU
oracle (1e-10 / 1e-8 relative), and one run records the per-level device
timestamps.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle  # noqa: E402
from oracle import gradients as ograd  # noqa: E402
from paper_2303_08879_gb300 import fockdiag as fd  # noqa: E402
from paper_2303_08879_gb300 import inputs  # noqa: E402


def cuda(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128).cuda()


def errors(got, ref, floor):
    """(largest relative error where |ref| > floor, largest absolute error
    below it, as a multiple of floor)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    big = np.abs(ref) > floor
    rel = float(np.max(np.abs(got - ref)[big] / np.abs(ref[big]))) if big.any() else 0.0
    small = float(np.max(np.abs(got - ref)[~big])) / floor if (~big).any() else 0.0
    return [rel, small]


def oracle_case(cut, withb, batch, seed):
    rng = np.random.default_rng(seed)
    scale = 0.2 if len(cut) <= 4 else 0.12
    A, b, c, P, G, rA, rb = [], [], [], [], [], [], []
    w = rng.normal(size=(batch,) + cut) + 1j * rng.normal(size=(batch,) + cut)
    for i in range(batch):
        Ai, bi = inputs.random_symmetric(2 * len(cut), rng, scale=scale, with_b=withb)
        ci = 0.8 - 0.1j
        Gi = oracle.full_lattice(Ai, bi, ci, oracle.dm_dims(cut))
        gfull = np.zeros_like(Gi)
        pi = np.zeros(cut, np.complex128)
        for n in np.ndindex(*cut):
            k = tuple(v for a in n for v in (a, a))
            pi[n] = Gi[k]
            gfull[k] = w[i][n]
        gA, gb, _ = ograd.vjp(Gi, gfull, ci)
        A.append(Ai); b.append(bi); c.append(ci); P.append(pi); rA.append(gA); rb.append(gb)
    return np.stack(A), np.stack(b), np.array(c), np.stack(P), w, np.stack(rA), np.stack(rb)


def debug_record(ws):
    cnt, site, idx, lo, hi = fd.fk_workspace_debug(ws)
    return {"violations": cnt, "first": None if cnt == 0 else
            {"line": site, "index": idx, "box": [lo, hi]}}


def main():
    out = {"debug_build": fd.fk_debug_checks(), "cases": []}
    for engine, ename in ((fd.FK_ENGINE_FP64, "fp64"), (fd.FK_ENGINE_TENSOR, "tensor")):
        fd.fk_diag_set_engine(engine)
        # one shape per launch: 3 modes (KS = 1), 5 and 8 modes (KS = 2), 9 modes (KS = 3)
        for cut, withb, seed in (((3, 4, 3), True, 1), ((2, 3, 2, 2, 3), False, 2),
                                 ((3, 2, 2, 2, 2, 2, 2, 3), True, 3), ((2,) * 9, False, 4)):
            A, b, c, P, w, rA, rb = oracle_case(cut, withb, 2, seed)
            Ad, bd, cd = cuda(A), cuda(b), cuda(c)
            flags = 0 if withb else fd.FK_FLAG_B_ZERO
            p, ws = fd.fock_diag_probs_batched(Ad, bd, cd, cut, flags=flags)
            fwd = debug_record(ws)
            gA, gb, gc = fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(w), ws, flags=flags)
            vjp = debug_record(ws)
            st = fd.fk_workspace_status(ws)
            floorA = 1e-12 * max(1.0, float(np.max(np.abs(rA))))
            out["cases"].append({
                "what": f"{ename} one shape {cut} b{'!=' if withb else '='}0", "status": st,
                "forward": fwd, "vjp": vjp,
                "probs_err": errors(p.cpu().numpy(), P, 1e-12),
                "gradA_err": errors(gA.cpu().numpy(), rA, floorA),
                "gradb_err": errors(gb.cpu().numpy(), rb, floorA) if withb else [0.0, 0.0]})
        # several shapes in one launch
        rng = np.random.default_rng(5)
        cuts = np.array([[3, 4, 3], [2, 3, 1], [4, 2, 2]], np.int32)
        trip = [inputs.random_symmetric(6, rng, scale=0.2, with_b=True) for _ in range(3)]
        A = cuda(np.stack([t[0] for t in trip])); b = cuda(np.stack([t[1] for t in trip]))
        c = cuda(np.full(3, 0.8 + 0.1j))
        p, offs, ws = fd.fock_diag_probs_multi_batched(A, b, c, cuts)
        fwd = debug_record(ws)
        g = fd.fock_diag_probs_multi_vjp_batched(A, b, c, cuts, torch.ones_like(p), ws)
        vjp = debug_record(ws)
        out["cases"].append({"what": f"{ename} several shapes", "status": fd.fk_workspace_status(ws),
                             "forward": fwd, "vjp": vjp,
                             "finite": bool(torch.isfinite(torch.view_as_real(p)).all()
                                            and all(torch.isfinite(torch.view_as_real(x)).all() for x in g))})
        # global photon cutoff and the early stop
        A1, b1 = inputs.random_symmetric(8, rng, scale=0.2, with_b=True)
        A = cuda(A1[None]); b = cuda(b1[None]); c = cuda(np.array([0.8 + 0.0j]))
        p, ws = fd.fock_diag_probs_global_batched(A, b, c, 6)
        fwd = debug_record(ws)
        fd.fock_diag_probs_global_vjp_batched(A, b, c, 6, torch.ones_like(p), ws)
        out["cases"].append({"what": f"{ename} global cutoff", "status": fd.fk_workspace_status(ws),
                             "forward": fwd, "vjp": debug_record(ws)})
        p, levels, ws = fd.fock_diag_probs_stop_batched(A, b, c, (4, 4, 3, 3), 1e-3)
        fwd = debug_record(ws)
        fd.fock_diag_probs_stop_vjp_batched(A, b, c, (4, 4, 3, 3), 1e-3, torch.ones_like(p), ws)
        out["cases"].append({"what": f"{ename} early stop", "status": fd.fk_workspace_status(ws),
                             "forward": fwd, "vjp": debug_record(ws)})
    # conditional states (Algorithm 2): two undetected-mode layouts, b != 0,
    # against the oracle's full density matrix
    for (cut, mask, seed), (fl, ename) in [(case, e) for case in (((3, 4, 3), (1, 1, 0), 7), ((3, 2, 3, 3), (0, 0, 1, 1), 8))
                                           for e in ((fd.FK_FLAG_ENGINE_TENSOR, "tensor"), (fd.FK_FLAG_ENGINE_FP64, "fp64"))]:
        rng = np.random.default_rng(seed)
        A1, b1 = inputs.random_symmetric(2 * len(cut), rng, with_b=True)
        ref = oracle.full_dm_conditional(A1, b1, 0.6, cut, mask)
        A = cuda(A1[None]); b = cuda(b1[None]); c = cuda(np.array([0.6 + 0.0j]))
        rho, offs, ws = fd.fock_conditional_dm_batched(A, b, c, [cut], mask, flags=fl)
        fwd = debug_record(ws)
        got = fd.conditional_blocks(rho, [cut], mask)[0].cpu().numpy()
        g = fd.fock_conditional_dm_vjp_batched(A, b, c, [cut], mask, torch.ones_like(rho), ws, flags=fl)
        out["cases"].append({"what": f"conditional {ename} {cut} mask {mask}", "status": fd.fk_workspace_status(ws),
                             "forward": fwd, "vjp": debug_record(ws),
                             "probs_err": errors(got, ref, 1e-12),
                             "finite": bool(all(torch.isfinite(torch.view_as_real(x)).all() for x in g))})
    # per-level device timestamps of one forward + VJP (tensor engine, b = 0)
    fd.fk_diag_set_engine(fd.FK_ENGINE_TENSOR)
    buf = torch.zeros(1 + 2 * 256, dtype=torch.int64, device="cuda")
    fd.fk_debug_set_trace(buf)
    cut = (2, 3, 2, 2, 3)
    A, b, c, _, w, _, _ = oracle_case(cut, False, 1, 6)
    p, ws = fd.fock_diag_probs_batched(cuda(A), cuda(b), cuda(c), cut, flags=fd.FK_FLAG_B_ZERO)
    fd.fock_diag_probs_vjp_batched(cuda(A), cuda(b), cuda(c), cut, cuda(w), ws, flags=fd.FK_FLAG_B_ZERO)
    torch.cuda.synchronize()
    fd.fk_debug_set_trace(None)
    fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    t = buf.cpu().numpy().astype(np.uint64)
    n = int(t[0])
    out["trace"] = {"levels": int(sum(c - 1 for c in cut)), "count": n,
                    "tags": [int(x) for x in t[1:1 + 2 * n:2]],
                    "ns": [int(x) for x in t[2:2 + 2 * n:2]]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
