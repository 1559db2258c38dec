"""Device timings of the walk's variants on the bench circuits (CUDA events,
tensor-core engine where it applies): the probability-sum early stop
(Sec. 2.3), the global photon-number cutoff and the state-vector walk of pure
states (Sec. 2.2), each forward and VJP.

    python -m paper_2303_08879_gb300.rows [--cond]

--cond runs only the 64-circuit conditional workload (forward + VJP, twice).
"""
from __future__ import annotations

import json

import numpy as np


def _time(fn, reps=5, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def cond_once(reps=2):
    """The 64-circuit conditional workload, forward + VJP, reps times (for
    profiling the conditional-walk kernels)."""
    import torch
    from . import fockdiag as fd
    from . import inputs
    mask = (1, 1, 0)
    circs = inputs.workload("cond_m3_batch64")
    cuts = [cc.cutoffs for cc in circs]
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = torch.tensor(np.stack([t[0] for t in trip]), device="cuda")
    b = torch.tensor(np.stack([t[1] for t in trip]), device="cuda")
    c = torch.tensor(np.array([t[2] for t in trip], np.complex128), device="cuda")
    rho, offs, ws = fd.fock_conditional_dm_batched(A, b, c, cuts, mask)
    g = torch.ones_like(rho)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd = vjp = 0.0
    for _ in range(reps):
        ev[0].record()
        fd.fock_conditional_dm_batched(A, b, c, cuts, mask, rho=rho, ws=ws)
        ev[1].record()
        fd.fock_conditional_dm_vjp_batched(A, b, c, cuts, mask, g, ws)
        ev[2].record()
        torch.cuda.synchronize()
        fwd += ev[0].elapsed_time(ev[1]); vjp += ev[1].elapsed_time(ev[2])
    fd.check_workspace(ws)
    print(json.dumps({"conditional_outputs": int(offs[-1]), "reps": reps, "forward_ms": fwd / reps,
                      "vjp_ms": vjp / reps}))


def main():
    import sys
    if "--cond" in sys.argv:
        cond_once()
        return
    import torch
    from . import fockdiag as fd
    from . import inputs

    dev = torch.device("cuda")
    circs = inputs.workload("gbs_m8_c6_batch16")
    cut = circs[0].cutoffs
    M = len(cut)
    trip = [fd.fk_gaussian_to_triple(c.V, c.mean) for c in circs]
    A = torch.tensor(np.stack([t[0] for t in trip]), device=dev)
    b = torch.tensor(np.stack([t[1] for t in trip]), device=dev)
    c = torch.tensor(np.array([t[2] for t in trip], np.complex128), device=dev)
    flags = fd.FK_FLAG_B_ZERO
    fd.fk_diag_set_engine(fd.FK_ENGINE_TENSOR)
    out = {"circuits": len(circs), "modes": M, "cutoff": int(cut[0]), "engine": "tensor"}
    g = tuple(torch.empty_like(x) for x in (A, b, c))

    # early stop at eps = 1e-3
    eps = 1e-3
    p, lv, ws = fd.fock_diag_probs_stop_batched(A, b, c, cut, eps, flags=flags)
    w = torch.ones_like(p)
    fwd = _time(lambda: fd.fock_diag_probs_stop_batched(A, b, c, cut, eps, probs=p, flags=flags, ws=ws))
    vjp = _time(lambda: fd.fock_diag_probs_stop_vjp_batched(A, b, c, cut, eps, w, ws, flags=flags))
    fd.check_workspace(ws)
    out["early_stop"] = {"eps": eps, "photon_numbers_completed_mean": float(lv.float().mean()),
                         "forward_ms": fwd, "vjp_ms": vjp}
    del p, w, ws
    torch.cuda.empty_cache()

    # global cutoff: every pattern with fewer than n_max photons
    n_max = 8
    p, ws = fd.fock_diag_probs_global_batched(A, b, c, n_max, flags=flags)
    w = torch.ones_like(p)
    fwd = _time(lambda: fd.fock_diag_probs_global_batched(A, b, c, n_max, probs=p, flags=flags, ws=ws))
    vjp = _time(lambda: fd.fock_diag_probs_global_vjp_batched(A, b, c, n_max, w, ws, flags=flags, out=g))
    fd.check_workspace(ws)
    out["global_cutoff"] = {"n_max": n_max, "outputs_per_circuit": fd.fk_global_size(M, n_max),
                            "forward_ms": fwd, "vjp_ms": vjp}
    del p, w, ws
    torch.cuda.empty_cache()

    # state-vector walk of 16 pure 8-mode states (no loss), cutoff 6 per mode
    rng = np.random.default_rng(11)
    pure = [inputs.make_circuit(M, rng, r_range=(0.1, 0.8), eta_range=(1.0, 1.0), alpha_var=0.3,
                                cutoffs=cut) for _ in range(len(circs))]
    pt = [fd.fk_gaussian_to_pure_triple(pc.V, pc.mean) for pc in pure]
    Ap = torch.tensor(np.stack([t[0] for t in pt]), device=dev)
    bp = torch.tensor(np.stack([t[1] for t in pt]), device=dev)
    cp = torch.tensor(np.array([t[2] for t in pt], np.complex128), device=dev)
    psi, ws = fd.fock_pure_amplitudes_batched(Ap, bp, cp, cut)
    w = torch.ones_like(psi)
    fwd = _time(lambda: fd.fock_pure_amplitudes_batched(Ap, bp, cp, cut, psi=psi, ws=ws))
    vjp = _time(lambda: fd.fock_pure_amplitudes_vjp_batched(Ap, bp, cp, cut, w, ws))
    fd.check_workspace(ws)
    out["state_vector"] = {"amplitudes_per_state": int(np.prod(cut)), "forward_ms": fwd,
                           "vjp_ms": vjp, "engine": "fp64"}
    fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
