"""Benchmark of the all-detected Fock walk (Algorithm 1) forward + VJP.

Workload: 16 synthetic noisy GBS circuits, M = 8 modes, all PNR-detected,
cutoff C = 6 per mode (6^8 = 1.68 M probabilities each), squeezing
r ~ U[0.3, 1], Haar 8x8 interferometer, loss eta ~ U[0.6, 1], no
displacement (b = 0).  One step = the forward walk of all 16 circuits plus
the VJP of L = sum_n w_n Re p_n (w ~ N(0, 1)) with respect to A, b and c.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  ``value`` = probabilities (diagonal Fock amplitudes)
per second over the whole job, inputs resident on the device; ``e2e`` = the
same through the public API with pinned host buffers (every step's
host<->device copies inside the timed region, on a copy stream that overlaps
them with the neighbouring steps' walks); ``vs_plain`` = batched forward + VJP
circuits/s over the same circuits run as single-circuit calls.  ``rows``
holds the other workloads: the 64-circuit conditional walk, the BF16 MLP
step, the 2-mode latency case, the 12-mode circuit, Fig. 10b timings and the
learned-proposal comparison.  Under torchrun each rank runs its own 16
circuits (weak scaling, no collective on the data path).
``--impl reference`` times the CPU oracle (naive Algorithm 1) instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "gbs_m8_c6_batch16"
METRIC = "Fock diag amplitudes/s (c128); fwd+VJP circuits/s vs plain, rel err<=1e-10"
UNIT = "amplitudes/s"
NCIRC = 16

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# each walk kernel on this 16-circuit workload, captured with ncu on a
# 2-circuit launch and scaled by 8: circuits share no data, so traffic grows
# in proportion to them.  Valid only for the kernel source it was measured on
# (sha256 prefix of csrc/walk_diag_impl.cuh + walk_digits.cuh + walk_common.cuh)
# and the engine / tile shape; reported as null once either differs.
TRAFFIC = {"kernel_sha": "9b3fd66c1972b7e8", "tuning": ["tensor", 128, 4, 0],
           "bytes_per_launch": {"diag_forward_kernel": 8 * (496652800 + 853942272),
                                "diag_vjp_kernel": 8 * (707781888 + 722182144),
                                "diag_vjp_partials_kernel": 8 * (1729087744 + 132293120)}}

FALLBACK_HBM_GBS = 6800.0


def measured_hbm_gbs():
    """HBM copy bandwidth of this GPU model from MEASURED_PEAKS.json."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def kernel_sha():
    """sha256 prefix of the walk kernels' source (csrc/walk_diag_impl.cuh, the
    digit primitives of csrc/walk_digits.cuh and the grid barrier and helpers
    of csrc/walk_common.cuh)."""
    h = hashlib.sha256()
    for name in ("walk_diag_impl.cuh", "walk_digits.cuh", "walk_common.cuh"):
        with open(os.path.join(ROOT, "paper_2303_08879_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------- counting
def algorithmic_flops(cut, has_b=False):
    """8 x sum over written amplitudes of their complex terms (counts.py)."""
    from paper_2303_08879_gb300 import counts
    return counts.diag_flops(cut, has_b)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle
def oracle_sample(budget_s, first_circuit=0):
    """Time the oracle's naive Algorithm 1 walk on a sub-box of one circuit's
    probabilities sized to ~budget_s seconds (forward only)."""
    import oracle
    from oracle import triple as ot
    from paper_2303_08879_gb300 import inputs
    circ = inputs.workload(WORKLOAD, 1, start=first_circuit)[0]
    A, b, c = ot.gaussian_to_triple(circ.V, circ.mean)
    cut = list(circ.cutoffs)
    rate_guess = 6.0e4                     # probabilities per second, one core
    while np.prod(cut) > rate_guess * budget_s and min(cut) > 1:
        j = max(i for i in range(len(cut)) if cut[i] == max(cut))
        cut[j] -= 1
    t0 = time.perf_counter()
    w = oracle.Walk(A, b, c, tuple(cut))
    P = w.all_probs()
    dt = time.perf_counter() - t0
    w.close()
    return int(P.size), dt, tuple(cut)


def host_cpu():
    """CPU model and the cores this process may use (for the baseline lines)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            model = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            model = next((ln.split(":", 1)[1].strip() for ln in model.splitlines()
                          if ln.lower().startswith("model name")), None)
        except Exception:
            model = None
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    import platform
    return {"model": model or platform.processor() or platform.machine(), "nproc": n,
            "machine": platform.machine()}


def _oracle_worker(job):
    budget, circuit = job
    return oracle_sample(budget, circuit)


def oracle_all_cores(budget_s, n_workers):
    """The same bounded oracle sample on every host core at once, one circuit
    per process (spawned, so no process is forked from a CUDA context):
    probabilities of all processes over the wall time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(n_workers) as pool:
        res = pool.map(_oracle_worker, [(budget_s, i % NCIRC) for i in range(n_workers)])
    wall = time.perf_counter() - t0
    return sum(r[0] for r in res), wall, res[0][2]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup):
        oracle_sample(budget, i % NCIRC)
    n_tot, t_tot, cut = 0, 0.0, None
    for i in range(args.steps):
        n, dt, cut = oracle_sample(budget, (args.warmup + i) % NCIRC)
        n_tot += n
        t_tot += dt
    value = n_tot / t_tot
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": config_block(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host": host_cpu(),
                         "sample": f"naive Algorithm 1 walk (forward only), probabilities of the "
                                   f"sub-box n < {list(cut)} of one circuit per step, one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def config_block():
    return {"workload": f"{WORKLOAD}: {NCIRC} circuits, M=8 modes all PNR-detected, cutoff 6 "
                        "(6^8 probabilities each), b=0, forward + VJP of sum_n w_n Re p_n",
            "circuits_per_gpu": NCIRC, "modes": 8, "cutoff": 6,
            "l2": "walk state per step 5.6 GB > 129 MB L2 (no flush needed)"}


# ------------------------------------------------------------------- GPU
def measure_fp64_peak(torch):
    """FP64 roof: the larger of the library's FMA-chain probe and cuBLAS
    DGEMM (8192^3, best of 5), both measured live (TFLOP/s)."""
    from paper_2303_08879_gb300 import fockdiag as fd
    fma = fd.fk_measure_fp64_fma_rate()
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ a
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(); a @ a; e1.record(); torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a
    torch.cuda.empty_cache()
    return max(fma, best), {"fma_probe": fma, "dgemm": best}


def measured_bf16_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback (1.9 PFLOP/s, one earlier GB300 measurement)"


def _event_ms(torch, fn, reps, warmup=2):
    """Mean CUDA-event time of fn() on the current stream after warm-up."""
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


def _triples(fd, circs, dev):
    import torch
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = torch.from_numpy(np.stack([t[0] for t in trip])).to(dev)
    b = torch.from_numpy(np.stack([t[1] for t in trip])).to(dev)
    c = torch.from_numpy(np.array([t[2] for t in trip], np.complex128)).to(dev)
    return A, b, c


def small_circuit_row(torch, fd, inputs, dev, fp64_peak):
    """1 circuit, M = 2, C = 10, b = 0: latency of one forward and one
    forward + VJP call (launch-bound), and the same shape batched."""
    from paper_2303_08879_gb300 import counts
    out = {"workload": "gbs_m2_c10: M=2 both detected, C=10, b=0 (100 probabilities)"}
    for n in (1, 4096):
        circs = inputs.workload("gbs_m2_c10", n)
        cut = circs[0].cutoffs
        A, b, c = _triples(fd, circs, dev)
        flags = fd.FK_FLAG_B_ZERO
        p, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags)
        w = torch.ones_like(p)
        g = tuple(torch.empty_like(x) for x in (A, b, c))
        fwd = _event_ms(torch, lambda: fd.fock_diag_probs_batched(A, b, c, cut, probs=p, flags=flags, ws=ws), 20)
        both = _event_ms(torch, lambda: (fd.fock_diag_probs_batched(A, b, c, cut, probs=p, flags=flags, ws=ws),
                                         fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags, out=g)), 20)
        fd.check_workspace(ws, where="config-1 row")
        flops = n * 3 * counts.diag_flops(cut)        # forward + VJP (two MACs per term)
        stored = fd.fk_describe_diag_schedule(2, cut, flags)["stored"]
        key = "single_circuit" if n == 1 else f"batch_{n}"
        out[key] = {"circuits": n, "forward_ms": fwd, "forward_vjp_ms": both,
                    "probabilities_per_s": n * int(np.prod(cut)) / (both * 1e-3),
                    "circuits_per_s": n / (both * 1e-3),
                    "roofline": {"bound": "alu", "achieved": flops / (both * 1e-3) / 1e12,
                                 "peak": fp64_peak, "unit": "TFLOP/s",
                                 "frac": flops / (both * 1e-3) / 1e12 / fp64_peak,
                                 "algorithmic_flops": flops, "walk_amplitudes_per_circuit": stored}}
        del p, ws, w
    return out


def large_circuit_row(torch, fd, inputs, dev, fp64_peak, hbm):
    """1 circuit, M = 12, C = 5 (4.63 G walk amplitudes, 244 M probabilities),
    forward + VJP with the forward's amplitudes kept (no checkpointing), on
    the default engine (the tensor engine up to 12 kept modes), with the
    roofline of the roof that binds that engine."""
    from paper_2303_08879_gb300 import counts
    circs = inputs.workload("gbs_m12_c5")
    cut = circs[0].cutoffs
    A, b, c = _triples(fd, circs, dev)
    flags = fd.FK_FLAG_B_ZERO
    # the engine the default picks: its VJP workspace is the tensor engine's
    ws_default = fd.fk_workspace_size(len(cut), cut, 1, fd.FK_OP_DIAG_VJP, flags)
    ws_tensor = fd.fk_workspace_size(len(cut), cut, 1, fd.FK_OP_DIAG_VJP, flags | fd.FK_FLAG_ENGINE_TENSOR)
    engine = "tensor" if ws_default == ws_tensor else "fp64"
    p, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags)
    w = torch.randn(p.shape, dtype=torch.float64, device=dev,
                    generator=torch.Generator(device=dev).manual_seed(5)).to(torch.complex128)
    g = tuple(torch.empty_like(x) for x in (A, b, c))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags, out=g)
    torch.cuda.synchronize()
    ev[0].record()
    fd.fock_diag_probs_batched(A, b, c, cut, probs=p, flags=flags, ws=ws)
    ev[1].record()
    fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags, out=g)
    ev[2].record()
    torch.cuda.synchronize()
    fd.check_workspace(ws, where="config-5 row")
    fwd, vjp = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    stored = fd.fk_describe_diag_schedule(12, cut, flags)["stored"]
    nout = int(np.prod(cut))
    f_fwd = counts.diag_flops(cut)
    by_fwd, by_vjp = 32 * stored + 16 * nout, 48 * stored + 16 * nout
    wsb = ws.numel()
    del p, ws, w
    torch.cuda.empty_cache()
    return {"workload": "gbs_m12_c5: 1 circuit, M=12 all detected, C=5, b=0; VJP of sum_n w_n Re p_n",
            "engine": engine, "forward_ms": fwd, "vjp_ms": vjp,
            "probabilities_per_s": nout / ((fwd + vjp) * 1e-3), "walk_amplitudes": stored,
            "workspace_bytes": wsb,
            "roofline": _large_circuit_roofline(engine, f_fwd, fwd, vjp, by_fwd, by_vjp, fp64_peak, hbm)}


def _large_circuit_roofline(engine, f_fwd, fwd, vjp, by_fwd, by_vjp, fp64_peak, hbm):
    """The roof that binds the engine: HBM for the tensor engine (the digit
    products leave the FP64 pipe), the FP64 pipe for the FP64 engine; the
    other one beside it."""
    t = (fwd + vjp) * 1e-3
    fp64 = {"achieved": 3 * f_fwd / t / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": 3 * f_fwd / t / 1e12 / fp64_peak, "algorithmic_flops_forward": f_fwd,
            "forward_frac": f_fwd / (fwd * 1e-3) / 1e12 / fp64_peak,
            "vjp_frac": 2 * f_fwd / (vjp * 1e-3) / 1e12 / fp64_peak}
    mem = {"achieved": (by_fwd + by_vjp) / t / 1e9, "peak": hbm, "unit": "GB/s",
           "frac": (by_fwd + by_vjp) / t / 1e9 / hbm, "algorithmic_bytes": by_fwd + by_vjp}
    if engine == "tensor":
        return dict(bound="hbm", **mem, fp64_equivalent=fp64)
    return dict(bound="alu", **fp64, hbm=mem)


def fig10_row(torch, fd):
    """Fig. 10b: device time per circuit against a common cutoff at M = 4
    (64 circuits per launch), both product engines, and the fitted slopes."""
    from paper_2303_08879_gb300 import scaling
    cs = [4, 5, 6, 7, 8, 10, 12, 14, 16]
    out = {"modes": 4, "cutoffs": cs, "circuits_per_launch": 64}
    try:
        for engine, name in ((fd.FK_ENGINE_FP64, "fp64"), (fd.FK_ENGINE_TENSOR, "tensor")):
            fd.fk_diag_set_engine(engine)
            tt = scaling.time_table(4, cs)
            out[name] = {"forward_ms_per_circuit": [r["forward_ms_per_circuit"] for r in tt],
                         "vjp_ms_per_circuit": [r["vjp_ms_per_circuit"] for r in tt],
                         "slopes": {k: scaling.slope(cs, [r[k] for r in tt])
                                    for k in ("forward_ms_per_circuit", "vjp_ms_per_circuit",
                                              "workspace_bytes_per_circuit")}}
        out["workspace_bytes_per_circuit"] = [r["workspace_bytes_per_circuit"] for r in tt]
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    return out


def learned_row():
    """Learned proposals: dataset of 2^20 circuits from the batched conditional walk,
    BF16 MLP training, then 32 MLP-proposed starts against 32 random starts,
    each refined by the same exact-gradient steps (wall times measured)."""
    from paper_2303_08879_gb300 import proposal
    res = proposal.compare(n_train=1 << 20, log=lambda m: None)
    keep = ("wall_s", "start_s", "J_start_best", "J_start_median", "J_best", "F_best", "P_best", "reach")
    return {"workload": "M=3 heralded cat preparation: modes 0,1 detected at n*=(3,3) (walked at "
                        "cutoffs 4,4: the block is cutoff-independent), mode 2 undetected C=40; "
                        "15 circuit parameters; MLP 15-256-256-256-2 BF16",
            "train_circuits": 1 << 20, "dataset_s": res["timings"]["dataset_s"],
            "train_s": res["timings"]["train_s"], "train_loss": [res["losses"][0][1], res["losses"][-1][1]],
            "mlp_proposed": {k: res["mlp"][k] for k in keep},
            "plain_random_starts": {k: res["plain"][k] for k in keep}}


def secondary_rows(torch, fd, inputs, dev, fp64_peak, reps=5):
    """The other hot-path rows on their own workloads, CUDA-event timed after
    warm-up (reported beside the headline; not part of ``value``)."""
    from paper_2303_08879_gb300 import counts
    rows = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # Algorithm 2 forward + VJP: 64 conditional circuits, per-circuit cutoffs, b != 0
    mask = (1, 1, 0)
    circs = inputs.workload("cond_m3_batch64")
    cuts = [cc.cutoffs for cc in circs]
    A, b, c = _triples(fd, circs, dev)
    hbm, _ = measured_hbm_gbs()

    def time_cond(flags):
        rho, offs, ws = fd.fock_conditional_dm_batched(A, b, c, cuts, mask, flags=flags)
        g = torch.randn(rho.shape, dtype=torch.float64, device=dev).to(torch.complex128)
        out = tuple(torch.empty_like(x) for x in (A, b, c))
        for _ in range(3):
            fd.fock_conditional_dm_batched(A, b, c, cuts, mask, rho=rho, ws=ws, flags=flags)
            fd.fock_conditional_dm_vjp_batched(A, b, c, cuts, mask, g, ws, out=out, flags=flags)
        torch.cuda.synchronize()
        t0, t1, t2 = ev(), ev(), ev()
        fwd = vjp = 0.0
        for _ in range(reps):
            t0.record()
            fd.fock_conditional_dm_batched(A, b, c, cuts, mask, rho=rho, ws=ws, flags=flags)
            t1.record()
            fd.fock_conditional_dm_vjp_batched(A, b, c, cuts, mask, g, ws, out=out, flags=flags)
            t2.record()
            torch.cuda.synchronize()
            fwd += t0.elapsed_time(t1); vjp += t1.elapsed_time(t2)
        fd.check_workspace(ws, where="conditional rows")
        n_out = int(offs[-1])
        del rho, ws, g
        return fwd / reps, vjp / reps, n_out

    fwd, vjp, n_out = time_cond(fd.FK_FLAG_ENGINE_TENSOR)
    fwd64, vjp64, _ = time_cond(fd.FK_FLAG_ENGINE_FP64)
    f_fwd = sum(counts.cond_flops(cu, mask) for cu in cuts)
    n_amp = sum(counts.cond_amplitudes(cu, mask) for cu in cuts)
    # algorithmic bytes: 16 B written + 16 B read per walk amplitude and 16 B
    # per output (forward); the VJP reads the value and writes and reads the
    # adjoint (48 B) plus 16 B per upstream gradient
    b_fwd = 32 * n_amp + 16 * n_out
    b_vjp = 48 * n_amp + 16 * n_out
    rows["conditional_walk"] = {
        "workload": "cond_m3_batch64: 64 circuits, modes 0,1 detected (C 10..20), mode 2 "
                    "undetected (C 20..30), b != 0",
        "engine": "tensor", "forward_ms": fwd, "vjp_ms": vjp, "outputs": n_out,
        "walk_amplitudes": n_amp,
        "outputs_per_s": n_out / ((fwd + vjp) * 1e-3),
        "circuits_per_s": 64 / ((fwd + vjp) * 1e-3),
        # the slower of the two roofs (FP64 flops at the FP64 peak, bytes at
        # the HBM peak) binds here: the counted FP64 flops take 8x longer than
        # the bytes, and the tensor engine stays below the FP64 roof
        "roofline": {"bound": "alu", "achieved": f_fwd / (fwd * 1e-3) / 1e12, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": f_fwd / (fwd * 1e-3) / 1e12 / fp64_peak,
                     "kernel": "cond_forward_kernel", "algorithmic_flops_forward": f_fwd,
                     "vjp_frac": 2 * f_fwd / (vjp * 1e-3) / 1e12 / fp64_peak,
                     "note": "FP64-equivalent rate of the tensor engine (8 flops per counted complex "
                             "term); the VJP performs two complex MACs per term",
                     "hbm": {"peak_gbs": hbm,
                             "forward": {"achieved_gbs": b_fwd / (fwd * 1e-3) / 1e9,
                                         "frac": b_fwd / (fwd * 1e-3) / 1e9 / hbm,
                                         "algorithmic_bytes_per_launch": b_fwd},
                             "vjp": {"achieved_gbs": b_vjp / (vjp * 1e-3) / 1e9,
                                     "frac": b_vjp / (vjp * 1e-3) / 1e9 / hbm,
                                     "algorithmic_bytes_per_launch": b_vjp}}},
        "fp64_engine": {"forward_ms": fwd64, "vjp_ms": vjp64,
                        "forward_frac_of_fp64_peak": f_fwd / (fwd64 * 1e-3) / 1e12 / fp64_peak,
                        "vjp_frac_of_fp64_peak": 2 * f_fwd / (vjp64 * 1e-3) / 1e12 / fp64_peak}}
    # BF16 MLP training step (15-256-256-256-2, forward + backward + Adam): the
    # training batch (2048) and a large batch (65536) for the GEMM roofline
    from paper_2303_08879_gb300.mlp import MLP, init_params, IN, HIDDEN, OUT
    macs = IN * HIDDEN + 2 * HIDDEN * HIDDEN + HIDDEN * OUT
    peak, src = measured_bf16_tflops()
    res = {}
    for batch in (2048, 65536):
        mlp = MLP(init_params(0), batch, dev)
        gen = torch.Generator(device=dev); gen.manual_seed(0)
        X = torch.rand((batch, IN), device=dev, generator=gen) * 2 - 1
        Y = torch.rand((batch, OUT), device=dev, generator=gen)
        for _ in range(5):
            mlp.train_step(X, Y)
        torch.cuda.synchronize()
        steps = 20
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(steps):
            mlp.train_step(X, Y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        tf = 3 * 2 * batch * macs / (ms * 1e-3) / 1e12   # forward + two backward GEMMs per layer
        res[batch] = (ms, tf)
        del mlp
    ms, tf = res[65536]
    rows["mlp_train_step"] = {
        "workload": "BF16 MLP 15-256-256-256-2, forward + backward + Adam",
        "train_batch_2048_ms": res[2048][0], "batch_65536_ms": ms,
        "samples_per_s": 65536 / (ms * 1e-3),
        "roofline": {"bound": "tensor", "batch": 65536, "achieved": tf, "peak": peak,
                     "unit": "TFLOP/s", "frac": tf / peak, "peak_source": src}}
    torch.cuda.empty_cache()
    rows["m2_c10_latency"] = small_circuit_row(torch, fd, inputs, dev, fp64_peak)
    torch.cuda.empty_cache()
    rows["m12_c5_large"] = large_circuit_row(torch, fd, inputs, dev, fp64_peak, hbm)
    rows["fig10b_time_vs_cutoff"] = fig10_row(torch, fd)
    torch.cuda.empty_cache()
    rows["learned_proposal"] = learned_row()
    torch.cuda.empty_cache()
    return rows


# ------------------------------------------------------------- multi-rank
def rank_circuits(rank, n):
    """The n circuits of rank `rank`: consecutive, disjoint slices of the
    workload, so the work per GPU is fixed as ranks are added (weak scaling)."""
    from paper_2303_08879_gb300 import inputs
    return inputs.workload(WORKLOAD, n, start=rank * n)


def max_over_ranks(x, device):
    """The largest of a per-rank time over all ranks (x itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, n_per_rank, units_per_circuit, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time per step."""
    return world * n_per_rank * units_per_circuit / (ms * 1e-3)


def run_gpu(args):
    if not args.no_cpu_baseline and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        import oracle                  # compile the oracle before any CUDA work
        oracle.build()
    import torch
    import torch.distributed as dist
    from paper_2303_08879_gb300 import fockdiag as fd
    from paper_2303_08879_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    circs = rank_circuits(rank, NCIRC)
    cut = circs[0].cutoffs
    M = len(cut)
    trip = [fd.fk_gaussian_to_triple(c.V, c.mean) for c in circs]
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    A_h = pin(np.stack([t[0] for t in trip]))
    b_h = pin(np.stack([t[1] for t in trip]))
    c_h = pin(np.array([t[2] for t in trip], np.complex128))
    rng = np.random.default_rng(1000 + rank)
    w_h = pin(rng.normal(size=(NCIRC,) + cut).astype(np.complex128))
    dev = torch.device("cuda", local)
    A, b, c, w = (x.to(dev) for x in (A_h, b_h, c_h, w_h))
    flags = fd.FK_FLAG_B_ZERO
    probs = torch.empty((NCIRC,) + cut, dtype=torch.complex128, device=dev)
    gA, gb, gc = torch.empty_like(A), torch.empty_like(b), torch.empty_like(c)
    from paper_2303_08879_gb300 import autotune
    best, times = (autotune.TENSOR, 128, 4, 0), None
    if args.tuning:
        parts = args.tuning.split("/")
        if len(parts) == 3:
            parts = [autotune.FP64] + parts
        best = (parts[0],) + tuple(int(v) for v in parts[1:])
    elif not args.no_autotune:
        best, times = autotune.tune_diag(A, b, c, cut, w, flags=flags)
    autotune.apply(best)
    tuning = {"engine": best[0], "tile_pivots": best[1], "chunk_rows": best[2],
              "blocks_per_sm_cap": best[3], "ms_per_candidate": times}
    ws = fd.workspace(fd.fk_workspace_size(M, cut, NCIRC, fd.FK_OP_DIAG_VJP, flags), dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    split = best[0] == autotune.TENSOR   # the VJP is two launches: reverse walk, partial pass

    def step(tk=None):
        if tk is not None:
            tk[0].record(stream)
        fd.fock_diag_probs_batched(A, b, c, cut, probs=probs, flags=flags, ws=ws)
        if tk is not None:
            tk[1].record(stream)
            if split:
                fd.fk_diag_set_vjp_split_event(tk[3])   # recorded between the two launches
        fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags, out=(gA, gb, gc))
        if tk is not None:
            tk[2].record(stream)

    for _ in range(args.warmup):
        step()
    fd.check_workspace(ws, where="warm-up")
    barrier(); torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    marks = [[ev(), ev(), ev(), ev()] for _ in range(args.steps)]
    for m in marks:
        m[3].record(stream)   # creates the event the library records between the VJP launches
    t0, t1 = ev(), ev()
    t0.record(stream)
    for i in range(args.steps):
        step(marks[i])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    fd.check_workspace(ws, where="timed steps")
    ms = t0.elapsed_time(t1) / args.steps
    fd.fk_diag_set_vjp_split_event(None)
    fwd_ms = statistics.mean(m[0].elapsed_time(m[1]) for m in marks)
    vjp_ms = statistics.mean(m[1].elapsed_time(m[2]) for m in marks)
    if split:
        walk_ms = statistics.mean(m[1].elapsed_time(m[3]) for m in marks)
        part_ms = statistics.mean(m[3].elapsed_time(m[2]) for m in marks)
        kernel_ms = {"diag_forward_kernel": fwd_ms, "diag_vjp_kernel": walk_ms,
                     "diag_vjp_partials_kernel": part_ms}
    else:
        kernel_ms = {"diag_forward_kernel": fwd_ms, "diag_vjp_kernel": vjp_ms}
    ms = max_over_ranks(ms, dev)

    # the plain single-circuit method: the same circuits as NCIRC batch-1 forward + VJP
    # calls (same engine and accuracy), each with a one-circuit workspace
    ws1 = fd.workspace(fd.fk_workspace_size(M, cut, 1, fd.FK_OP_DIAG_VJP, flags), dev)

    def plain_step():
        for i in range(NCIRC):
            sl = slice(i, i + 1)
            fd.fock_diag_probs_batched(A[sl], b[sl], c[sl], cut, probs=probs[sl], flags=flags, ws=ws1)
            fd.fock_diag_probs_vjp_batched(A[sl], b[sl], c[sl], cut, w[sl], ws1, flags=flags,
                                           out=(gA[sl], gb[sl], gc[sl]))

    plain_step(); torch.cuda.synchronize()
    fd.check_workspace(ws1, where="plain single-circuit steps")
    barrier()
    q0, q1 = ev(), ev()
    q0.record(stream)
    for _ in range(args.steps):
        plain_step()
    q1.record(stream)
    torch.cuda.synchronize()
    plain_ms = max_over_ranks(q0.elapsed_time(q1) / args.steps, dev)
    fd.check_workspace(ws1, where="plain single-circuit steps")
    del ws1

    # end to end through the public API, pinned host buffers in and out.  Two
    # device buffer sets: a copy stream brings step i+1's inputs in (and step
    # i's gradients out) while step i computes; every step's copies are inside
    # the timed region.
    gA_h, gb_h, gc_h = (torch.empty_like(x, device="cpu").pin_memory() for x in (A_h, b_h, c_h))
    host_in = (A_h, b_h, c_h, w_h)
    bufs = [(A, b, c, w), tuple(torch.empty_like(x) for x in (A, b, c, w))]
    outs = [(gA, gb, gc), tuple(torch.empty_like(x) for x in (gA, gb, gc))]
    cstream = torch.cuda.Stream(dev)
    mk = lambda: torch.cuda.Event()

    def e2e_run(nsteps, u0=None, u1=None):
        ready = [mk() for _ in range(nsteps)]
        done = [mk() for _ in range(nsteps)]
        fetched = [mk() for _ in range(nsteps)]

        def h2d(i):
            with torch.cuda.stream(cstream):
                if i >= 2:
                    cstream.wait_event(done[i - 2])        # buffer i % 2 is free again
                for dst, src in zip(bufs[i % 2], host_in):
                    dst.copy_(src, non_blocking=True)
                ready[i].record(cstream)

        if u0 is not None:
            u0.record(stream)
            cstream.wait_event(u0)
        h2d(0)
        for i in range(nsteps):
            if i + 1 < nsteps:
                h2d(i + 1)
            Ab, bb, cb, wb = bufs[i % 2]
            stream.wait_event(ready[i])
            if i >= 2:
                stream.wait_event(fetched[i - 2])        # gradients of step i-2 are on the host
            fd.fock_diag_probs_batched(Ab, bb, cb, cut, probs=probs, flags=flags, ws=ws)
            fd.fock_diag_probs_vjp_batched(Ab, bb, cb, cut, wb, ws, flags=flags, out=outs[i % 2])
            done[i].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(done[i])
                for dst, src in zip((gA_h, gb_h, gc_h), outs[i % 2]):
                    dst.copy_(src, non_blocking=True)
                fetched[i].record(cstream)
        stream.wait_event(fetched[nsteps - 1])
        if u1 is not None:
            u1.record(stream)

    e2e_run(2); torch.cuda.synchronize()
    barrier()
    u0, u1 = ev(), ev()
    e2e_run(args.steps, u0, u1)
    torch.cuda.synchronize()
    e2e_ms = u0.elapsed_time(u1) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, dev)
    fd.check_workspace(ws, where="e2e steps")
    # the last step's gradients on the host equal the device-resident run's
    assert torch.equal(gA_h, outs[(args.steps - 1) % 2][0].cpu())

    h2d = sum(x.numel() * x.element_size() for x in (A_h, b_h, c_h, w_h))
    d2h = sum(x.numel() * x.element_size() for x in (gA_h, gb_h, gc_h))
    out = None
    if rank == 0:
        flops_fwd = NCIRC * algorithmic_flops(cut)
        flops_vjp = 2 * flops_fwd
        peak, peaks = measure_fp64_peak(torch)
        fp64_eq = flops_vjp / (vjp_ms * 1e-3) / 1e12
        sha = kernel_sha()
        shape = list(best)
        traffic = (TRAFFIC["bytes_per_launch"]
                   if TRAFFIC["kernel_sha"] == sha and TRAFFIC["tuning"] == shape else {})
        stored = fd.fk_describe_diag_schedule(M, cut, flags)["stored"]
        nout = int(np.prod(cut))
        bytes_fwd = NCIRC * (32 * stored + 16 * nout)
        bytes_vjp = NCIRC * (48 * stored + 16 * nout)
        if best[0] == autotune.TENSOR:
            hbm, hbm_src = measured_hbm_gbs()
            # algorithmic bytes per launch: forward 32 B per walk amplitude (value read and
            # written) + 16 B per output; reverse walk 32 B per walk amplitude (adjoint read
            # and written) + 16 B per upstream gradient; partial pass 32 B per walk amplitude
            # (value and adjoint read)
            alg = {"diag_forward_kernel": bytes_fwd,
                   "diag_vjp_kernel": NCIRC * (32 * stored + 16 * nout),
                   "diag_vjp_partials_kernel": NCIRC * 32 * stored}
            per = {k: {"ms": kernel_ms[k], "achieved": alg[k] / (kernel_ms[k] * 1e-3) / 1e9,
                       "frac": alg[k] / (kernel_ms[k] * 1e-3) / 1e9 / hbm,
                       "algorithmic_bytes_per_launch": alg[k], "traffic": traffic.get(k)}
                   for k in kernel_ms}
            top = max(kernel_ms, key=kernel_ms.get)   # the dominant kernel
            roof = {"bound": "hbm", "kernel": top, "achieved": per[top]["achieved"], "peak": hbm,
                    "unit": "GB/s", "frac": per[top]["frac"], "traffic": per[top]["traffic"],
                    "algorithmic_bytes_per_launch": alg[top],
                    "peak_source": hbm_src,
                    "kernels": per,
                    "forward": {"achieved": bytes_fwd / (fwd_ms * 1e-3) / 1e9,
                                "frac": bytes_fwd / (fwd_ms * 1e-3) / 1e9 / hbm,
                                "algorithmic_bytes_per_launch": bytes_fwd},
                    "fp64_equivalent": {"achieved_tflops": fp64_eq, "fp64_peak_tflops": peak,
                                        "ratio": fp64_eq / peak, "peaks_measured": peaks,
                                        "forward_tflops": flops_fwd / (fwd_ms * 1e-3) / 1e12}}
        else:
            roof = {"bound": "alu", "kernel": "diag_vjp_kernel", "achieved": fp64_eq,
                    "peak": peak, "unit": "TFLOP/s", "frac": fp64_eq / peak,
                    "traffic": traffic.get("diag_vjp_kernel"),
                    "peak_source": "measured live: max of FP64 FMA-chain probe and cuBLAS DGEMM",
                    "peaks_measured": peaks, "peak_nominal": 1.25,
                    "forward": {"achieved": flops_fwd / (fwd_ms * 1e-3) / 1e12,
                                "frac": flops_fwd / (fwd_ms * 1e-3) / 1e12 / peak}}
        out = {
            "metric": METRIC, "value": job_rate(world, NCIRC, int(np.prod(cut)), ms), "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": config_block(),
            "circuits_per_s": world * NCIRC / (ms * 1e-3),
            # batched forward + VJP against the same circuits as single-circuit calls
            "vs_plain": plain_ms / ms,
            "plain_single_circuit": {
                "ms_per_step": plain_ms, "circuits_per_s": world * NCIRC / (plain_ms * 1e-3),
                "value": job_rate(world, NCIRC, int(np.prod(cut)), plain_ms), "unit": UNIT,
                "method": f"{NCIRC} batch-1 forward + VJP calls per step, same engine and tuning"},
            "kernel_ms": kernel_ms, "vjp_ms": vjp_ms,
            "e2e": {"value": job_rate(world, NCIRC, int(np.prod(cut)), e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            # forward: one launch; VJP: the reverse walk plus (tensor engine) the partial pass
            "gpu_launches": (3 if tuning["engine"] == "tensor" else 2) * args.steps,
            "roofline": roof,
            "clocks": clocks,
            "autotune": tuning,
        }
        if world == 1 and not args.no_rows:
            del ws
            torch.cuda.empty_cache()
            out["rows"] = secondary_rows(torch, fd, inputs, dev, peak)
        if world == 1 and not args.no_cpu_baseline:
            host = host_cpu()
            n, dt, scut = oracle_sample(15.0)
            n_all, wall, _ = oracle_all_cores(10.0, host["nproc"])
            out["cpu_baseline"] = {
                "value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host,
                "sample": f"naive Algorithm 1 walk (forward only) of one circuit, probabilities "
                          f"of the sub-box n < {list(scut)}, one thread, {dt:.1f} s",
                "all_cores": {"value": n_all / wall, "unit": UNIT, "cores": host["nproc"],
                              "sample": f"{host['nproc']} processes at once, one circuit each, "
                                        f"the same kind of sub-box sized to ~10 s per process, "
                                        f"{wall:.1f} s wall"},
                "note": "forward only: the oracle's gradients are the closed form on the full "
                        "density-matrix lattice (6^16 entries at this size) or forward-mode "
                        "tangents, one direction per walk (272 directions)"}
    if world > 1:
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


def main():
    global NCIRC
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the secondary rows (conditional walk, MLP step)")
    ap.add_argument("--tuning", default=None,
                    help="fixed engine and tile shape 'tensor|fp64/pivots/rows/cap' instead of "
                         "the autotuner ('pivots/rows/cap' = fp64)")
    ap.add_argument("--circuits", type=int, default=NCIRC,
                    help="circuits per GPU (default 16; smaller only for profiler captures)")
    args = ap.parse_args()
    NCIRC = args.circuits
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
