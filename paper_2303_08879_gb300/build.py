"""Build libfockdiag.so (the C-ABI library) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2303_08879_gb300/libfockdiag.so``.  Objects go to ``_build/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfockdiag.so")
# the debug-checks variant (-DFK_DEBUG_CHECKS: storage-box checks of every
# walk access and per-level timestamps), built on request only
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libfockdiag_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cpp", "circuit.cpp", "walk_diag.cu", "walk_cond.cu", "mlp.cu", "herald.cu", "probe.cu", "static_ws.cu",
           "walk_pure.cu", "multi.cpp", "walk_diag_tc1.cu", "walk_diag_tc2.cu", "walk_diag_tc3.cu", "mlp_tc.cu",
           "walk_cond_k0.cu", "walk_cond_k1.cu", "walk_cond_k2.cu", "walk_cond_k3.cu"]
# walk_diag_fp64.cu once per FP64 tile shape (pivots per tile, rows per chunk)
FP64_SHAPES = [(128, 8), (128, 4), (64, 8), (64, 4), (256, 8)]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfockdiag")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + list(extra)


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Compile the library (``debug``: the debug-checks variant) and return its path."""
    build_dir, lib_path = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    if debug:
        extra_flags = list(extra_flags) + ["-DFK_DEBUG_CHECKS"]
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))]
    cc = nvcc()
    jobs = []
    objs = []
    units = [(src, src + ".o", []) for src in SOURCES]
    units += [("walk_diag_fp64.cu", f"walk_diag_fp64_{t}_{c}.o", [f"-DFK_TPB={t}", f"-DFK_CH={c}"])
              for t, c in FP64_SHAPES]
    for src, oname, defs in units:
        path = os.path.join(CSRC, src)
        obj = os.path.join(build_dir, oname)
        objs.append(obj)
        if _stale(obj, [path, __file__] + headers):
            cmd = [cc] + _flags(extra_flags) + defs + ["-c", path, "-o", obj]
            if src.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    # the heaviest units first, so the parallel build ends soon after them
    jobs.sort(key=lambda c: 0 if ("walk_diag" in c[-3] or "walk_cond_k" in c[-3]) else 1)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    if jobs or not os.path.exists(lib_path) or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError(f"link of {os.path.basename(lib_path)} failed")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
