"""Host-side checks of the C-ABI library (no GPU needed).

* the library builds, loads, and exports every function include/fockdiag.h
  declares;
* the storage geometry (fk_describe_diag_schedule) matches, level by level
  and type by type, the amplitudes and pivots the oracle's naive walk of
  Algorithm 1 touches (App. B.2: the structure is dense, each amplitude is
  written once);
* the host Gaussian -> (A, b, c) map agrees with the oracle's;
* argument errors are reported before any device work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from oracle import triple as otriple
from paper_2303_08879_gb300 import build as pbuild
from paper_2303_08879_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))]


@pytest.fixture(scope="module")
def fd():
    pbuild.build()
    from paper_2303_08879_gb300 import fockdiag
    fockdiag.lib()
    return fockdiag


def declared_functions():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_library_exports_every_declared_symbol(fd):
    names = declared_functions()
    assert len(names) >= 10
    lib = ctypes.CDLL(fd.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(fd.EXPORTS)


def test_status_strings(fd):
    L = fd.lib()
    assert L.fk_status_string(0) == b"ok"
    assert b"timed out" in L.fk_status_string(6)
    assert L.fk_version() >= 100


def test_gaussian_to_triple_matches_oracle(fd):
    for name, n in (("gbs_m2_c10", 1), ("cond_m3_batch64", 3), ("gbs_m8_c6_batch16", 2)):
        for circ in inputs.workload(name, n):
            A1, b1, c1 = fd.fk_gaussian_to_triple(circ.V, circ.mean)
            A2, b2, c2 = otriple.gaussian_to_triple(circ.V, circ.mean)
            assert np.max(np.abs(A1 - A2)) < 1e-13
            assert np.max(np.abs(b1 - b2)) < 1e-13
            assert abs(c1 - c2) < 1e-14 * abs(c2)


SCHED_CASES = [((5, 4), True), ((3, 4, 3), True), ((4, 4, 4), False), ((2, 5, 1), True),
               ((1, 3), False), ((6,), True), ((3, 3, 2, 3), False), ((2, 2, 2, 2), True),
               ((1, 1), True), ((7, 2, 5), True), ((2, 6, 3, 4), False), ((4, 1, 3, 2), True),
               ((3, 3, 3, 3, 3), True)]


@pytest.mark.parametrize("cut,withb", SCHED_CASES)
def test_schedule_matches_oracle_walk(fd, cut, withb):
    rng = np.random.default_rng(sum(cut) + 31 * len(cut))
    D = 2 * len(cut)
    A, b = inputs.random_symmetric(D, rng, with_b=withb)
    w = oracle.Walk(A, b, 0.5, cut)
    w.all_probs()
    flags = 0 if withb else fd.FK_FLAG_B_ZERO
    desc = fd.fk_describe_diag_schedule(len(cut), cut, flags)
    st = w.stats()
    assert desc["stored"] == st["stored"]
    assert desc["pivots"] == st["pivots"]
    lev = desc["levels"]
    h = w.level_hist(lev + 1)
    ours = desc["per_level"]
    # columns: diag, offset_1 (ket + bra), offset_2, 1010, 1001
    np.testing.assert_array_equal(ours[:, 0], h[:lev, 0])
    np.testing.assert_array_equal(ours[:, 1], h[:lev, 1] + h[:lev, 2])
    np.testing.assert_array_equal(ours[:, 2:5], h[:lev, 3:6])
    assert h[lev:].sum() == 0


def test_argument_errors_are_reported(fd):
    L = fd.lib()
    n = ctypes.c_size_t(0)
    cut = (ctypes.c_int * 2)(3, 0)
    assert L.fk_workspace_size(2, cut, None, 1, fd.FK_OP_DIAG, 0, ctypes.byref(n)) == 1
    cut13 = (ctypes.c_int * 13)(*([2] * 13))
    assert L.fk_workspace_size(13, cut13, None, 1, fd.FK_OP_DIAG, 0, ctypes.byref(n)) == 2
    big = (ctypes.c_int * 1)(65)
    assert L.fk_workspace_size(1, big, None, 1, fd.FK_OP_DIAG, 0, ctypes.byref(n)) == 2
    ok = (ctypes.c_int * 2)(3, 3)
    assert L.fk_workspace_size(2, ok, None, 1, fd.FK_OP_DIAG, 0, ctypes.byref(n)) == 0
    assert n.value > 0
    # null device pointers are rejected before any CUDA call
    assert L.fock_diag_probs_batched(1, None, None, None, 2, ok, None, 0, None, 0, None) == 1
    assert L.fk_selftest_wait_timeout(None, 0, 1000, None) == 3


def test_workspace_size_monotone_in_batch_and_b(fd):
    s1 = fd.fk_workspace_size(3, (4, 5, 3), 1, fd.FK_OP_DIAG, 0)
    s2 = fd.fk_workspace_size(3, (4, 5, 3), 4, fd.FK_OP_DIAG, 0)
    s0 = fd.fk_workspace_size(3, (4, 5, 3), 1, fd.FK_OP_DIAG, fd.FK_FLAG_B_ZERO)
    assert s2 > s1 > s0


def test_pure_triple_matches_oracle(fd):
    """fk_gaussian_to_pure_triple (host C++) against the oracle's pure triple;
    mixed states are refused."""
    from oracle import triple as otriple
    from paper_2303_08879_gb300 import inputs
    rng = np.random.default_rng(12)
    for M in (1, 2, 4):
        circ = inputs.make_circuit(M, rng, r_range=(0.1, 1.0), eta_range=(1.0, 1.0), alpha_var=0.5,
                                   cutoffs=(2,) * M)
        A, b, c = fd.fk_gaussian_to_pure_triple(circ.V, circ.mean)
        Ao, bo, co = otriple.pure_triple(circ.V, circ.mean)
        assert np.max(np.abs(A - Ao)) < 1e-13 and np.max(np.abs(b - bo)) < 1e-13 and abs(c - co) < 1e-14
    lossy = inputs.make_circuit(2, rng, r_range=(0.4, 0.5), eta_range=(0.5, 0.6), cutoffs=(2, 2))
    with pytest.raises(fd.FockError):
        fd.fk_gaussian_to_pure_triple(lossy.V, lossy.mean)


def test_per_call_tuning_flags(fd):
    """Engine and tile bits for one call: encoded by fk_diag_tuning_flags,
    validated on the host (uncompiled shapes, caps outside 0..32, both engine
    bits at once) before any device work."""
    assert fd.fk_diag_tuning_flags(fd.FK_ENGINE_AUTO) == 0
    assert fd.fk_diag_tuning_flags(fd.FK_ENGINE_FP64) == fd.FK_FLAG_ENGINE_FP64
    assert fd.fk_diag_tuning_flags(fd.FK_ENGINE_TENSOR) == fd.FK_FLAG_ENGINE_TENSOR
    f = fd.fk_diag_tuning_flags(fd.FK_ENGINE_FP64, 64, 4, 3)
    assert f & fd.FK_FLAG_ENGINE_FP64 and (f >> 8) & 15 == 4 and (f >> 12) & 63 == 3
    for bad in ((3, 0, 0, 0), (0, 96, 8, 0), (0, 128, 8, 33), (0, 0, 0, 2), (0, 128, 2, 0)):
        with pytest.raises(fd.FockError):
            fd.fk_diag_tuning_flags(*bad)
    L = fd.lib()
    need = ctypes.c_size_t(0)
    cut = (ctypes.c_int * 2)(3, 3)
    both = fd.FK_FLAG_ENGINE_FP64 | fd.FK_FLAG_ENGINE_TENSOR
    for flags in (both, 9 << 8, (1 << 8) | (40 << 12)):
        assert L.fk_workspace_size(2, cut, None, 1, fd.FK_OP_DIAG, flags, ctypes.byref(need)) == 1
    # the tile bits select the FP64 shape only; the forward layout does not depend on them
    ok = [L.fk_workspace_size(2, cut, None, 1, fd.FK_OP_DIAG, fl, ctypes.byref(need)) for fl in
          (0, fd.fk_diag_tuning_flags(fd.FK_ENGINE_FP64, 256, 8, 0), fd.FK_FLAG_CHECK_FINITE)]
    assert ok == [0, 0, 0]
