"""The debug-checks build (a stand-in for a memory checker, which this pool
does not offer): libfockdiag_debug.so, compiled with -DFK_DEBUG_CHECKS,
checks the index of every amplitude, adjoint, scratch, output and
pivot-geometry access of the all-detected walk against the storage box of
its App. B.2 type (the conditional walk's against its circuit's arrays) and
records per-level device timestamps.  The walks of
tests/debug_checks_cases.py run on it in a process of their own; no access
may leave its box, the results must still match the oracle, and the trace
must show one timestamp per level barrier in walk order.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def report():
    from paper_2303_08879_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, FOCKDIAG_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_checks_cases.py")],
                       capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_is_loaded(report):
    assert report["debug_build"] is True


def test_no_access_leaves_its_storage_box(report):
    assert len(report["cases"]) == 18
    for case in report["cases"]:
        assert case["status"] == 0, case
        assert case["forward"]["violations"] == 0, case
        assert case["vjp"]["violations"] == 0, case
        if "finite" in case:
            assert case["finite"], case


def test_checked_walks_match_the_oracle(report):
    one_shape = [c for c in report["cases"] if "one shape" in c["what"]]
    assert len(one_shape) == 8
    for c in one_shape:
        assert c["probs_err"][0] <= 1e-10 and c["probs_err"][1] <= 1.0, c
        assert c["gradA_err"][0] <= 1e-8 and c["gradA_err"][1] <= 1.0, c
        assert c["gradb_err"][0] <= 1e-8 and c["gradb_err"][1] <= 1.0, c
    cond = [c for c in report["cases"] if c["what"].startswith("conditional")]
    assert len(cond) == 4
    for c in cond:
        assert c["probs_err"][0] <= 1e-10 and c["probs_err"][1] <= 1.0, c


def test_level_timestamps(report):
    """One record per grid barrier: the forward's levels ascending, the
    reverse walk's descending, then the final reduction; times never go
    back."""
    tr = report["trace"]
    L = tr["levels"]
    assert tr["count"] == 2 * L + 1
    fwd = [((t >> 24), (t >> 8) & 0xffff, t & 1) for t in tr["tags"]]
    assert fwd[:L] == [(1, lev, 0) for lev in range(L)]
    assert fwd[L:2 * L] == [(2, lev, 0) for lev in range(L - 1, -1, -1)]
    assert fwd[2 * L] == (3, 0, 0)
    ns = tr["ns"]
    assert all(b >= a for a, b in zip(ns, ns[1:]))
    assert ns[-1] > ns[0]
