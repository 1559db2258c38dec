"""The roofline work counts (paper_2303_08879_gb300/counts.py) against direct
enumeration: the closed-form sums over pivots must equal a plain loop over
every pivot of the walk, and the number of amplitudes they say are written
must equal the library's storage schedule (fk_describe_diag_schedule)."""
import itertools

import numpy as np
import pytest

from paper_2303_08879_gb300 import build as pbuild
from paper_2303_08879_gb300 import counts


@pytest.fixture(scope="module")
def fd():
    pbuild.build()
    from paper_2303_08879_gb300 import fockdiag
    fockdiag.lib()
    return fockdiag


def brute_terms_writes(cutoffs, has_b):
    C = [c for c in cutoffs if c >= 2]
    M = len(C)
    terms = writes = 0
    for K in range(M):
        for e in itertools.product(*([range(C[K] - 1)] + [range(c) for c in C[K + 1:]])):
            P = [0] * (2 * M)                      # pivot e + 1_{2K} as a lattice vector
            for i, m in enumerate(range(K, M)):
                P[2 * m] = P[2 * m + 1] = e[i]
            P[2 * K] += 1
            t = sum(1 for v in P if v >= 1) + (1 if has_b else 0)
            w = 1 + (e[0] <= C[K] - 3) + 2 * sum(1 for i, m in enumerate(range(K + 1, M), 1) if e[i] <= C[m] - 2)
            terms += t * w
            writes += w
    if has_b and M:
        for d in itertools.product(*([range(C[0] - 1)] + [range(c) for c in C[1:]])):
            t = 1 + 2 * sum(1 for v in d if v >= 1)
            w = 1 + (d[0] <= C[0] - 3) + 2 * sum(1 for q in range(1, M) if d[q] <= C[q] - 2)
            terms += t * w
            writes += w
    return terms, writes


@pytest.mark.parametrize("cut", [(4,), (3, 5), (6, 6, 6), (2, 3, 4, 2), (5, 1, 4), (3, 3, 3, 3, 3)])
@pytest.mark.parametrize("has_b", [False, True])
def test_closed_form_matches_enumeration(cut, has_b):
    assert counts.diag_terms_writes(cut, has_b) == brute_terms_writes(cut, has_b)


@pytest.mark.parametrize("cut", [(4,), (3, 5), (6, 6, 6), (2, 3, 4, 2), (6,) * 8, (5,) * 12])
@pytest.mark.parametrize("has_b", [False, True])
def test_writes_match_library_schedule(fd, cut, has_b):
    stored = fd.fk_describe_diag_schedule(len(cut), cut, 0 if has_b else fd.FK_FLAG_B_ZERO)["stored"]
    assert counts.diag_terms_writes(cut, has_b)[1] == stored - 1


def test_cond_terms_small_case_by_enumeration():
    """Two detected modes and one undetected mode: step 2 adds, for every
    detected amplitude and every u, the detected pivot's terms (b included)
    and one term per nonzero undetected index; step 1 walks u alone."""
    cut, det = (3, 2, 3), (1, 1, 0)
    dt, dw = brute_terms_writes((3, 2), True)
    CU = 3
    step1 = 0
    for k in range(CU):
        for l in range(CU):
            if k == 0 and l == 0:
                continue
            P = [k - 1, l] if k > 0 else [0, l - 1]
            step1 += 1 + sum(1 for v in P if v >= 1)
    nzsum = sum((k >= 1) + (l >= 1) for k in range(CU) for l in range(CU))
    assert counts.cond_terms(cut, det) == step1 + CU * CU * dt + dw * nzsum


def test_cond_amplitudes_small_case_by_enumeration():
    """Stored amplitudes of the conditional walk: every u of the u-block at
    the vacuum position and at every detected amplitude the walk writes."""
    cut, det = (3, 2, 3), (1, 1, 0)
    _, dw = brute_terms_writes((3, 2), True)
    assert counts.cond_amplitudes(cut, det) == 9 * (1 + dw)
    assert counts.cond_amplitudes((4, 3, 2, 5), (1, 0, 1, 0)) == \
        (3 * 3 * 5 * 5) * (1 + brute_terms_writes((4, 2), True)[1])

