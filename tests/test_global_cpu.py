"""Global photon-number cutoff (Sec. 2.3 eq. global_boundary_conditions applied
to Algorithm 1): host-side geometry, no GPU.

Pins: output count binomial(n_max - 1 + M, M) (stars and bars); the packed
output order (total photon number, then lexicographic); the pivot count of
App. B.1 evaluated from its printed per-N terms.
"""
import itertools
from math import comb

import pytest

from paper_2303_08879_gb300 import fockdiag as fd


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08879_gb300 import build
    build.build()


@pytest.mark.parametrize("M,n", [(1, 1), (1, 7), (2, 5), (3, 4), (4, 6), (6, 3), (8, 6), (12, 4)])
def test_output_count_is_binomial(M, n):
    assert fd.fk_global_size(M, n) == comb(n - 1 + M, M)


@pytest.mark.parametrize("M,n", [(1, 5), (2, 6), (3, 5), (4, 4)])
def test_pattern_index_is_level_major_bijection(M, n):
    pats = [p for p in itertools.product(range(n), repeat=M) if sum(p) < n]
    order = sorted(pats, key=lambda p: (sum(p), p))
    idx = [fd.fk_global_pattern_index(M, n, p) for p in order]
    assert idx == list(range(len(pats)))
    assert fd.fk_global_pattern_index(M, n, (n,) + (0,) * (M - 1)) == -1
    assert fd.fk_global_pattern_index(M, n, (-1,) + (0,) * (M - 1)) == -1


def paper_pivots(M, N_max, with_b):
    """App. B.1: sum over N < N_max of binom(N+M-1, M-1) diagonal pivots (b != 0
    only) plus sum_{K=1..M} binom(N+M-K, M-K) off-diagonal pivots."""
    tot = 0
    for N in range(N_max):
        if with_b:
            tot += comb(N + M - 1, M - 1)
        tot += sum(comb(N + M - K, M - K) for K in range(1, M + 1))
    return tot


@pytest.mark.parametrize("M,n", [(1, 4), (2, 6), (3, 5), (4, 6), (5, 3), (8, 6)])
def test_pivot_count_matches_appendix(M, n):
    # the walk applies the pivots of total photon number N <= n - 2: their
    # diagonal writes complete every pattern with fewer than n photons
    d = fd.fk_describe_global_schedule(M, n, 0)
    assert d["pivots"] == paper_pivots(M, n - 1, True)
    d0 = fd.fk_describe_global_schedule(M, n, fd.FK_FLAG_B_ZERO)
    assert d0["pivots"] == paper_pivots(M, n - 1, False)
    # the per-N sum in closed form (hockey stick): binom(Nm+M-1, M) + binom(Nm+M, M) - 1
    Nm = n - 1
    assert d["pivots"] == comb(Nm + M - 1, M) + comb(Nm + M, M) - 1
    assert d["outputs"] == comb(n - 1 + M, M)


def test_storage_grows_binomially():
    # M = 8, n_max = 6: a few times binomial(13, 8) = 1287 amplitudes, far below 6^8
    d = fd.fk_describe_global_schedule(8, 6, fd.FK_FLAG_B_ZERO)
    assert d["outputs"] == 1287
    assert d["allocated"] < 40 * 1287 < 6 ** 8


def test_global_arguments_rejected():
    with pytest.raises(fd.FockError):
        fd.fk_global_size(0, 3)
    with pytest.raises(fd.FockError):
        fd.fk_global_size(3, 0)
    with pytest.raises(fd.FockError):
        fd.fk_global_size(3, 65)
