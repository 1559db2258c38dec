"""Counters of Fig. 8 / Fig. 10 (paper_2303_08879_gb300/scaling.py), pinned to
the paper's statements and App. B formulas; CPU only."""
import pytest

from paper_2303_08879_gb300 import scaling


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08879_gb300 import build
    build.build()


def appb_written_b0(M, C):
    """App. B.2 counts for b = 0: C^M diagonal, (C-2) sum_K C^(M-K-1) of offset_2,
    (C-1)^2 sum_K (M-K-1) C^(M-K-2) each of offset_1010 and offset_1001."""
    t2 = (C - 2) * sum(C ** (M - K - 1) for K in range(M))
    p = (C - 1) ** 2 * sum((M - K - 1) * C ** (M - K - 2) for K in range(M - 1))
    return C ** M + t2 + 2 * p


@pytest.mark.parametrize("M,C", [(1, 7), (2, 5), (3, 6), (4, 10)])
def test_buffer_curve_endpoints(M, C):
    bc = scaling.buffer_curve((C,) * M)
    # with the buffer only the diagonal is left at the end (Fig. 8, dashed line C^M)
    assert bc["buffer"][-1] == C ** M
    # without a buffer every written amplitude stays (App. B.2)
    assert bc["no_buffer"][-1] == appb_written_b0(M, C)
    # b = 0: the off-diagonal pivots of App. B.1 only, C^M - 1 of them
    assert bc["pivots"][-1] == C ** M - 1
    assert bc["buffer_peak_during"].max() < bc["no_buffer"][-1] or M == 1


def test_counters_match_library_schedule():
    from paper_2303_08879_gb300 import fockdiag as fd
    for cut in ((10, 10, 10, 10), (6, 4, 5), (3, 7)):
        bc = scaling.buffer_curve(cut)
        d = fd.fk_describe_diag_schedule(len(cut), list(cut), fd.FK_FLAG_B_ZERO)
        assert d["stored"] == bc["no_buffer"][-1]
        assert d["pivots"] == bc["pivots"][-1]


def test_space_slopes():
    cs = [8, 10, 12, 14, 16, 20, 24]
    sp = scaling.space_table(4, cs)
    sl = lambda k: scaling.slope(cs, [r[k] for r in sp])
    assert abs(sl("state_vector") - 4) < 1e-9 and abs(sl("naive_dm") - 8) < 1e-9
    # Algorithm 1 and its pivots scale like C^M (App. B), the buffer peak more slowly
    assert 3.9 < sl("algorithm1") < 4.2 and 3.99 < sl("pivots") < 4.01
    assert sl("algorithm1_buffer_peak") < sl("algorithm1")
