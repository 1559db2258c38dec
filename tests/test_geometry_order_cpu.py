"""The pivot geometry table of the all-detected walk is built with the AP
pivots numbered densely over (anchor K, level, rank) and handed out
grid-stride; each thread advances its (K, level) position as its numbers
grow.  This models that loop on the host and checks that, for any grid size,
every record of the table (K, level, rank) is produced exactly once at the
position the walk reads it from (family offset + levels below + rank)."""
import itertools

import numpy as np


def ap_counts(C):
    """cnt[K][lev]: AP(K) pivots (e_i = 0 for i < K, e_K <= C_K - 2) of digit sum lev."""
    M, L = len(C), sum(c - 1 for c in C)
    cnt = np.zeros((M, L), np.int64)
    for K in range(M):
        ranges = [range(C[K] - 1)] + [range(C[m]) for m in range(K + 1, M)]
        for e in itertools.product(*ranges):
            if sum(e) < L:
                cnt[K][sum(e)] += 1
    return cnt


def family_offsets(cnt):
    """off_ap[K]: the first record of family K (families stored one after another)."""
    return np.concatenate([[0], np.cumsum(cnt.sum(axis=1))[:-1]])


def nested_order(cnt):
    """(K, lev, r) -> record index, as the walk's readers compute it."""
    M, L = cnt.shape
    off_ap = family_offsets(cnt)
    out = {}
    for K in range(M):
        off = off_ap[K]
        for lev in range(L):
            for r in range(cnt[K][lev]):
                out[(K, lev, r)] = off + r
            off += cnt[K][lev]
    return out


def threaded_order(cnt, gsz):
    """The build loop of every thread of a grid of gsz threads."""
    M, L = cnt.shape
    off_ap = family_offsets(cnt)
    made = []
    for tid in range(gsz):
        K = lev = 0
        kbase = lbase = 0
        c = cnt[0][0]
        t = tid
        while True:
            done = False
            while t >= lbase + c:
                lbase += c
                lev += 1
                if lev >= L:
                    K += 1
                    if K >= M:
                        done = True
                        break
                    lev = 0
                    kbase = lbase
                c = cnt[K][lev]
            if done:
                break
            r = t - lbase
            made.append(((K, lev, r), off_ap[K] + (lbase - kbase) + r))
            t += gsz
    return made


def test_every_record_built_once_where_it_is_read():
    for C in [(3, 2, 4), (2, 2, 2, 2, 3), (6, 6, 6), (4, 2, 5, 3)]:
        cnt = ap_counts(C)
        ref = nested_order(cnt)
        for gsz in (1, 7, 64, 1000):
            made = threaded_order(cnt, gsz)
            keys = [k for k, _ in made]
            assert len(keys) == len(set(keys)) == len(ref)
            for k, idx in made:
                assert ref[k] == idx, (C, gsz, k)
