"""The reverse of step 1 of the conditional walk (Algorithm 2, the undetected
sub-lattice walked by eq. (recrel)) runs in pull form: each point v gathers
its adjoint from its readers instead of each reader pushing into it.  The
forward writes u from the pivot P = u - 1_w, w the first nonzero position of
u, reading P (the b term) and P - 1_t for every t with P_t > 0 (the A term).
The pull form claims the readers of v are exactly u = v + 1_w (b term) and
u = v + 1_t + 1_w with t >= w (A term), for every w not above the first
nonzero position of v, inside the box.  This checks that claim against the
push form on random mixed-radix boxes, edge by edge."""
import itertools
from collections import Counter

import numpy as np


def push_edges(C):
    """(reader u, target, term, t) of the forward rule, over the whole box."""
    edges = Counter()
    for u in itertools.product(*[range(c) for c in C]):
        if not any(u):
            continue
        w = next(q for q, d in enumerate(u) if d > 0)
        P = list(u)
        P[w] -= 1
        edges[(u, tuple(P), "b", -1)] += 1
        for t in range(len(C)):
            if P[t] > 0:
                r = list(P)
                r[t] -= 1
                edges[(u, tuple(r), "A", t)] += 1
    return edges


def pull_edges(C):
    """The same edges as the pull form enumerates them, target by target."""
    edges = Counter()
    n = len(C)
    for v in itertools.product(*[range(c) for c in C]):
        f0 = next((q for q, d in enumerate(v) if d > 0), n)
        for w in range(n):
            if w > f0:
                break
            if v[w] + 1 >= C[w]:
                continue
            u1 = list(v)
            u1[w] += 1
            edges[(tuple(u1), v, "b", -1)] += 1
            for t in range(w, n):
                u2 = list(u1)
                u2[t] += 1
                if u2[t] >= C[t]:
                    continue
                edges[(tuple(u2), v, "A", t)] += 1
    return edges


def test_pull_enumerates_the_push_edges_exactly():
    rng = np.random.default_rng(5)
    boxes = [(3, 3), (1, 4), (5, 2), (2, 2, 2, 2), (3, 1, 4, 2), (4, 4, 3, 3)]
    boxes += [tuple(int(x) for x in rng.integers(1, 5, size=int(rng.integers(2, 7)))) for _ in range(6)]
    for C in boxes:
        assert pull_edges(C) == push_edges(C), C


def test_readers_lie_one_or_two_levels_above():
    # the level order the block walks (top down) finalises every reader first
    for C in [(3, 4), (2, 3, 2, 3)]:
        for (u, v, term, _), k in push_edges(C).items():
            assert k == 1
            assert sum(u) - sum(v) == (1 if term == "b" else 2)
