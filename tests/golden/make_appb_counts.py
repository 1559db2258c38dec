"""Write appb_counts.txt: the counts printed in App. B of arXiv 2303.08879.

App. B.1 (total number of pivots, equal cutoffs C):  2 C^M - C^{M-1} - 1.
App. B.3 (written amplitudes per offset type, equal cutoffs C):
  offset_1     (C-1) C^{M-1} + (C-2) C^{M-1} + (2M-2)(C-1)^2 C^{M-2}
  offset_0     C^M
  offset_2     (C-2) sum_{K=0}^{M-1} C^{M-K-1}
  offset_1010  (C-1)^2 sum_{K=0}^{M-1} (M-K-1) C^{M-K-2}
  offset_1001  same as offset_1010
The script only evaluates those printed formulas; it calls nothing else.
"""
import os
from fractions import Fraction


def counts(M, C):
    C = Fraction(C)
    off1 = (C - 1) * C ** (M - 1) + (C - 2) * C ** (M - 1) + (2 * M - 2) * (C - 1) ** 2 * C ** (M - 2)
    off0 = C ** M
    off2 = (C - 2) * sum(C ** (M - K - 1) for K in range(M))
    o1010 = (C - 1) ** 2 * sum((M - K - 1) * C ** (M - K - 2) for K in range(M))
    piv = 2 * C ** M - C ** (M - 1) - 1
    return [int(v) for v in (off1, off0, off2, o1010, o1010, piv)]


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "appb_counts.txt")
    with open(out, "w") as f:
        f.write("# App. B.1 and B.3 of arXiv 2303.08879 (Algorithm 1, equal cutoffs C, M modes)\n")
        f.write("# M C offset_1 offset_0 offset_2 offset_1010 offset_1001 pivots\n")
        for M in (1, 2, 3, 4, 5):
            for C in (2, 3, 4, 6, 10):
                if C ** M > 20000:
                    continue
                f.write(" ".join(str(v) for v in [M, C] + counts(M, C)) + "\n")
