"""The FP32 tournament's blocked elimination, restated in exact rationals,
selects the same rows as unblocked partial-pivoting elimination.

The kernel updates, at each column of a block of 8, only the block's own
columns, and at the block end applies the rest of the block's eight rank-1
updates at once as a -= sum_u c_u a^_u, where a^_u is pivot u's row as it was
at the block start and c solves c^T (I + L) = l^T (l: the row's multipliers
in the block; L: the pivots' own multipliers with respect to the block's
earlier pivots).  In exact arithmetic that equals unblocked elimination, so
the selections must agree exactly; this pins the algebra the kernel relies
on (its FP32 rounding is covered by the GPU tests)."""
import random
from fractions import Fraction

import pytest

from tests import exact_tournament as ex

BLK = 8


def blocked_select(block):
    S = [list(r) for r in block]
    r = len(S)
    w = len(S[0]) if r else 0
    used = [False] * r
    order = []
    npiv = min(r, w)
    for j0 in range(0, npiv, BLK):
        nb = min(BLK, npiv - j0)
        start = [list(row) for row in S]          # rows at the block start
        lb = [[Fraction(0)] * BLK for _ in range(r)]
        piv = []
        for U in range(nb):
            j = j0 + U
            cand = [i for i in range(r) if not used[i]]
            best = cand[0]
            for i in cand[1:]:
                if abs(S[i][j]) > abs(S[best][j]):
                    best = i
            used[best] = True
            order.append(best)
            piv.append(best)
            p = S[best][j]
            for i in range(r):
                if used[i]:
                    continue
                l = S[i][j] / p if p != 0 else Fraction(0)
                lb[i][U] = l
                for k in range(j + 1, j0 + BLK):   # in-block columns only
                    if k < w:
                        S[i][k] -= l * S[best][k]
        if j0 + BLK >= npiv:
            break
        L = [[lb[piv[u]][t] if t < u else Fraction(0) for t in range(BLK)] for u in range(nb)]
        for i in range(r):
            if used[i]:
                continue
            c = [Fraction(0)] * nb
            for u in range(nb - 1, -1, -1):
                t = lb[i][u]
                for u2 in range(u + 1, nb):
                    t -= c[u2] * L[u2][u]
                c[u] = t
            for k in range(j0 + BLK, w):
                S[i][k] -= sum(c[u] * start[piv[u]][k] for u in range(nb))
    return order


@pytest.mark.parametrize("seed", range(12))
def test_blocked_equals_unblocked(seed):
    rnd = random.Random(seed)
    r = rnd.choice([9, 16, 24, 40])
    w = rnd.choice([5, 8, 13, 20, 24])
    zeros = seed % 3 == 0
    M = [[Fraction(rnd.randint(-9, 9) if not zeros else rnd.choice([0, 0, 1, -1, 2]), rnd.choice([1, 2, 3, 4]))
          for _ in range(w)] for _ in range(r)]
    assert blocked_select(M) == ex._select(M)


def test_blocked_equals_unblocked_with_exact_ties():
    M = [[Fraction(1 if (i + k) % 3 == 0 else 0) for k in range(17)] for i in range(30)]
    assert blocked_select(M) == ex._select(M)
