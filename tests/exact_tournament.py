"""Exact-rational restatement of the tournament-pivoting LU rule, used only to
pin the C oracle (tests).  Written independently of oracle/cf_oracle.c, in
Python ``fractions``, from the same reading of TournPivot (Alg. 1,
Sec. 7.3): leaves of h consecutive panel rows choose their local candidates
by partial-pivoting elimination; playoff nodes stack the candidates of
``arity`` adjacent children (original panel values) and choose again; the
root's choice, in order, gives the pivots of the step.  Ties go to the
smallest stacked position.
"""
from fractions import Fraction


def _select(block):
    """Partial-pivoting selection on a list of rows (lists of Fractions).
    Returns the stacked indices of the chosen rows in pivot order."""
    S = [list(r) for r in block]
    r = len(S)
    w = len(S[0]) if r else 0
    live = list(range(r))
    order = []
    for j in range(min(r, w)):
        best = live[0]
        for i in live[1:]:
            if abs(S[i][j]) > abs(S[best][j]):
                best = i
        order.append(best)
        live.remove(best)
        p = S[best][j]
        if p != 0:
            for i in live:
                f = S[i][j] / p
                for k in range(j + 1, w):
                    S[i][k] -= f * S[best][k]
    return order


def tourn_select(panel, h, arity):
    """panel: list of m rows (each a list of w Fractions)."""
    m = len(panel)
    nodes = []
    for r0 in range(0, m, h):
        rows = list(range(r0, min(r0 + h, m)))
        o = _select([panel[i] for i in rows])
        nodes.append([rows[i] for i in o])
    while len(nodes) > 1:
        nxt = []
        for g in range(0, len(nodes), arity):
            grp = nodes[g:g + arity]
            if len(grp) == 1:
                nxt.append(grp[0])
                continue
            rows = [i for c in grp for i in c]
            o = _select([panel[i] for i in rows])
            nxt.append([rows[i] for i in o])
        nodes = nxt
    return nodes[0]


def getrf(A, v, h, arity):
    """A: list of n rows of Fractions (modified copy).  Returns (LU rows,
    1-based ipiv)."""
    A = [list(r) for r in A]
    n = len(A)
    ipiv = [0] * n
    for k0 in range(0, n, v):
        w = min(v, n - k0)
        panel = [A[i][k0:k0 + w] for i in range(k0, n)]
        win = tourn_select(panel, h, arity)
        label = list(range(n - k0))          # label at each position
        for j, lab in enumerate(win):
            p = label.index(lab)
            ipiv[k0 + j] = k0 + p + 1
            if p != j:
                A[k0 + j], A[k0 + p] = A[k0 + p], A[k0 + j]
                label[j], label[p] = label[p], label[j]
        for k in range(k0, k0 + w):
            piv = A[k][k]
            for i in range(k + 1, n):
                if piv != 0:
                    A[i][k] = A[i][k] / piv
                f = A[i][k]
                if f != 0:
                    rowk = A[k]
                    rowi = A[i]
                    for j in range(k + 1, n):
                        rowi[j] -= f * rowk[j]
    return A, ipiv


def to_fractions(M):
    return [[Fraction(float(x)) for x in row] for row in M]
