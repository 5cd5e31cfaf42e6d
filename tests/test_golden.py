"""The oracle against the hand-worked fixtures in tests/golden/ (each fixture
states its rule and derivation): tournament pivoting on an 8 x 2 panel at
every tree level, the first step of an LU with v = 2 on it, partial pivoting
on a 3 x 3 matrix and Cholesky on a 3 x 3 matrix with an integer factor.
All values are exact in binary, so equality is exact."""
import numpy as np

import oracle
from paper_2108_09337_gb300 import inputs
from tests import exact_tournament as ex
from tests.golden_fixtures import load

T = load("tournament_8x2_h2.txt")
P = T["panel"]
H = int(T["h"][0])
AR = int(T["arity"][0])


def _sel(rows):
    """Winners of the sub-tree over panel rows `rows` (consecutive), as
    global row indices."""
    win, _ = oracle.tourn_select(P[rows], h=H, arity=AR)
    return [rows.start + int(i) for i in win]


def test_tournament_levels():
    leaves = [_sel(slice(r, r + H)) for r in range(0, 8, H)]
    assert sum(leaves, []) == T["leaf_winners"].astype(int).tolist()
    nodes = [_sel(slice(0, 4)), _sel(slice(4, 8))]
    assert sum(nodes, []) == T["node_winners"].astype(int).tolist()
    assert _sel(slice(0, 8)) == T["root_winners"].astype(int).tolist()


def test_tournament_root_and_exact_restatement():
    root = T["root_winners"].astype(int)
    win, gap = oracle.tourn_select(P, h=H, arity=AR)
    np.testing.assert_array_equal(win, root)
    np.testing.assert_array_equal(ex.tourn_select(ex.to_fractions(P), H, AR), root)


def test_partial_pivoting_differs_on_this_panel():
    win, _ = oracle.tourn_select(P, h=8, arity=AR)      # one leaf over all rows
    np.testing.assert_array_equal(win, T["gepp_winners"].astype(int))
    assert not np.array_equal(win, T["root_winners"].astype(int))


def test_first_lu_step_on_the_panel():
    A = np.zeros((8, 8))
    A[:, :2] = P
    A[:, 2:] = inputs.uniform_pm1(8, seed=11, m=6)      # later columns: any values
    LU, ipiv, info, _, _ = oracle.getrf(A, v=2, h=H, arity=AR)
    np.testing.assert_array_equal(ipiv[:2], T["ipiv_first2"].astype(int))
    np.testing.assert_array_equal(LU[:2, :2].ravel(), [T["u00"][0], T["u00"][1], T["l00_21"][0], T["u00"][3]])
    got = sorted(map(tuple, LU[2:, :2].tolist()))
    want = sorted(map(tuple, T["l10_pairs"].reshape(-1, 2).tolist()))
    assert got == want
    assert np.abs(LU[2:, :2]).max() == 1.125              # |L| > 1 under tournament pivoting


def test_lu_partial_pivoting_3x3():
    G = load("lu_gepp_3x3.txt")
    LU, ipiv, info, _, _ = oracle.getrf(G["a"], v=2, h=128, arity=2)
    assert info == 0
    np.testing.assert_array_equal(ipiv, G["ipiv"].astype(int))
    np.testing.assert_array_equal(LU, G["lu"])
    sign = (-1) ** int(np.sum(ipiv != np.arange(1, 4)))
    assert sign * np.prod(np.diag(LU)) == G["det"][0]


def test_cholesky_3x3():
    G = load("cholesky_3x3.txt")
    L, info, _ = oracle.potrf(G["a"])
    assert info == 0
    np.testing.assert_array_equal(L, G["l"])
    assert np.prod(np.diag(L)) ** 2 == G["det"][0]


S = load("tournament_9x2_short_leaf.txt")


def _sel9(rows):
    win, _ = oracle.tourn_select(S["panel"][rows], h=int(S["h"][0]), arity=int(S["arity"][0]))
    return [rows.start + int(i) for i in win]


def test_short_leaf_pass_through_and_node_tie():
    P9 = S["panel"]
    h, ar = int(S["h"][0]), int(S["arity"][0])
    leaves = [_sel9(slice(r, min(r + h, 9))) for r in range(0, 9, h)]
    assert sum(leaves, []) == S["leaf_winners"].astype(int).tolist()
    level1 = _sel9(slice(0, 4)) + _sel9(slice(4, 8)) + _sel9(slice(8, 9))
    assert level1 == S["level1_winners"].astype(int).tolist()
    level2 = _sel9(slice(0, 8)) + _sel9(slice(8, 9))
    assert level2 == S["level2_winners"].astype(int).tolist()
    win, gap = oracle.tourn_select(P9, h=h, arity=ar)
    np.testing.assert_array_equal(win, S["root_winners"].astype(int))
    assert gap == 0.0                                    # the exact node tie is logged
    np.testing.assert_array_equal(ex.tourn_select(ex.to_fractions(P9), h, ar), S["root_winners"].astype(int))
    gepp, _ = oracle.tourn_select(P9, h=9, arity=ar)
    np.testing.assert_array_equal(gepp, S["gepp_winners"].astype(int))
