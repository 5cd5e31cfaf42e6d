"""Property-based checks of the oracle's tournament (hypothesis): on random
shapes, leaf heights and arities, the selection is min(m, w) distinct rows,
and wherever the oracle's logged gaps are at least 1e-3 it equals the exact
rational restatement; with one leaf over the whole panel it is partial
pivoting (LAPACK's choice)."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from tests import exact_tournament as ex  # noqa: E402


@settings(max_examples=60, deadline=None)
@given(m=st.integers(1, 40), w=st.integers(1, 12), h=st.integers(1, 16), arity=st.integers(2, 4),
       seed=st.integers(0, 10 ** 6))
def test_tournament_selection_properties(m, w, h, arity, seed):
    P = np.random.default_rng(seed).uniform(-1, 1, (m, w))
    win, gap = oracle.tourn_select(P, h=h, arity=arity)
    assert len(win) == min(m, w) and len(set(win.tolist())) == len(win)
    assert win.min() >= 0 and win.max() < m
    if gap >= 1e-3:
        np.testing.assert_array_equal(win, ex.tourn_select(ex.to_fractions(P), h, arity))


@settings(max_examples=40, deadline=None)
@given(m=st.integers(2, 60), w=st.integers(1, 12), seed=st.integers(0, 10 ** 6))
def test_single_leaf_is_partial_pivoting(m, w, seed):
    """The first w pivots of LAPACK's partial pivoting depend only on the
    first w columns, so pad the panel with random columns to a square."""
    import scipy.linalg as sla
    if m < w:
        return
    rng = np.random.default_rng(seed)
    P = rng.uniform(-1, 1, (m, w))
    win, gap = oracle.tourn_select(P, h=m, arity=2)
    if gap < 1e-3:
        return
    _, piv = sla.lu_factor(np.hstack([P, rng.uniform(-1, 1, (m, m - w))]))
    perm = np.arange(m)
    for i, p in enumerate(piv[:w]):
        perm[[i, p]] = perm[[p, i]]
    np.testing.assert_array_equal(win, perm[:w])
