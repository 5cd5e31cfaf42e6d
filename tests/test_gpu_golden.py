"""The CUDA path against the hand-worked fixtures in tests/golden/, through
the C ABI: the FP64 and FP32 tournaments on the 8 x 2 panel, the first LU
step with v = 2 on it, partial pivoting and Cholesky on 3 x 3 matrices.
Every value is exact in binary (dyadic multipliers, integer Cholesky
factor), so both precisions must reproduce them exactly."""
import numpy as np
import pytest
import torch

from paper_2108_09337_gb300 import inputs
from tests.golden_fixtures import load

pytestmark = pytest.mark.gpu

T = load("tournament_8x2_h2.txt")


@pytest.fixture(scope="module")
def cf():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2108_09337_gb300 import cf as _cf
    return _cf


def _dev(A, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(A.T.astype(dtype))).cuda().t()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tournament_panel(cf, dtype):
    h, ar = int(T["h"][0]), int(T["arity"][0])
    win = cf.tourn_select(_dev(T["panel"], dtype), leaf_h=h, arity=ar).cpu().numpy()
    np.testing.assert_array_equal(win, T["root_winners"].astype(int))
    win = cf.tourn_select(_dev(T["panel"], dtype), leaf_h=8, arity=ar).cpu().numpy()
    np.testing.assert_array_equal(win, T["gepp_winners"].astype(int))


def test_first_lu_step(cf):
    A = np.zeros((8, 8))
    A[:, :2] = T["panel"]
    A[:, 2:] = inputs.uniform_pm1(8, seed=11, m=6)
    dA = _dev(A)
    ipiv, info = cf.getrf(dA, v=2, leaf_h=int(T["h"][0]), arity=int(T["arity"][0]))
    LU = dA.cpu().numpy()
    np.testing.assert_array_equal(ipiv.cpu().numpy()[:2], T["ipiv_first2"].astype(int))
    u = T["u00"]
    np.testing.assert_array_equal(LU[:2, :2].ravel(), [u[0], u[1], T["l00_21"][0], u[3]])
    got = sorted(map(tuple, LU[2:, :2].tolist()))
    assert got == sorted(map(tuple, T["l10_pairs"].reshape(-1, 2).tolist()))


def test_lu_and_cholesky_3x3(cf):
    G = load("lu_gepp_3x3.txt")
    dA = _dev(G["a"])
    ipiv, info = cf.getrf(dA, v=2, leaf_h=128, arity=2)
    assert int(info.item()) == 0
    np.testing.assert_array_equal(ipiv.cpu().numpy(), G["ipiv"].astype(int))
    np.testing.assert_array_equal(dA.cpu().numpy(), G["lu"])
    C = load("cholesky_3x3.txt")
    dS = _dev(C["a"])
    info = cf.potrf(dS)
    assert int(info.item()) == 0
    S = dS.cpu().numpy()
    np.testing.assert_array_equal(np.tril(S), C["l"])
    np.testing.assert_array_equal(np.triu(S, 1), np.triu(C["a"], 1))   # upper triangle untouched


def test_tournament_short_leaf_and_node_tie_fp64(cf):
    """A short last leaf passing through two levels and an exact tie at a
    playoff node (tests/golden/tournament_9x2_short_leaf.txt), FP64."""
    S = load("tournament_9x2_short_leaf.txt")
    h, ar = int(S["h"][0]), int(S["arity"][0])
    win = cf.tourn_select(_dev(S["panel"]), leaf_h=h, arity=ar).cpu().numpy()
    np.testing.assert_array_equal(win, S["root_winners"].astype(int))
    win = cf.tourn_select(_dev(S["panel"]), leaf_h=9, arity=ar).cpu().numpy()
    np.testing.assert_array_equal(win, S["gepp_winners"].astype(int))
