"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- LAPACK (scipy) in the special case the rule reduces to, exact
constructed factors, exact rational arithmetic, permutation-expansion
determinants, the error bound of backward-stable elimination, and the closed
forms the paper states.  A plausible slip in the oracle (a dropped update, a
wrong sign or index, a transposed operand, candidates taken from eliminated
instead of original values, a wrong tie rule) fails at least one of them.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2108_09337_gb300 import inputs
from tests import exact_tournament as ex


def _scipy_ipiv(A):
    _, piv = sla.lu_factor(A)
    return piv.astype(np.int64) + 1


# ---------------------------------------------------------------- GEPP mode
@pytest.mark.parametrize("n,v", [(16, 4), (64, 16), (200, 32), (300, 128)])
def test_gepp_mode_recovers_constructed_permutation(n, v):
    """h >= n: the tournament is partial pivoting; on A = P^T L U with every
    argmax separated by >= 1e-3 it must return P exactly and match LAPACK's
    pivots and factors (to rounding: both are the same elimination in a
    different summation order), with a backward error below 10 n u."""
    A, perm, L, U = inputs.constructed_plu(n, seed=n)
    LU, ipiv, info, gaps, _ = oracle.getrf(A, v=v, h=n + 1)
    assert info == 0
    assert gaps.min() >= 1e-3 * 0.5
    np.testing.assert_array_equal(oracle.perm_from_ipiv(ipiv, n), perm)
    np.testing.assert_array_equal(ipiv, _scipy_ipiv(A))
    lu_s, _ = sla.lu_factor(A)
    assert np.abs(LU - lu_s).max() <= 1e-9 * np.abs(lu_s).max()
    assert oracle.lu_residual(A, LU, ipiv) <= 10


@pytest.mark.parametrize("seed", range(6))
def test_gepp_mode_matches_lapack_on_random(seed):
    n = 96
    A = inputs.uniform_pm1(n, seed=seed)
    LU, ipiv, info, gaps, _ = oracle.getrf(A, v=32, h=10 ** 6)
    lu_s, piv_s = sla.lu_factor(A)
    if gaps.min() >= 1e-3:
        np.testing.assert_array_equal(ipiv, piv_s + 1)
        assert np.abs(LU - lu_s).max() <= 1e-10
    assert oracle.lu_residual(A, LU, ipiv) <= 10


@pytest.mark.parametrize("n", [8, 33, 64])
def test_dyadic_exact_recovery(n):
    """Every intermediate value is exact in binary64: elimination must
    reproduce L and U bit for bit."""
    A, perm, L, U = inputs.dyadic_plu(n, seed=100 + n)
    for v in (1, 5, 16, 64):
        LU, ipiv, info, _, _ = oracle.getrf(A, v=v, h=10 ** 6)
        assert info == 0
        np.testing.assert_array_equal(oracle.perm_from_ipiv(ipiv, n), perm)
        Lo, Uo = oracle.split_lu(LU)
        np.testing.assert_array_equal(Lo, L)
        np.testing.assert_array_equal(Uo, U)


# ------------------------------------------------------ tournament (exact)
CASES = [(n, v, h, a) for n in (5, 9, 16) for v in (2, 3, 4)
         for h in (2, 3, 5, 10 ** 6) for a in (2, 3)]


@pytest.mark.parametrize("n,v,h,arity", CASES)
def test_tournament_matches_exact_rational(n, v, h, arity):
    """The oracle's pivots equal an exact-rational restatement of the rule
    whenever every logged gap is >= 1e-3; factors agree to rounding."""
    checked = 0
    for seed in range(40):
        A = inputs.uniform_pm1(n, seed=1000 * n + 10 * v + seed)
        LU, ipiv, info, gaps, _ = oracle.getrf(A, v=v, h=h, arity=arity)
        if gaps.min() < 1e-3:
            continue
        LUx, ipx = ex.getrf(ex.to_fractions(A), v, h, arity)
        np.testing.assert_array_equal(ipiv, ipx)
        LUf = np.array([[float(x) for x in r] for r in LUx])
        scale = max(1.0, np.abs(LUf).max())
        assert np.abs(LU - LUf).max() <= 1e-11 * scale
        checked += 1
        if checked >= 3:
            break
    assert checked >= 1


def test_tournament_select_matches_exact_on_tall_panel():
    m, w = 60, 4
    for seed in range(10):
        P = inputs.uniform_pm1(m, seed=seed, m=w)
        for h, a in ((7, 2), (12, 3), (5, 4)):
            win, gap = oracle.tourn_select(P, h=h, arity=a)
            if gap < 1e-3:
                continue
            wx = ex.tourn_select(ex.to_fractions(P), h, a)
            np.testing.assert_array_equal(win, wx)


def test_playoff_uses_original_values_not_eliminated():
    """A hand-made panel where a playoff on eliminated values would choose a
    different second pivot than the rule (original values) does."""
    # Leaf 0 = rows 0,1 ; leaf 1 = rows 2,3 ; h = 2, w = 2.
    P = np.array([[4.0, 1.0],
                  [1.0, 4.0],    # leaf-0 winners: row 0 then row 1
                  [3.0, 0.0],
                  [2.0, 3.0]])  # leaf-1 winners: row 2 then row 3
    win, _ = oracle.tourn_select(P, h=2, arity=2)
    wx = ex.tourn_select(ex.to_fractions(P), 2, 2)
    np.testing.assert_array_equal(win, wx)
    # Root on original values: col 0 picks row 0 (4); after eliminating with
    # row 0: row1 -> 4-0.25 = 3.75, row2 -> 0-0.75 = -0.75, row3 -> 3-0.5 = 2.5
    np.testing.assert_array_equal(win, [0, 1])


def test_tie_goes_to_smallest_stacked_position():
    P = np.array([[1.0, 0.0], [-1.0, 2.0], [1.0, -3.0]])
    win, gap = oracle.tourn_select(P, h=10, arity=2)
    assert win[0] == 0 and gap == 0.0
    # after eliminating with row 0: row1 col1 = 2, row2 col1 = -3 -> row 2
    assert win[1] == 2


def test_tournament_differs_from_partial_pivoting_somewhere():
    diffs = 0
    for seed in range(20):
        A = inputs.uniform_pm1(64, seed=seed)
        _, ip_t, _, _, _ = oracle.getrf(A, v=16, h=8)
        _, ip_g, _, _, _ = oracle.getrf(A, v=16, h=10 ** 6)
        diffs += int(not np.array_equal(ip_t, ip_g))
    assert diffs > 0


# ------------------------------------------------------------- stability
@pytest.mark.parametrize("n,v,h,a", [(200, 32, 50, 2), (333, 64, 40, 3),
                                     (257, 128, 128, 2), (128, 128, 128, 2)])
def test_tournament_backward_error(n, v, h, a):
    A = inputs.uniform_pm1(n, seed=n)
    LU, ipiv, info, _, _ = oracle.getrf(A, v=v, h=h, arity=a)
    assert info == 0
    assert oracle.lu_residual(A, LU, ipiv) <= 10


# ---------------------------------------------------------- determinants
def _leibniz(M):
    n = M.shape[0]
    tot = Fraction(0)
    for p in itertools.permutations(range(n)):
        sgn = 1
        for i in range(n):
            for j in range(i + 1, n):
                if p[i] > p[j]:
                    sgn = -sgn
        prod = Fraction(1)
        for i in range(n):
            prod *= Fraction(float(M[i, p[i]]))
        tot += sgn * prod
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_lu_determinant_equals_permutation_expansion(n):
    for seed in range(5):
        A = inputs.small_int(n, seed=10 * n + seed)
        det = _leibniz(A)
        for v, h in ((n, 10 ** 6), (2, 2), (1, 3)):
            LU, ipiv, info, _, _ = oracle.getrf(A, v=v, h=h)
            sign = (-1) ** int(np.sum(ipiv != np.arange(1, n + 1)))
            d = sign * np.prod(np.diag(LU))
            if det == 0:
                assert abs(d) <= 1e-9 * max(1.0, np.abs(A).max() ** n)
            else:
                assert abs(d - float(det)) <= 1e-12 * abs(float(det)) + 1e-12


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_cholesky_determinant_equals_permutation_expansion(n):
    A, _ = inputs.integer_l0(n, seed=n)
    L, info, _ = oracle.potrf(A)
    assert info == 0
    assert float(_leibniz(A)) == pytest.approx(np.prod(np.diag(L)) ** 2,
                                               rel=1e-13)


# ---------------------------------------------------------------- Cholesky
@pytest.mark.parametrize("n", [1, 7, 32, 64])
def test_cholesky_exact_recovery_integer_l0(n):
    A, L0 = inputs.integer_l0(n, seed=200 + n)
    L, info, _ = oracle.potrf(A)
    assert info == 0
    np.testing.assert_array_equal(L, L0)


@pytest.mark.parametrize("n", [50, 300])
def test_cholesky_matches_lapack(n):
    A = inputs.spd_gram(n, seed=1)
    L, info, _ = oracle.potrf(A)
    Ls = sla.cholesky(A, lower=True)
    assert info == 0
    assert np.abs(L - Ls).max() <= 1e-12 * np.abs(Ls).max()
    assert oracle.chol_residual(A, L) <= 10


def test_cholesky_reads_lower_triangle_only():
    A = inputs.spd_gram(40, seed=3)
    B = A.copy(order="F")
    B[np.triu_indices(40, 1)] = np.nan
    L1, _, _ = oracle.potrf(A)
    L2, _, _ = oracle.potrf(B)
    np.testing.assert_array_equal(L1, L2)


def test_cholesky_not_spd_info():
    A = np.asfortranarray(np.diag([4.0, 1.0, -1.0, 2.0]))
    _, info, _ = oracle.potrf(A)
    assert info == 3
    A = inputs.spd_gram(20, seed=1)
    A[7, 7] = -50.0
    _, info, _ = oracle.potrf(A)
    Ls_ok = True
    try:
        sla.cholesky(A[:7, :7], lower=True)
    except np.linalg.LinAlgError:
        Ls_ok = False
    assert Ls_ok and info == 8


# ------------------------------------------------------------ singular LU
def test_zero_column_sets_info():
    n = 12
    A = inputs.uniform_pm1(n, seed=5)
    A[:, 4] = 0.0
    for v, h in ((4, 10 ** 6), (4, 3), (12, 5)):
        LU, ipiv, info, _, _ = oracle.getrf(A, v=v, h=h)
        assert info == 5
        assert np.isfinite(LU).all()


# ------------------------------------------------------------------ solves
def test_getrs_potrs_against_lapack():
    n = 150
    A = inputs.uniform_pm1(n, seed=9)
    B = inputs.rhs_normal(n, 3, seed=2)
    LU, ipiv, _, _, _ = oracle.getrf(A, v=32, h=40)
    X = oracle.getrs(LU, ipiv, B)
    Xs = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A, 1)
    assert np.abs(X - Xs).max() <= kappa * 1e3 * oracle.EPS * np.abs(Xs).max()
    assert oracle.backward_error(A, X, B).max() <= 1e-14
    S = inputs.spd_gram(n, seed=1)
    L, _, _ = oracle.potrf(S)
    X = oracle.potrs(L, B)
    assert np.abs(X - np.linalg.solve(S, B)).max() <= 1e-12 * np.abs(X).max()


# ------------------------------------------------------------- residual
def test_compensated_residual_is_nearly_exact():
    rng = np.random.default_rng(4)
    n = 40
    A = np.asfortranarray(rng.standard_normal((n, n)))
    X = np.asfortranarray(rng.standard_normal((n, 2)))
    B = np.asfortranarray(A @ X)  # residual is tiny: cancellation-heavy
    R = oracle.residual(A, X, B)
    for c in range(2):
        for i in range(n):
            exact = Fraction(float(B[i, c])) - sum(
                Fraction(float(A[i, j])) * Fraction(float(X[j, c]))
                for j in range(n))
            scale = sum(abs(float(A[i, j]) * float(X[j, c])) for j in range(n))
            assert abs(R[i, c] - float(exact)) <= 4 * oracle.EPS ** 2 * scale \
                + 2 * oracle.EPS * abs(float(exact))


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [1, 2, 17, 100])
def test_statement_counts_match_closed_forms(n):
    A = inputs.uniform_pm1(n, seed=1)
    _, _, _, _, nupd = oracle.getrf(A, v=7, h=5)
    assert nupd == oracle.lu_update_count(n)
    S = inputs.spd_gram(n, seed=1)
    _, _, nupd = oracle.potrf(S)
    assert nupd == oracle.chol_update_count(n)


def test_flop_conventions_are_leading_terms():
    n = 10 ** 5
    assert 2 * oracle.lu_update_count(n) / oracle.lu_flops(n) == pytest.approx(1, rel=1e-4)
    assert 2 * oracle.chol_update_count(n) / oracle.chol_flops(n) == pytest.approx(1, rel=1e-4)
    # Sec. 6.1 counts |V2| = N(N-1)(N-2)/3 with its own index convention;
    # its double sum sum_k (N-k)(N-k-1) gives exactly that value.
    N = 50
    assert sum((N - k) * (N - k - 1) for k in range(1, N + 1)) == N * (N - 1) * (N - 2) // 3


def test_io_bounds_closed_forms():
    P, M = 152.0, 484 * 1024 / 8
    for N in (2048.0, 32768.0, 1e7):
        lb = oracle.io_lower_bound_lu(N, P, M)
        assert lb > 0
    # COnfLUX's leading term is 3/2 of the LU lower bound (Sec. 7.4).
    N = 1e9
    assert oracle.io_conflux(N, P, M) / oracle.io_lower_bound_lu(N, P, M) == pytest.approx(1.5, rel=1e-3)
    # Cholesky's lower bound has half the leading term of LU's.
    assert oracle.io_lower_bound_chol(N, P, M) / oracle.io_lower_bound_lu(N, P, M) == pytest.approx(0.5, rel=1e-3)
