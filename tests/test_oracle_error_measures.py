"""Pins for the oracle's error measures, which decide every parity verdict:
the solve backward error eta (R-2), the factorization residuals of LU and
Cholesky, and the probabilistic residual used at large n.

Each expected value is worked out by hand (exact in binary or in rationals)
from the definition; the wrong-answer cases check that a slip in a measure
would show.  The matrices are chosen so that the 1-norm, the inf-norm, the
Frobenius norm and max |a_ij| of A all differ, and the right-hand sides so
that dropping ||b||, or taking a maximum along the wrong axis, changes the
value.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2108_09337_gb300 import inputs

U53 = Fraction(1, 2 ** 53)

# A = [[3, 4], [0, 1]]: ||A||_inf = 7, ||A||_1 = 5, ||A||_F = sqrt(26),
# max |a_ij| = 4.
A2 = np.array([[3.0, 4.0], [0.0, 1.0]], order="F")


def test_backward_error_hand_values():
    """x1 = (1, 1): A x1 = (7, 1); b1 = (7, 1 + 2^-10) leaves r1 = (0, 2^-10),
    so eta1 = 2^-10 / (7 * 1 + 7) = 1/14336.
    x2 = (2, -1): A x2 = (2, -1); b2 = (2 + 2^-9, -1) leaves r2 = (2^-9, 0),
    so eta2 = 2^-9 / (7 * 2 + 2 + 2^-9) = 1/8193."""
    X = np.array([[1.0, 2.0], [1.0, -1.0]], order="F")
    B = np.array([[7.0, 2.0 + 2.0 ** -9], [1.0 + 2.0 ** -10, -1.0]], order="F")
    eta = oracle.backward_error(A2, X, B)
    assert eta.shape == (2,)
    assert eta[0] == pytest.approx(1.0 / 14336, rel=1e-15)
    assert eta[1] == pytest.approx(1.0 / 8193, rel=1e-15)
    # the slips this rules out, each computed from the same r, x, b
    wrong = {
        "1-norm of A": [2.0 ** -10 / (5 + 7), 2.0 ** -9 / (5 * 2 + 2 + 2.0 ** -9)],
        "dropped ||b||": [2.0 ** -10 / 7, 2.0 ** -9 / 14],
        "Frobenius norm of A": [2.0 ** -10 / (26 ** 0.5 + 7), 2.0 ** -9 / (2 * 26 ** 0.5 + 2 + 2.0 ** -9)],
    }
    for name, w in wrong.items():
        assert not np.allclose(eta, w, rtol=1e-6), name


def test_backward_error_zero_solution_and_exact_solution():
    """x = 0 gives r = b and eta = ||b|| / ||b|| = 1 exactly; an exact solution
    gives eta = 0."""
    B = np.array([[5.0], [-3.0]], order="F")
    assert oracle.backward_error(A2, np.zeros((2, 1)), B)[0] == 1.0
    X = np.array([[1.0], [-2.0]])
    assert oracle.backward_error(A2, X, A2 @ X)[0] == 0.0


def test_backward_error_is_rigal_gaches_perturbation():
    """Rigal & Gaches (1967): eta is the smallest e with (A + dA) x = b + db,
    ||dA||_inf <= e ||A||_inf, ||db||_inf <= e ||b||_inf.  The perturbation
    that attains it, dA = ||A|| r z^T / d, db = -||b|| r / d with
    d = ||A|| ||x|| + ||b|| and z the dual vector of x (z^T x = ||x||_inf,
    ||z||_1 = 1), must solve the system exactly and have those norms, on a
    row-scaled random system (rows scaled by 2^-8 .. 2^8)."""
    rng = np.random.default_rng(11)
    n = 40
    D = 2.0 ** rng.integers(-8, 9, n)
    A = np.asfortranarray(D[:, None] * rng.standard_normal((n, n)))
    x = rng.standard_normal(n)
    b = A @ x + 1e-6 * rng.standard_normal(n)
    eta = oracle.backward_error(A, x.reshape(n, 1), b.reshape(n, 1))[0]
    r = b - A @ x
    na, nb, nx = np.linalg.norm(A, np.inf), np.abs(b).max(), np.abs(x).max()
    k = int(np.argmax(np.abs(x)))
    z = np.zeros(n)
    z[k] = np.sign(x[k])
    d = na * nx + nb
    dA = na * np.outer(r, z) / d
    db = -nb * r / d
    assert np.abs((A + dA) @ x - (b + db)).max() <= 1e-6 * np.abs(r).max()
    assert np.linalg.norm(dA, np.inf) == pytest.approx(eta * na, rel=1e-12)
    assert np.abs(db).max() == pytest.approx(eta * nb, rel=1e-12)


def test_backward_error_is_scale_invariant():
    """eta is homogeneous of degree 0 in (A, b) and in (x, b): scaling the
    system by 2^40, or the solution and right-hand side by 2^-40, leaves it
    unchanged bit for bit (a measure with a squared or missing norm would
    not be)."""
    rng = np.random.default_rng(5)
    n = 16
    A = np.asfortranarray(rng.uniform(-1, 1, (n, n)) + 4 * np.eye(n))
    x = rng.standard_normal((n, 2))
    b = A @ x + 1e-9 * rng.standard_normal((n, 2))
    e0 = oracle.backward_error(A, x, b)
    s = 2.0 ** 40
    np.testing.assert_array_equal(oracle.backward_error(np.asfortranarray(s * A), x, s * b), e0)
    np.testing.assert_array_equal(oracle.backward_error(A, x / s, b / s), e0)


# 3 x 3 LU worked by hand: L = [[1,0,0],[1/2,1,0],[1/4,-1/2,1]],
# U = [[4,2,-2],[0,2,1],[0,0,3]], L U = [[4,2,-2],[2,3,0],[1,-1/2,2]], and
# P A = L U with (P A)[i] = A[p[i]], p = (2, 0, 1), i.e. LAPACK ipiv = (3, 3, 3):
# A = [[2,3,0],[1,-1/2,2],[4,2,-2]]; ||A||_1 = 7, ||A||_inf = 8.
L3 = np.array([[1, 0, 0], [0.5, 1, 0], [0.25, -0.5, 1]])
U3 = np.array([[4.0, 2, -2], [0, 2, 1], [0, 0, 3]])
A3 = np.asfortranarray([[2.0, 3, 0], [1, -0.5, 2], [4, 2, -2]])
IPIV3 = np.array([3, 3, 3], dtype=np.int32)


def test_lu_residual_exact_factors_is_zero():
    LU = np.asfortranarray(np.tril(L3, -1) + U3)
    assert oracle.lu_residual(A3, LU, IPIV3) == 0.0
    np.testing.assert_array_equal(oracle.perm_from_ipiv(IPIV3, 3), [2, 0, 1])


def test_lu_residual_hand_value():
    """U' = U + d e_0 e_1^T (d = 2^-30) leaves P A - L U' = -L d e_0 e_1^T, whose
    only column is d (1, 1/2, 1/4): ||.||_1 = 7d/4, ||.||_inf = d.  The measure
    is 7d/4 / (3 u 7) = 2^23 / 12; the inf-norm would give 2^23 / 24."""
    d = 2.0 ** -30
    LU = np.asfortranarray(np.tril(L3, -1) + U3)
    LU[0, 1] += d
    got = oracle.lu_residual(A3, LU, IPIV3)
    want = Fraction(7, 4) * Fraction(d) / (3 * U53 * 7)
    assert got == pytest.approx(float(want), rel=1e-12)
    assert float(want) == pytest.approx(2 ** 23 / 12, rel=1e-15)


def test_lu_residual_wrong_pivots_or_factor_entry_score_high():
    """On a random matrix the oracle's factors score <= 10; the same factors
    with one interchange changed, or one entry of L or U off by 1e-6, score
    far above 20."""
    n = 64
    A = inputs.uniform_pm1(n, seed=3)
    LU, ipiv, info, _, _ = oracle.getrf(A, v=16, h=32)
    assert info == 0 and oracle.lu_residual(A, LU, ipiv) <= 10
    bad = ipiv.copy()
    bad[5] = 1 if bad[5] != 1 else 2
    assert oracle.lu_residual(A, LU, bad) > 1e6
    for (i, j) in [(40, 3), (3, 40)]:
        LU2 = LU.copy(order="F")
        LU2[i, j] += 1e-6
        assert oracle.lu_residual(A, LU2, ipiv) > 1e6


# Cholesky worked by hand: L0 = [[2,0,0],[1,3,0],[-1,2,1]],
# A = L0 L0^T = [[4,2,-2],[2,10,5],[-2,5,6]], ||A||_1 = 17.
L0 = np.array([[2.0, 0, 0], [1, 3, 0], [-1, 2, 1]])
S3 = np.asfortranarray(L0 @ L0.T)


def test_chol_residual_hand_value():
    """L'(2,0) = -1 + d (d = 2^-20, so every product is exact) changes
    A - L' L'^T by -2d at (2,0) and (0,2), -d at (2,1) and (1,2), 2d - d^2 at
    (2,2): ||.||_1 = 5d - d^2, so the measure is (5d - d^2) / (3 u 17).
    Garbage in the strict upper triangle of L' is ignored; the full symmetric
    A is used (its lower triangle alone would give a different value)."""
    np.testing.assert_array_equal(S3, [[4, 2, -2], [2, 10, 5], [-2, 5, 6]])
    assert oracle.chol_residual(S3, L0) == 0.0
    d = 2.0 ** -20
    L = L0.copy()
    L[2, 0] += d
    L[0, 2] = 123.0
    L[1, 2] = -7.0
    got = oracle.chol_residual(S3, np.asfortranarray(L))
    dd = Fraction(d)
    want = (5 * dd - dd * dd) / (3 * U53 * 17)
    assert got == pytest.approx(float(want), rel=1e-12)
    lower_only = np.linalg.norm(np.tril(S3) - np.tril(L) @ np.tril(L).T, 1) / (3 * oracle.EPS * 17)
    assert abs(lower_only - got) > 1.0


def test_chol_residual_perturbed_factor_scores_high():
    n = 48
    S = inputs.spd_gram(n, seed=4)
    L, info, _ = oracle.potrf(S)
    assert info == 0 and oracle.chol_residual(S, L) <= 10
    L2 = L.copy(order="F")
    L2[30, 7] *= 1 + 1e-8
    assert oracle.chol_residual(S, L2) > 100


def _projection(A, LU, ipiv, nvec=4, seed=0):
    n = A.shape[0]
    L, U = oracle.split_lu(LU)
    p = oracle.perm_from_ipiv(ipiv, n)
    return oracle.lu_random_projection_error(lambda Z: A[p] @ Z, lambda Z: L @ Z, lambda Z: U @ Z, n,
                                             np.linalg.norm(A, "fro"), nvec=nvec, seed=seed)


def test_random_projection_error_bounds():
    """For E = P A - L U: rounding level for exact factors; never above ||E||_2 / ||A||_F;
    for a rank-one E = u v^T it equals max_k ||u|| |v.z_k| / (||A||_F ||z_k||)
    (checked with the same z_k drawn independently), and a wrong interchange
    gives a value of order one."""
    LU = np.asfortranarray(np.tril(L3, -1) + U3)
    assert _projection(A3, LU, IPIV3) <= 4 * oracle.EPS
    d = 2.0 ** -30
    LU[0, 1] += d
    got = _projection(A3, LU, IPIV3, nvec=4, seed=9)
    u = -d * L3[:, 0]                        # E = P A - L U' = u e_1^T
    Z = np.random.default_rng(9).standard_normal((3, 4))
    want = max(np.linalg.norm(u) * abs(Z[1, k]) / (np.linalg.norm(A3, "fro") * np.linalg.norm(Z[:, k]))
               for k in range(4))
    assert got == pytest.approx(want, rel=1e-6)
    assert got <= np.linalg.norm(u) / np.linalg.norm(A3, "fro") * (1 + 1e-12)
    n = 64
    A = inputs.uniform_pm1(n, seed=3)
    LUr, ipiv, _, _, _ = oracle.getrf(A, v=16, h=32)
    good = _projection(A, LUr, ipiv)
    assert good <= 10 * n * oracle.EPS
    bad = ipiv.copy()
    bad[5] = 1 if bad[5] != 1 else 2
    assert _projection(A, LUr, bad) > 1e-2
