"""The tensor-core residual's algorithm, emulated exactly on the CPU (numpy
int64 and Python rationals), against the exact residual.

R = B - A X is formed from integer digit slices:
* per row i of A, E_i is the exponent with max_j |a_ij| < 2^E_i (frexp);
  q_ij = round(a_ij 2^(62 - E_i)) (to nearest, ties away from zero), so
  |q_ij| <= 2^62; per column k of X the same with F_k, giving p_jk;
* q = sum_s d_s 256^(7 - s) with eight balanced base-256 digits (the seven
  low ones in [-128, 127], the top one in [-64, 64]), likewise p with e_t;
* Q_d = sum_{s + t = d} sum_j d_s(q_ij) e_t(p_jk) for d = 0..7: every digit
  and every product is an integer exact in BF16 / FP32, and every partial sum
  over a chunk of 128 consecutive j stays below 2^24, so the tensor cores'
  FP32 accumulation of a chunk is exact whatever its order; chunks add up
  exactly in int64;
* (A X)_ik ~ 2^(E_i + F_k - 68) sum_d Q_d 256^(7 - d) (the digit pairs with
  s + t > 7 are dropped), and R = B - A X in double-double.

The error must stay within 2^-56 of ||A||_inf ||x||_inf + ||b||_inf on rows
that cancel (eight times below FP64's unit roundoff), and the exactness
bounds must hold; dropping the digit pairs of one more diagonal, or keeping
fewer digits, must fail that bound.
"""
from fractions import Fraction

import numpy as np
import pytest

S = 8            # digits per element
D = 7            # largest digit diagonal kept (s + t <= D)
KC = 128         # K chunk accumulated in FP32 before it is added in int64


def _fixed(v, E, bits=8 * S - 2):
    """round(v 2^(bits - E)) to nearest, ties away from zero, as int64."""
    w = np.ldexp(v, bits - E)
    a = np.abs(w)
    big = a >= 2.0 ** 52                      # already integers
    r = np.where(big, a, np.floor(a + 0.5))
    return (np.sign(w) * r).astype(np.int64)


def _digits(q, nd=S):
    """Balanced base-256 digits of int64 q, most significant first."""
    out = []
    for _ in range(nd - 1):
        d = ((q + 128) & 255) - 128
        out.append(d)
        q = (q - d) >> 8
    out.append(q)
    return out[::-1]


def _exps(M, axis):
    m = np.abs(M).max(axis=axis)
    return np.frexp(m)[1].astype(np.int64)       # m < 2^E (E = -1022 floor for zero)


def sliced_residual(A, X, B, nd=S, dmax=D, kc=KC, stats=None):
    E = _exps(A, 1)
    F = _exps(X, 0)
    bits = 8 * nd - 2
    dA = _digits(_fixed(A, E[:, None], bits), nd)
    dX = _digits(_fixed(X, F[None, :], bits), nd)
    n = A.shape[1]
    Q = []
    worst_chunk = 0
    for d in range(dmax + 1):
        acc = np.zeros((A.shape[0], X.shape[1]), dtype=np.int64)
        for j0 in range(0, n, kc):
            part = np.zeros_like(acc)
            for s in range(max(0, d - nd + 1), min(d, nd - 1) + 1):
                part += dA[s][:, j0:j0 + kc] @ dX[d - s][j0:j0 + kc, :]
            worst_chunk = max(worst_chunk, int(np.abs(part).max()))
            acc += part
        Q.append(acc)
    if stats is not None:
        stats["worst_chunk"] = worst_chunk
        stats["max_digit"] = max(int(np.abs(x).max()) for x in dA + dX)
    R = np.empty_like(B)
    for i in range(A.shape[0]):
        for k in range(X.shape[1]):
            T = sum(Fraction(int(Q[d][i, k])) * 256 ** (dmax - d) for d in range(dmax + 1))
            ax = T * Fraction(2) ** int(E[i] + F[k] - 2 * bits + 8 * (2 * (nd - 1) - dmax))
            R[i, k] = float(Fraction(float(B[i, k])) - ax)
    return R


def _exact_residual(A, X, B):
    R = np.empty_like(B)
    for i in range(A.shape[0]):
        for k in range(X.shape[1]):
            s = Fraction(float(B[i, k])) - sum(Fraction(float(a)) * Fraction(float(x))
                                               for a, x in zip(A[i], X[:, k]))
            R[i, k] = float(s)
    return R


def _cancelling_system(n, nrhs, seed, scale_a=1.0, scale_x=1.0):
    """A with a dominant diagonal, b = A x rounded, so that r cancels to about
    1e-16 of ||A|| ||x||, plus a few rows with an exact zero and tiny entries."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (n, n)) + 2 * np.sqrt(n) * np.eye(n)
    A[3, 5] = 0.0
    A[7, :4] = 1e-30
    A *= scale_a
    X = rng.standard_normal((n, nrhs)) * scale_x
    X[9, 0] = 0.0
    B = A @ X
    B[:, 1] += 1e-13 * np.abs(B[:, 1]).max()
    return A, X, B


@pytest.mark.parametrize("n,nrhs,sa,sx", [(300, 3, 1.0, 1.0), (257, 2, 2.0 ** -700, 2.0 ** 600),
                                          (200, 2, 2.0 ** 300, 2.0 ** -900)])
def test_sliced_residual_within_bound(n, nrhs, sa, sx):
    A, X, B = _cancelling_system(n, nrhs, seed=n, scale_a=sa, scale_x=sx)
    st = {}
    R = sliced_residual(A, X, B, stats=st)
    Re = _exact_residual(A, X, B)
    den = np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0)
    err = (np.abs(R - Re).max(0) / den).max()
    assert err <= 2.0 ** -56, err
    # the exactness arguments
    assert st["max_digit"] <= 128
    assert st["worst_chunk"] < 2 ** 24
    # worst case of a chunk: 128 terms of 6 digit pairs of 128 x 128 and of 2
    # pairs with a top digit (<= 64)
    assert KC * (6 * 128 * 128 + 2 * 64 * 128) < 2 ** 24


def test_sliced_residual_slips_fail_the_bound():
    A, X, B = _cancelling_system(300, 2, seed=1)
    Re = _exact_residual(A, X, B)
    den = np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0)
    for kw in ({"dmax": 6}, {"nd": 7, "dmax": 6}):
        R = sliced_residual(A, X, B, **kw)
        err = (np.abs(R - Re).max(0) / den).max()
        assert err > 2.0 ** -56, (kw, err)


def test_digits_reconstruct_and_are_balanced():
    rng = np.random.default_rng(0)
    q = rng.integers(-(2 ** 62), 2 ** 62, 5000, dtype=np.int64)
    q[:4] = [2 ** 62, -(2 ** 62), 0, 128]
    ds = _digits(q)
    back = np.zeros_like(q)
    for d in ds:
        back = back * 256 + d
    np.testing.assert_array_equal(back, q)
    assert np.abs(ds[0]).max() <= 64
    for d in ds[1:]:
        assert d.min() >= -128 and d.max() <= 127
