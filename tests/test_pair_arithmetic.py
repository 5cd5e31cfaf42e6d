"""The pair-arithmetic residual's algorithm, emulated on the CPU in float32
(numpy), against the exact residual: r = b - A x with every a_ij split into
ah + al (the leading 24 bits of a 2^-ea truncated, the next 29 rounded to
24), every x_j into xh + xl (x 2^-sx rounded to FP32, then the remainder),
each term ah xh formed exactly as p + e (TwoProduct), the cross terms
ah xl + al xh added to the low word, p added to the running high word by
Knuth's TwoSum, and the pair folded into an FP64 accumulator every 16 terms.
The error must stay within the bound the library documents: a few 2^-48 of
the largest 16-term partial sums, so below 5e-14 of ||A|| ||x|| + ||b||
even on rows whose terms cancel to 1e-12."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def _fma32(a, b, c):
    # a b is exact in float64 (24 + 24 bits); the sum is rounded once more to
    # float32 (double rounding can differ from a fused FMA in rare ties, which
    # an error-bound test tolerates)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    err = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, err


def _split_a(a, ea):
    v = np.float64(a) * 2.0 ** -ea
    if v == 0.0 or abs(v) < 2.0 ** -74:
        return f32(0), f32(0)
    bits = np.array([v]).view(np.uint64)[0]
    hi = np.array([bits & ~np.uint64((1 << 29) - 1)], dtype=np.uint64).view(np.float64)[0]   # 24 leading bits
    return f32(hi), f32(v - hi)


def pair_residual(A, x, b, chunk=16):
    n = A.shape[1]
    ea = int(np.ceil(np.log2(np.abs(A).max()))) + 1
    sx = int(np.floor(np.log2(np.abs(x).max())))
    xs = x * 2.0 ** -sx
    xh = xs.astype(f32)
    xl = (xs - xh.astype(np.float64)).astype(f32)
    r = np.empty(A.shape[0])
    for i in range(A.shape[0]):
        acc = 0.0
        hi, lo = f32(0), f32(0)
        for j in range(n):
            ah, al = _split_a(A[i, j], ea)
            p = f32(ah * xh[j])
            e = _fma32(ah, xh[j], -p)
            l = _fma32(ah, xl[j], lo)
            l = _fma32(al, xh[j], l)
            l = f32(l + e)
            hi, t = _two_sum(hi, p)
            lo = f32(l + t)
            if (j + 1) % chunk == 0 or j == n - 1:
                acc += np.float64(hi) + np.float64(lo)
                hi, lo = f32(0), f32(0)
        r[i] = b[i] - acc * 2.0 ** (ea + sx)
    return r


@pytest.mark.parametrize("n,seed", [(64, 0), (200, 1), (333, 2)])
def test_pair_residual_error_bound(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (24, n)) * np.exp2(rng.integers(-6, 7, (24, n)))
    x = rng.standard_normal(n)
    b = A @ x                                   # the residual cancels
    exact = np.array([float(Fraction(b[i]) - sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(n)))
                      for i in range(A.shape[0])])
    r = pair_residual(A, x, b)
    scale = np.abs(A).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max()
    err = np.abs(r - exact).max() / scale
    assert err <= 5e-14, err
    # and it is far better than a plain FP32 product
    r32 = b - (A.astype(f32) @ x.astype(f32)).astype(np.float64)
    assert np.abs(r32 - exact).max() / scale > 1e3 * err


def test_split_is_exact_to_47_bits():
    rng = np.random.default_rng(5)
    for a in rng.standard_normal(200) * np.exp2(rng.integers(-20, 20, 200)):
        ea = int(np.ceil(np.log2(abs(a)))) + 1
        ah, al = _split_a(a, ea)
        v = a * 2.0 ** -ea
        assert abs((np.float64(ah) + np.float64(al)) - v) <= 2.0 ** -47 * abs(v)
