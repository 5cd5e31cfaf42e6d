"""GPU parity of the tensor-core FP64-accurate residual (cf_residual_tc)
against the oracle's compensated residual, through the C ABI, and of the
exactness the method rests on: the tensor cores' FP32 accumulation of integer
digit products.

Bar: |R - R_oracle| <= 1e-15 (||A||_inf ||x_k||_inf + ||b_k||_inf) per column
(the method's error is a few 2^-56 of max_j |a_ij| ||x_k|| per term, the
oracle's ~u^2; the pair-arithmetic kernel is held to 5e-14 and the FP64 one
to 4 n u), on systems whose residual cancels to 1e-12, under power-of-two
scalings far outside FP32 range, with exact zeros, tiny entries, ragged
shapes and more than 16 right-hand sides.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    assert torch.cuda.is_available()
    from paper_2108_09337_gb300 import cf as _cf
    return _cf


def _dev(A, ld=None):
    n, m = A.shape
    if ld is None or ld == n:
        return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    big = torch.zeros((m, ld), dtype=torch.float64)
    big[:, :n] = torch.from_numpy(np.ascontiguousarray(A.T))
    return big.cuda().t()[:n, :]


def _host(t):
    return np.asfortranarray(t.cpu().numpy())


def _err(A, X, B, R):
    Ro = oracle.residual(A, X, B)
    den = np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0)
    return (np.abs(R - Ro).max(0) / den).max()


def test_fp32_accumulation_of_integer_products_is_exact(cf):
    """The premise: BF16 integer operands in [-128, 128] and K = 512 (sums up
    to 2^23) through the tensor-core update give C = -A B^T exactly."""
    rng = np.random.default_rng(0)
    m, n, k = 256, 256, 512
    A = rng.integers(-128, 129, (m, k))
    B = rng.integers(-128, 129, (n, k))
    A[0, :] = 128
    B[0, :] = 128                                  # one entry at 512 * 2^14 = 2^23
    dA = torch.from_numpy(A.astype(np.float32)).to(torch.bfloat16).cuda()
    dB = torch.from_numpy(B.astype(np.float32)).to(torch.bfloat16).cuda()
    C = torch.zeros((n, m), dtype=torch.float32, device="cuda").t()
    cf.schur_update_lp(dA, dB, C)
    ref = -(A.astype(np.int64) @ B.T.astype(np.int64))
    np.testing.assert_array_equal(C.cpu().numpy().astype(np.int64), ref)


@pytest.mark.parametrize("m,n,nrhs,ld", [(129, 129, 3, None), (1000, 1000, 8, None), (2000, 2000, 17, None),
                                         (777, 1500, 1, 781), (9728, 600, 16, None), (3000, 257, 5, 3001),
                                         (64, 1, 2, None)])
def test_residual_tc_accuracy(cf, m, n, nrhs, ld):
    rng = np.random.default_rng(m + n)
    A = rng.uniform(-1.0, 1.0, (m, n))
    k = min(m, n)
    A[np.arange(k), np.arange(k)] += 2 * np.sqrt(n)
    X = rng.standard_normal((n, nrhs)) * 0.1
    B = A @ X + 1e-12 * rng.standard_normal((m, nrhs))
    R = _host(cf.residual_tc(_dev(A, ld), _dev(X), _dev(B)))
    assert _err(A, X, B, R) <= 1e-15


def test_residual_tc_scale_invariance(cf):
    """Scalings of A and X by 2^-700 / 2^600 and 2^300 / 2^-900, an exact-zero
    column of A and a row 1e-30 below the others."""
    n, nrhs = 700, 4
    rng = np.random.default_rng(7)
    A = rng.uniform(-1.0, 1.0, (n, n)) + 2 * np.sqrt(n) * np.eye(n)
    A[:, 5] = 0.0
    A[3, :] *= 1e-30
    X = rng.standard_normal((n, nrhs))
    B = A @ X
    for sa, sx in ((0, 0), (-700, 600), (300, -900)):
        As, Xs, Bs = np.ldexp(A, sa), np.ldexp(X, sx), np.ldexp(B, sa + sx)
        R = _host(cf.residual_tc(_dev(As), _dev(Xs), _dev(Bs)))
        assert np.isfinite(R).all()
        assert _err(As, Xs, Bs, R) <= 1e-15


def test_residual_tc_nonfinite_alias_zero_column(cf):
    """A NaN or inf in A gives NaN in its row only; R may alias B; a zero X
    column gives R = B exactly in the other rows."""
    n, nrhs = 300, 3
    rng = np.random.default_rng(11)
    A = rng.uniform(-1.0, 1.0, (n, n)) + 20 * np.eye(n)
    A[17, 40] = np.nan
    A[99, 3] = np.inf
    X = rng.standard_normal((n, nrhs))
    X[:, 2] = 0.0
    B = rng.standard_normal((n, nrhs))
    dB = _dev(B)
    cf.residual_tc(_dev(A), _dev(X), dB, R=dB)
    R = _host(dB)
    assert np.isnan(R[17]).all() and np.isnan(R[99]).all()
    ok = np.ones(n, bool)
    ok[[17, 99]] = False
    assert not np.isnan(R[ok]).any()
    Ac = A.copy()
    Ac[~ok] = 0.0
    assert _err(Ac[ok], X, B[ok], R[ok]) <= 1e-15
    np.testing.assert_array_equal(R[ok, 2], B[ok, 2])


def test_residual_tc_matches_fp64_kernel_at_benchmark_scale(cf):
    """N = 8192, 16 right-hand sides, the benchmark's LU matrix: against the
    oracle on 256 sampled rows, and within the FP64 kernel's own error of it."""
    from paper_2108_09337_gb300 import inputs
    n, nrhs = 8192, 16
    dA = inputs.uniform_pm1_torch(n, seed=0, shift=2.0 * np.sqrt(n), device="cuda")
    dX = inputs.rhs_normal_torch(n, nrhs, seed=3, device="cuda")
    dB = (dA @ dX).t().contiguous().t()
    R = _host(cf.residual_tc(dA, dX, dB))
    R64 = _host(cf.residual(dA, dX, dB))
    A = _host(dA)
    X, B = _host(dX), _host(dB)
    rows = np.random.default_rng(1).choice(n, 256, replace=False)
    Ro = oracle.residual(np.asfortranarray(A[rows]), X, np.asfortranarray(B[rows]))
    den = np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0)
    assert (np.abs(R[rows] - Ro).max(0) / den).max() <= 1e-15
    assert (np.abs(R - R64).max(0) / den).max() <= 4 * n * oracle.EPS
