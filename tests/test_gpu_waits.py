"""The refinement's blocked triangular solve with FP32 factors (cf_trsv_f32)
against FP64 substitution, and failure detection of its bounded waits
(cf_trsv_f32_withheld, cf_device_status).

The failure is made on the host: the first block's ticket is taken before
the launch, so no CTA ever solves block 0 or raises its flag.  Every wait for
it must give up after its limit, the kernel must end, cf_device_status must
report CF_ERR_TIMEOUT once and then be clear, and the context must stay
usable: a following solve and a mixed-precision solve are correct.  Nothing
here faults, traps or hangs the GPU.

Tolerance of the FP32 solves: |x - x64| <= 1e-4 max |x64| on triangles with
condition number below 5 (FP32 substitution through 128 x 128 diagonal-block
inverses: error ~ n u32 cond).
"""
import time

import numpy as np
import pytest
import scipy.linalg as sla
import torch

import oracle
from paper_2108_09337_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    assert torch.cuda.is_available()
    from paper_2108_09337_gb300 import cf as _cf
    return _cf


def _tri(n, mode, seed):
    """A well-conditioned FP32 triangle for the mode (values exact in FP64)."""
    rng = np.random.default_rng(seed)
    E = rng.uniform(-1, 1, (n, n)) * (0.5 / n)
    if mode == 0:
        T = np.tril(E, -1) + np.triu(rng.uniform(-9, 9, (n, n)), 0)   # unit lower: diagonal and above ignored
    elif mode == 1:
        T = np.triu(E, 1) + np.diag(rng.uniform(1, 2, n)) + np.tril(rng.uniform(-9, 9, (n, n)), -1)
    else:
        T = np.tril(E, -1) + np.diag(rng.uniform(1, 2, n)) + np.triu(rng.uniform(-9, 9, (n, n)), 1)
    return np.asfortranarray(T.astype(np.float32).astype(np.float64))


def _reference(T, X, mode):
    """FP64 substitution: the oracle's getrs with identity pivots for the LU
    triangles (unit L with U = I, or U with L = I), scipy for the Cholesky
    ones."""
    n = T.shape[0]
    ident = np.arange(1, n + 1, dtype=np.int32)
    if mode == 0:
        return oracle.getrs(np.asfortranarray(np.tril(T, -1) + np.eye(n)), ident, X)
    if mode == 1:
        return oracle.getrs(np.asfortranarray(np.triu(T)), ident, X)
    L = np.tril(T)
    return sla.solve_triangular(L, X, lower=True) if mode == 2 else sla.solve_triangular(L.T, X, lower=False)


def _dev32(A):
    return torch.from_numpy(np.ascontiguousarray(A.T.astype(np.float32))).cuda().t()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (200, 3), (1000, 8), (2100, 5), (3000, 16), (5000, 1), (4100, 12)])
def test_trsv_f32_matches_fp64_substitution(cf, mode, n, nrhs):
    """Ragged last blocks (200, 2100, 3000, 4100, 5000 rows), one-block
    solves, every right-hand-side width class (<= 4, <= 8, <= 16)."""
    T = _tri(n, mode, seed=n + mode)
    X = inputs.rhs_normal(n, nrhs, seed=mode).astype(np.float32).astype(np.float64)
    dX = _dev32(X)
    cf.trsv_f32(_dev32(T), dX, mode)
    assert cf.device_status() == cf.CF_OK
    ref = _reference(T, X, mode)
    got = dX.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("n,spin", [(2560, 1 << 14), (256, 0)])
def test_bounded_wait_runs_out_and_recovers(cf, n, spin):
    """spin = 0 takes the library's own limit (2^22 polls, about a tenth of a
    second): the call must still come back within seconds."""
    assert cf.device_status() == 0 or cf.device_status() == 0    # start clear
    mode, nrhs = 0, 4
    T = _tri(n, mode, seed=7)
    X = inputs.rhs_normal(n, nrhs, seed=8).astype(np.float32).astype(np.float64)
    dT, dX = _dev32(T), _dev32(X)
    torch.cuda.synchronize()
    t0 = time.time()
    cf.trsv_f32_withheld(dT, dX, mode, spin_limit=spin)
    st = cf.device_status()                 # synchronises
    dt = time.time() - t0
    assert st == cf.CF_ERR_TIMEOUT
    assert dt < 30.0
    assert cf.device_status() == cf.CF_OK   # reported once, then cleared
    got = dX.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got[:128], X[:128])    # block 0 was never solved
    ref = _reference(T, X, mode)
    if n > 128:   # and the rest is wrong (far outside the solve's FP32 error, ~1e-7 here)
        assert np.abs(got - ref).max() > 1e-5 * np.abs(ref).max()
    # the context is usable: the same solve without the stall is right, and
    # reports no timeout
    dX = _dev32(X)
    cf.trsv_f32(dT, dX, mode)
    assert cf.device_status() == cf.CF_OK
    got = dX.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    # and so is a mixed-precision solve
    m = 1000
    A = inputs.uniform_pm1(m, seed=3, shift=2 * np.sqrt(m))
    B = inputs.rhs_normal(m, 2, seed=4)
    Xs, info, stats, status = cf.gesv_mixed(torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t(),
                                            torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t(), prec="f16")
    assert status == cf.CF_OK
    assert oracle.backward_error(A, Xs.cpu().numpy(), B).max() <= 1e-14
