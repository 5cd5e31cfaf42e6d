"""GPU parity of the FP64 path (cf_tourn_select, cf_getrf, cf_potrf,
cf_getrs, cf_potrs, cf_residual) against the CPU oracle, through the C ABI.

Tolerances (FP64, u = 2^-53):
* tournament selection on the same panel bytes: identical winners (both sides
  round every elimination step identically);
* pivot sequences: identical, except that a step whose oracle-logged argmax
  gap is below 1e-10 may differ (the two sides sum the Schur updates in a
  different order, so values differ by O(n u) relative);
* factors: max |GPU - oracle| <= 1e-9 max |oracle| (same pivots, backward
  stable both; differences are O(kappa n u));
* backward error ||PA - LU||_1 / (n u ||A||_1) <= 20, i.e. within the target
  20 n eps64 with room to spare.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_09337_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2108_09337_gb300 import cf as _cf
    return _cf


def _dev(A, ld=None):
    """Column-major device copy of a host matrix, optionally with ld > rows."""
    n, m = A.shape
    if ld is None or ld == n:
        return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    big = torch.zeros((m, ld), dtype=torch.float64)
    big[:, :n] = torch.from_numpy(np.ascontiguousarray(A.T))
    return big.cuda().t()[:n, :]


def _host(t):
    return np.asfortranarray(t.cpu().numpy())


# tournament arity the FP64 routines take by default
AR = 8


def _pivots_agree(ip_gpu, ip_or, gaps, v):
    if np.array_equal(ip_gpu, ip_or):
        return True
    first = int(np.argmax(ip_gpu != ip_or))
    step = first // v
    return gaps[: step + 1].min() < 1e-10


# ------------------------------------------------------------- LU-1 alone
@pytest.mark.parametrize("m,w,h,arity", [
    (128, 128, 128, 2), (1, 1, 128, 2), (50, 128, 128, 2), (1000, 128, 128, 2),
    (777, 100, 50, 3), (300, 17, 128, 4), (5000, 128, 128, 2), (4099, 64, 7, 2),
    (2000, 128, 128, 4), (129, 128, 128, 3), (2000, 128, 128, 8), (5000, 128, 100, 5), (1500, 128, 64, 6),
    (9000, 128, 128, 7), (130, 128, 128, 8), (40000, 128, 128, 8)])
def test_tourn_select_bit_identical(cf, m, w, h, arity):
    P = inputs.uniform_pm1(m, seed=m + w, m=w)
    win_o, _ = oracle.tourn_select(P, h=h, arity=arity)
    win = cf.tourn_select(_dev(P), leaf_h=h, arity=arity)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(win.cpu().numpy(), win_o)


def test_tourn_select_ties_and_zeros(cf):
    P = np.zeros((300, 8))
    P[::3, :] = 1.0           # many exact ties
    P[7, 0] = -1.0
    win_o, _ = oracle.tourn_select(P, h=16, arity=2)
    win = cf.tourn_select(_dev(P), leaf_h=16, arity=2)
    np.testing.assert_array_equal(win.cpu().numpy(), win_o)


@pytest.mark.parametrize("arity", [2, 8])
def test_tourn_select_full_height_panel(cf, arity):
    """The first panel of the N = 32768 LU workload (32768 x 128)."""
    m, w = 32768, 128
    P = inputs.uniform_pm1(m, seed=0, m=w)
    win_o, _ = oracle.tourn_select(P, h=128, arity=arity)
    win = cf.tourn_select(_dev(P), leaf_h=128, arity=arity)
    np.testing.assert_array_equal(win.cpu().numpy(), win_o)


# ------------------------------------------------------------------- LU
LU_CASES = [(1, 128, 128, 2), (2, 128, 128, 2), (5, 2, 3, 2), (127, 128, 128, 2), (128, 128, 128, 2),
            (129, 128, 128, 2), (300, 64, 40, 3), (515, 128, 128, 2), (700, 100, 128, 4), (1000, 128, 17, 2),
            (1000, 128, 128, 8), (2048, 128, 128, 8), (1200, 64, 32, 6)]


@pytest.mark.parametrize("n,v,h,arity", LU_CASES)
def test_getrf_matches_oracle(cf, n, v, h, arity):
    A = inputs.uniform_pm1(n, seed=n)
    dA = _dev(A)
    ipiv, info = cf.getrf(dA, v=v, leaf_h=h, arity=arity)
    LU = _host(dA)
    ip = ipiv.cpu().numpy()
    LUo, ipo, info_o, gaps, _ = oracle.getrf(A, v=v, h=h, arity=arity)
    assert int(info.item()) == info_o == 0
    assert _pivots_agree(ip, ipo, gaps, v)
    assert oracle.lu_residual(A, LU, ip) <= 20.0
    if np.array_equal(ip, ipo):
        assert np.abs(LU - LUo).max() <= 1e-9 * np.abs(LUo).max()


def test_getrf_first_step_bit_identical(cf):
    """Step 0 (tournament, swaps, A00, both panel solves) uses the oracle's
    rounding; only the Schur update differs.  Its A10/A01/A00 blocks must match
    bit for bit."""
    n, v = 600, 128
    A = inputs.uniform_pm1(n, seed=3)
    dA = _dev(A)
    ipiv, info = cf.getrf(dA, v=v)
    LU = _host(dA)
    LUo, ipo, _, _, _ = oracle.getrf(A, v=v, arity=AR)
    np.testing.assert_array_equal(ipiv.cpu().numpy()[:v], ipo[:v])
    np.testing.assert_array_equal(LU[:, :v], LUo[:, :v])
    np.testing.assert_array_equal(LU[:v, :], LUo[:v, :])


def test_getrf_lda_larger_than_n(cf):
    n, ld = 333, 400
    A = inputs.uniform_pm1(n, seed=11)
    dA = _dev(A, ld=ld)
    assert dA.stride(1) == ld
    ipiv, info = cf.getrf(dA)
    LU = _host(dA)
    LUo, ipo, _, gaps, _ = oracle.getrf(A, arity=AR)
    assert _pivots_agree(ipiv.cpu().numpy(), ipo, gaps, 128)
    assert oracle.lu_residual(A, LU, ipiv.cpu().numpy()) <= 20.0


def test_getrf_constructed_pivots_gepp_mode(cf):
    """n <= h: the tournament is partial pivoting; constructed A = P^T L U has
    every argmax separated by >= 1e-3, so P is recovered exactly."""
    n = 128
    A, perm, L, U = inputs.constructed_plu(n, seed=5)
    dA = _dev(A)
    ipiv, info = cf.getrf(dA, v=32, leaf_h=128)
    np.testing.assert_array_equal(oracle.perm_from_ipiv(ipiv.cpu().numpy(), n), perm)


def test_getrf_dyadic_exact(cf):
    n = 64
    A, perm, L, U = inputs.dyadic_plu(n, seed=7)
    dA = _dev(A)
    ipiv, info = cf.getrf(dA, v=16, leaf_h=128)
    LU = _host(dA)
    Lg, Ug = oracle.split_lu(LU)
    np.testing.assert_array_equal(Lg, L)
    np.testing.assert_array_equal(Ug, U)


def test_getrf_gap_audited_tournament_identity(cf):
    """Tournament mode (h < n) on seeds whose oracle gaps are all >= 1e-3:
    pivot sequences identical."""
    done = 0
    for seed in range(200):
        n = 96
        A = inputs.uniform_pm1(n, seed=seed)
        LUo, ipo, _, gaps, _ = oracle.getrf(A, v=16, h=8, arity=2)
        if gaps.min() < 1e-3:
            continue
        dA = _dev(A)
        ipiv, info = cf.getrf(dA, v=16, leaf_h=8, arity=2)
        np.testing.assert_array_equal(ipiv.cpu().numpy(), ipo)
        done += 1
        if done >= 3:
            break
    assert done >= 1


def test_getrf_singular_info(cf):
    n = 200
    A = inputs.uniform_pm1(n, seed=5)
    A[:, 150] = 0.0
    dA = _dev(A)
    ipiv, info = cf.getrf(dA)
    _, _, info_o, _, _ = oracle.getrf(A, arity=AR)
    assert int(info.item()) == info_o == 151


def test_getrf_n0_and_workspace_error(cf):
    dA = torch.zeros((0, 0), dtype=torch.float64, device="cuda")
    ipiv, info = cf.getrf(dA)
    assert int(info.item()) == 0
    A = _dev(inputs.uniform_pm1(10, seed=1))
    with pytest.raises(cf.CfError) as e:
        cf.getrf(A, work=torch.empty(1, dtype=torch.uint8, device="cuda"))
    assert e.value.status == cf.CF_ERR_WORKSPACE


# --------------------------------------------------------------- Cholesky
@pytest.mark.parametrize("n,v", [(1, 128), (64, 128), (129, 128), (300, 32), (1000, 128)])
def test_potrf_matches_oracle(cf, n, v):
    S = inputs.spd_gram(n, seed=1)
    dS = _dev(S)
    info = cf.potrf(dS, v=v)
    L = np.tril(_host(dS))
    Lo, info_o, _ = oracle.potrf(S)
    assert int(info.item()) == info_o == 0
    assert np.abs(L - Lo).max() <= 1e-12 * np.abs(Lo).max()
    assert oracle.chol_residual(S, L) <= 20.0


def test_potrf_leaves_upper_triangle(cf):
    n = 200
    S = inputs.spd_gram(n, seed=2)
    S2 = S.copy(order="F")
    iu = np.triu_indices(n, 1)
    S2[iu] = 12345.0
    dS = _dev(S2)
    cf.potrf(dS)
    out = _host(dS)
    assert (out[iu] == 12345.0).all()


def test_potrf_not_spd_info(cf):
    n = 300
    S = inputs.spd_gram(n, seed=1)
    S[200, 200] = -1.0
    dS = _dev(S)
    info = cf.potrf(dS)
    _, info_o, _ = oracle.potrf(S)
    assert int(info.item()) == info_o and info_o > 0


def test_potrf_integer_exact(cf):
    A, L0 = inputs.integer_l0(64, seed=9)
    dA = _dev(A)
    cf.potrf(dA, v=16)
    np.testing.assert_array_equal(np.tril(_host(dA)), L0)


# ------------------------------------------------------------------ solves
def test_getrs_potrs_residual(cf):
    n, nrhs = 700, 5
    A = inputs.uniform_pm1(n, seed=21)
    B = inputs.rhs_normal(n, nrhs, seed=2)
    dA = _dev(A)
    ipiv, info = cf.getrf(dA)
    dB = _dev(B)
    cf.getrs(dA, ipiv, dB)
    X = _host(dB)
    LUo, ipo, _, _, _ = oracle.getrf(A, arity=AR)
    Xo = oracle.getrs(LUo, ipo, B)
    assert oracle.backward_error(A, X, B).max() <= 1e-14
    assert np.abs(X - Xo).max() <= 1e-9 * np.abs(Xo).max()

    S = inputs.spd_gram(n, seed=1)
    dS = _dev(S)
    cf.potrf(dS)
    dB = _dev(B)
    cf.potrs(dS, dB)
    X = _host(dB)
    assert oracle.backward_error(S, X, B).max() <= 1e-14

    # residual kernel against the compensated oracle residual
    dX = _dev(X)
    R = _host(cf.residual(_dev(S), dX, _dev(B)))
    Ro = oracle.residual(S, X, B)
    scale = np.abs(S).sum(axis=1).max() * np.abs(X).max()
    assert np.abs(R - Ro).max() <= 4 * n * oracle.EPS * scale


@pytest.mark.parametrize("nrhs", [1, 3, 8, 16, 20])
def test_residual_shapes(cf, nrhs):
    m, n = 517, 300
    rng = np.random.default_rng(nrhs)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    X = np.asfortranarray(rng.standard_normal((n, nrhs)))
    B = np.asfortranarray(rng.standard_normal((m, nrhs)))
    R = _host(cf.residual(_dev(A), _dev(X), _dev(B)))
    Ro = oracle.residual(A, X, B)
    assert np.abs(R - Ro).max() <= 4 * n * oracle.EPS * np.abs(A).max() * np.abs(X).max() * n ** 0.5


# ---------------------------------------------------- full-size config 1
def test_config_n2048_lu_and_cholesky(cf):
    """N = 2048, uniform[-1,1] seed 0 (LU) and G G^T/N + I seed 1 (Cholesky),
    block size 128: the oracle runs fully."""
    n = 2048
    A = inputs.uniform_pm1(n, seed=0)
    dA = _dev(A)
    ipiv, info = cf.getrf(dA, v=128, leaf_h=128, arity=2)
    LU = _host(dA)
    ip = ipiv.cpu().numpy()
    LUo, ipo, info_o, gaps, _ = oracle.getrf(A, v=128, h=128, arity=2)
    assert int(info.item()) == 0
    assert _pivots_agree(ip, ipo, gaps, 128)
    assert oracle.lu_residual(A, LU, ip) <= 20.0
    S = inputs.spd_gram(n, seed=1)
    dS = _dev(S)
    info = cf.potrf(dS)
    L = np.tril(_host(dS))
    Lo, _, _ = oracle.potrf(S)
    assert int(info.item()) == 0
    assert np.abs(L - Lo).max() <= 1e-12 * np.abs(Lo).max()
    assert oracle.chol_residual(S, L) <= 20.0


def _pair_err(A, X, B, Rp):
    """max over columns of |Rp - R| / (||A||_inf ||x||_inf + ||b||_inf), R the
    oracle's compensated residual."""
    Ro = oracle.residual(A, X, B)
    den = np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0)
    return (np.abs(Rp - Ro).max(0) / den).max()


@pytest.mark.parametrize("m,n,nrhs,ld", [(129, 129, 3, None), (1000, 1000, 8, None), (2000, 2000, 17, None),
                                         (777, 1500, 1, 781), (9728, 600, 16, None), (3000, 257, 5, 3001)])
def test_residual_pair_accuracy(cf, m, n, nrhs, ld):
    """cf_residual_pair (FP32-pipe pair arithmetic) against the compensated
    oracle residual: error below 5e-14 of ||A|| ||x|| + ||b|| on a
    diagonally dominant system whose residual cancels to 1e-12 (the pair's
    floor is ~2^-48 sqrt(chunk) of a chunk's largest partial sums, here set
    by the diagonal term, ~1/12 of the row's norm at n = 2000).  Shapes cover the
    k-split with partial sums (small m), the direct grid (m = 304 row blocks),
    groups of 16 right-hand sides (17), odd leading dimensions and m != n."""
    rng = np.random.default_rng(m + n)
    A = rng.uniform(-1.0, 1.0, (m, n))
    k = min(m, n)
    A[np.arange(k), np.arange(k)] += 2 * np.sqrt(n)
    X = rng.standard_normal((n, nrhs)) * 0.1
    B = A @ X + 1e-12 * rng.standard_normal((m, nrhs))
    Rp = _host(cf.residual_pair(_dev(A, ld), _dev(X), _dev(B)))
    assert _pair_err(A, X, B, Rp) <= 5e-14


def test_residual_pair_scale_invariance(cf):
    """Power-of-two scaling of A and X by 2^-700 and 2^600 (far outside FP32
    range) gives the same error relative to ||A|| ||x||: the kernel scales by
    powers of two before splitting.  Exact zeros and entries far below
    max |a_ij| (dropped below 2^-74 of it) stay within the same bound."""
    n, nrhs = 700, 4
    rng = np.random.default_rng(7)
    A = rng.uniform(-1.0, 1.0, (n, n)) + 2 * np.sqrt(n) * np.eye(n)
    A[:, 5] = 0.0
    A[3, :] *= 1e-30
    X = rng.standard_normal((n, nrhs))
    B = A @ X
    for sa, sx in ((0, 0), (-700, 600), (300, -900)):
        As, Xs, Bs = np.ldexp(A, sa), np.ldexp(X, sx), np.ldexp(B, sa + sx)
        Rp = _host(cf.residual_pair(_dev(As), _dev(Xs), _dev(Bs)))
        assert np.isfinite(Rp).all()
        assert _pair_err(As, Xs, Bs, Rp) <= 5e-14


def test_residual_pair_nonfinite_and_alias(cf):
    """A NaN or inf in A gives NaN in its row only; R may alias B; a zero X
    column gives R = B exactly."""
    n, nrhs = 300, 3
    rng = np.random.default_rng(11)
    A = rng.uniform(-1.0, 1.0, (n, n)) + 20 * np.eye(n)
    A[17, 40] = np.nan
    A[99, 3] = np.inf
    X = rng.standard_normal((n, nrhs))
    X[:, 2] = 0.0
    B = rng.standard_normal((n, nrhs))
    dB = _dev(B)
    cf.residual_pair(_dev(A), _dev(X), dB, R=dB)
    R = _host(dB)
    assert np.isnan(R[17, :2]).all() and np.isnan(R[99, :2]).all()
    ok = np.ones(n, bool)
    ok[[17, 99]] = False
    Ac = A.copy()
    Ac[~ok] = 0.0
    assert _pair_err(Ac[ok], X, B[ok], R[ok]) <= 5e-14
    np.testing.assert_array_equal(R[ok, 2], B[ok, 2])


@pytest.mark.parametrize("n", [1000, 2500])
def test_lookahead_bit_identical(cf, n):
    """LU-6 look-ahead (two streams) computes exactly what the one-stream loop
    computes: the split of each step's update into the next panel's columns
    and the rest does not change any element's sequence of operations."""
    A = inputs.uniform_pm1(n, seed=n)
    S = inputs.spd_gram(n, seed=n + 1)
    out = {}
    for la in (0, 1):
        dA, dS = _dev(A), _dev(S)
        ipiv, info = cf.getrf(dA, lookahead=la)
        info2 = cf.potrf(dS, lookahead=la)
        torch.cuda.synchronize()
        assert int(info.item()) == 0 and int(info2.item()) == 0
        out[la] = (dA.cpu().numpy(), ipiv.cpu().numpy(), np.tril(dS.cpu().numpy()))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


# ------------------------------------------ config 2 (paper-like sizes)
def _projection_lu(A, LU, ip):
    """oracle.lu_random_projection_error for P A = L U on host copies."""
    n = A.shape[0]
    p = oracle.perm_from_ipiv(ip, n)
    Ls = np.tril(LU, -1)
    U = np.triu(LU)
    return oracle.lu_random_projection_error(lambda Z: A[p] @ Z, lambda Z: Ls @ Z + Z, lambda Z: U @ Z, n,
                                             np.linalg.norm(A, "fro"))


def _projection_chol(S, L):
    n = S.shape[0]
    return oracle.lu_random_projection_error(lambda Z: S @ Z, lambda Z: L @ Z, lambda Z: L.T @ Z, n,
                                             np.linalg.norm(S, "fro"))


@pytest.mark.parametrize("n", [8192])
def test_config2_fp64_lu_cholesky(cf, n):
    """The FP64 path at a paper-like size, look-ahead on (LU of U[-1,1] seed 0,
    Cholesky of G G^T / N + I seed 1, one N(0,1) right-hand side seed 2),
    checked on host copies by the oracle: the first panel's pivots equal the
    oracle's selection on the same panel bytes; the probabilistic factorization
    residual max_z ||(P A - L U) z|| / (||A||_F ||z||) over 4 random z is
    <= 20 n u (stated as such: the full ||P A - L U|| is O(n^3) on the host at
    this size); eta of the getrs / potrs solution by the oracle's compensated
    residual is <= 20 n u."""
    A = inputs.uniform_pm1(n, seed=0)
    b = inputs.rhs_normal(n, 1, seed=2)
    dA = _dev(A)
    win, _ = oracle.tourn_select(A[:, :128], h=128, arity=AR)
    ipiv, info = cf.getrf(dA, lookahead=1)
    db = _dev(b)
    cf.getrs(dA, ipiv, db)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    LU, ip, x = _host(dA), ipiv.cpu().numpy(), _host(db)
    del dA
    # LAPACK interchanges of step 0 from the oracle's winners (original panel
    # rows in pivot order): winner j moves from its current position q to j
    at, where = np.arange(n), np.arange(n)     # row at each position, and its inverse
    ip0 = np.zeros(128, dtype=np.int64)
    for j, r in enumerate(win):
        q = where[r]
        ip0[j] = q + 1
        rj = at[j]
        at[j], at[q] = r, rj
        where[r], where[rj] = j, q
    np.testing.assert_array_equal(ip[:128], ip0)
    bound = 20 * n * oracle.EPS
    assert _projection_lu(A, LU, ip) <= bound
    assert oracle.backward_error(A, x, b).max() <= bound
    del LU

    S = inputs.spd_gram(n, seed=1)
    dS = _dev(S)
    info = cf.potrf(dS, lookahead=1)
    db = _dev(b)
    cf.potrs(dS, db)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    L = np.tril(_host(dS))
    del dS
    assert _projection_chol(S, L) <= bound
    assert oracle.backward_error(S, _host(db), b).max() <= bound
