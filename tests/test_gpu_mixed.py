"""GPU checks of the mixed-precision refined solves through the C ABI
(cf_gesv_mixed, cf_posv_mixed): BF16 / FP16 tensor-core Schur updates on FP32
working storage, FP64 refinement.

Bar: backward error eta = max_j ||b_j - A x_j||_inf /
(||A||_inf ||x_j||_inf + ||b_j||_inf) <= 1e-14, computed here on the host by
the oracle's compensated residual from the returned x; the forward error
against the oracle's FP64 solution is bounded by kappa_inf(A) * eta * 4.
A and B must come back unchanged.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_09337_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    assert torch.cuda.is_available()
    from paper_2108_09337_gb300 import cf as _cf
    return _cf


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


def _check_solution(A, B, X, eta_tol=1e-14):
    eta = oracle.backward_error(A, X, B).max()
    assert eta <= eta_tol, eta
    Xs = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A, np.inf)
    fwd = np.abs(X - Xs).max() / np.abs(Xs).max()
    assert fwd <= 4 * kappa * max(eta, 1e-16) + 1e-13
    return eta


@pytest.mark.parametrize("v", [None, 128])       # None: the default (v = 64, wide tournament)
@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("n,nrhs,V", [(1, 1, 0), (37, 2, 0), (129, 3, 0), (512, 16, 256), (1000, 4, 256),
                                      (2048, 16, 0)])
def test_gesv_mixed_well_conditioned(cf, prec, n, nrhs, V, v):
    A = inputs.uniform_pm1(n, seed=0, shift=2 * np.sqrt(n))
    B = inputs.rhs_normal(n, nrhs, seed=3)
    dA, dB = _dev(A), _dev(B)
    X, info, stats, st = cf.gesv_mixed(dA, dB, prec=prec, outer_V=V, v=v)
    assert st == cf.CF_OK, stats.as_dict()
    assert int(info.item()) == 0 and stats.converged == 1
    np.testing.assert_array_equal(dA.cpu().numpy(), A)
    np.testing.assert_array_equal(dB.cpu().numpy(), B)
    _check_solution(A, B, X.cpu().numpy())
    assert stats.iterations <= 20


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("n,nrhs,V", [(1, 1, 0), (300, 2, 128), (1024, 8, 256), (2048, 8, 0)])
def test_posv_mixed(cf, prec, n, nrhs, V):
    S = inputs.spd_gram(n, seed=1)
    B = inputs.rhs_normal(n, nrhs, seed=4)
    dS, dB = _dev(S), _dev(B)
    X, info, stats, st = cf.posv_mixed(dS, dB, prec=prec, outer_V=V)
    assert st == cf.CF_OK, stats.as_dict()
    assert stats.converged == 1
    np.testing.assert_array_equal(dS.cpu().numpy(), S)
    _check_solution(S, B, X.cpu().numpy())


def test_gesv_mixed_unshifted_uniform_small(cf):
    """s = 0 (kappa ~ 1e3 at n = 256): FP16 factors still let classical
    refinement converge."""
    n = 256
    A = inputs.uniform_pm1(n, seed=0)
    B = inputs.rhs_normal(n, 2, seed=3)
    X, info, stats, st = cf.gesv_mixed(_dev(A), _dev(B), prec="f16")
    assert st == cf.CF_OK, stats.as_dict()
    _check_solution(A, B, X.cpu().numpy())


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_gesv_mixed_unshifted_uniform_gmres(cf, prec):
    """s = 0 at n = 2048 (kappa_inf ~ 1e5): classical refinement with BF16
    factors cannot contract (kappa u_f >> 1), so the solver must hand over to
    GMRES-IR and still reach eta <= 1e-14 with all 16 right-hand sides."""
    n = 2048
    A = inputs.uniform_pm1(n, seed=0)
    B = inputs.rhs_normal(n, 16, seed=3)
    X, info, stats, st = cf.gesv_mixed(_dev(A), _dev(B), prec=prec)
    d = stats.as_dict()
    assert st == cf.CF_OK, d
    assert d["converged"] == 1
    if prec == "bf16":
        assert d["solver"] == 1 and d["gmres_iterations"] > 0, d
    _check_solution(A, B, X.cpu().numpy())


@pytest.mark.parametrize("spd", [False, True])
def test_mixed_prescribed_condition(cf, spd):
    """Haar-random A with geometrically spaced singular values, kappa_2 =
    1e4 (n = 512), FP16 factors: refinement (classical, then GMRES-IR if
    needed) reaches eta <= 1e-14.  (BF16 factors leave kappa(M^{-1} A) ~ 1e4
    on this spectrum and restarted GMRES stagnates: a CPU emulation of the
    same algorithm stalls near eta ~ 2e-4, so that case is not asked for.)"""
    n = 512
    A = inputs.prescribed_cond(n, 1e4, seed=21, spd=spd)
    B = inputs.rhs_normal(n, 4, seed=5)
    fn = cf.posv_mixed if spd else cf.gesv_mixed
    X, info, stats, st = fn(_dev(A), _dev(B), prec="f16")
    d = stats.as_dict()
    assert st == cf.CF_OK, d
    _check_solution(A, B, X.cpu().numpy())


def test_gesv_mixed_not_converged_returns_best(cf):
    """An unreachable tolerance (1e-30): the call reports
    CF_ERR_NOT_CONVERGED after max_iter steps (or two failed GMRES-IR steps)
    and hands back the iterate with the smallest backward error seen, which
    is at the FP64 floor here."""
    n = 256
    A = inputs.uniform_pm1(n, seed=4, shift=2 * np.sqrt(n))
    B = inputs.rhs_normal(n, 2, seed=6)
    X, info, stats, st = cf.gesv_mixed(_dev(A), _dev(B), prec="bf16", tol=1e-30, max_iter=8)
    assert st == cf.CF_ERR_NOT_CONVERGED and stats.converged == 0
    Xh = X.cpu().numpy()
    assert np.isfinite(Xh).all()
    eta = oracle.backward_error(A, Xh, B).max()
    assert stats.eta <= 1e-15 and eta <= 2 * stats.eta + 1e-16, (eta, stats.as_dict())


@pytest.mark.parametrize("n,nrhs,V", [(1, 1, 0), (300, 2, 128), (1024, 8, 256), (2048, 8, 0)])
def test_posv_mixed_fp8(cf, n, nrhs, V):
    """FP8 e4m3 trailing updates with per-tile scales: refinement (classical,
    GMRES-IR once that stalls, a diagonal shift on breakdown) reaches
    eta <= 1e-14."""
    S = inputs.spd_gram(n, seed=1)
    B = inputs.rhs_normal(n, nrhs, seed=4)
    dS, dB = _dev(S), _dev(B)
    X, info, stats, st = cf.posv_mixed(dS, dB, prec="fp8", outer_V=V)
    assert st == cf.CF_OK, stats.as_dict()
    np.testing.assert_array_equal(dS.cpu().numpy(), S)
    _check_solution(S, B, X.cpu().numpy())


@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_posv_mixed_fp8_conditioned(cf, kappa):
    """The N = 65536 configuration's matrix family at n = 2048:
    A = G G^T / n + alpha I with alpha = lambda_max / (kappa - 1)
    (lambda_max of G G^T / n from the dense eigensolver), 8 right-hand sides,
    FP8 updates."""
    n = 2048
    S0 = inputs.spd_gram(n, seed=1, alpha=0.0)
    lam = np.linalg.eigvalsh(S0)[-1]
    S = S0 + (lam / (kappa - 1.0)) * np.eye(n)
    B = inputs.rhs_normal(n, 8, seed=4)
    X, info, stats, st = cf.posv_mixed(_dev(S), _dev(B), prec="fp8")
    assert st == cf.CF_OK, stats.as_dict()
    _check_solution(S, B, X.cpu().numpy())


@pytest.mark.parametrize("which", ["gesv_shifted", "gesv_s0", "posv"])
def test_mixed_split_bf16(cf, which):
    """CF_BF16X3 (split BF16 updates, hi.hi + hi.lo + lo.hi): converges on the
    well-conditioned and the unshifted (s = 0) LU matrices and on the SPD one."""
    n = 1500
    if which == "posv":
        A = inputs.spd_gram(n, seed=1)
    else:
        A = inputs.uniform_pm1(n, seed=0, shift=(2 * np.sqrt(n) if which == "gesv_shifted" else 0.0))
    B = inputs.rhs_normal(n, 3, seed=3)
    fn = cf.posv_mixed if which == "posv" else cf.gesv_mixed
    X, info, stats, st = fn(_dev(A), _dev(B), prec="bf16x3")
    assert st == cf.CF_OK, stats.as_dict()
    assert stats.escalated == 0
    _check_solution(A, B, X.cpu().numpy())


def test_gesv_mixed_escalates_to_split(cf):
    """s = 0 at n = 8192 with BF16 factors: GMRES-IR stalls (kappa(M^-1 A)
    too large), the solver refactors with split BF16 updates and converges."""
    n = 8192
    A = inputs.uniform_pm1(n, seed=0)
    B = inputs.rhs_normal(n, 4, seed=3)
    X, info, stats, st = cf.gesv_mixed(_dev(A), _dev(B), prec="bf16")
    d = stats.as_dict()
    assert st == cf.CF_OK, d
    assert d["escalated"] == 1, d
    eta = oracle.backward_error(A, X.cpu().numpy(), B).max()
    assert eta <= 1e-14, (eta, d)


def test_gesv_mixed_fp8_refused(cf):
    A = _dev(inputs.uniform_pm1(64, seed=1, shift=16.0))
    B = _dev(inputs.rhs_normal(64, 1))
    with pytest.raises(cf.CfError) as e:
        cf.gesv_mixed(A, B, prec="fp8")
    assert e.value.status == -9


def test_gesv_mixed_workspace_error(cf):
    A = _dev(inputs.uniform_pm1(64, seed=1, shift=16.0))
    B = _dev(inputs.rhs_normal(64, 1))
    with pytest.raises(cf.CfError) as e:
        cf.gesv_mixed(A, B, work=torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert e.value.status == cf.CF_ERR_WORKSPACE


# ---------------------------------------------------------- LU-1 in FP32
@pytest.mark.parametrize("m,w,h,arity", [(128, 128, 128, 2), (1000, 128, 128, 2), (777, 100, 50, 2),
                                         (5000, 128, 256, 2), (300, 17, 128, 2), (50, 128, 128, 2),
                                         (256, 128, 256, 2), (32768, 128, 128, 2),
                                         (32768, 128, 256, 2)])
def test_tourn_select_f32_gap_audited(cf, m, w, h, arity):
    """FP32 panel values (exact in FP64): where the FP64 oracle's gaps are all
    >= 1e-3 the FP32 elimination must pick the same rows in the same order;
    otherwise the selection must still be min(m, w) distinct rows."""
    P = inputs.uniform_pm1(m, seed=m + 7 * w, m=w).astype(np.float32).astype(np.float64)
    win_o, gap = oracle.tourn_select(P, h=h, arity=arity)
    dP = torch.from_numpy(np.ascontiguousarray(P.T.astype(np.float32))).cuda().t()
    win = cf.tourn_select(dP, leaf_h=h, arity=arity).cpu().numpy()
    assert len(win) == min(m, w) and len(set(win.tolist())) == len(win)
    assert win.min() >= 0 and win.max() < m
    if gap >= 1e-3:
        np.testing.assert_array_equal(win, win_o)


# The wide-node FP32 tournament (panels of <= 64 columns: leaves of up to 512
# rows, arity up to 8).  Random panels whose FP64-oracle gaps are all >= 1e-3
# (seeds found by a CPU search of inputs.uniform_pm1(m, seed=1000 s + m + 7 w,
# m=w)), which exercise the elimination arithmetic at every node.
@pytest.mark.parametrize("m,w,h,arity,s", [(512, 64, 512, 8, 7), (513, 64, 512, 8, 2), (1024, 64, 512, 2, 27),
                                           (1100, 64, 512, 3, 100), (700, 64, 100, 4, 149),
                                           (2048, 32, 256, 8, 46)])
def test_tourn_select_f32_wide_gap_audited(cf, m, w, h, arity, s):
    P = inputs.uniform_pm1(m, seed=1000 * s + m + 7 * w, m=w).astype(np.float32).astype(np.float64)
    win_o, gap = oracle.tourn_select(P, h=h, arity=arity)
    assert gap >= 1e-3
    dP = torch.from_numpy(np.ascontiguousarray(P.T.astype(np.float32))).cuda().t()
    win = cf.tourn_select(dP, leaf_h=h, arity=arity).cpu().numpy()
    np.testing.assert_array_equal(win, win_o)


@pytest.mark.parametrize("m,w,h,arity", [(32768, 64, 512, 8), (40000, 64, 512, 8), (32768, 64, 256, 4),
                                         (6400, 64, 512, 5), (4096, 64, 128, 4), (2048, 16, 256, 8),
                                         (32768, 64, 512, 2)])
def test_tourn_select_f32_wide_typed_panels(cf, m, w, h, arity):
    """Up to 40000 rows (79 leaves of 512, three playoff levels at arity 8,
    the last leaf 64 rows) on panels built so that every argmax is separated
    by 0.4% (inputs.typed_panel, audited by the oracle's gap log): the FP32
    selection must equal the oracle's."""
    P = inputs.typed_panel(m, w, seed=m + arity)
    win_o, gap = oracle.tourn_select(P, h=h, arity=arity)
    assert gap >= 1e-3
    dP = torch.from_numpy(np.ascontiguousarray(P.T.astype(np.float32))).cuda().t()
    win = cf.tourn_select(dP, leaf_h=h, arity=arity).cpu().numpy()
    np.testing.assert_array_equal(win, win_o)


@pytest.mark.parametrize("m,w,h,arity", [(32768, 64, 512, 8), (9999, 61, 333, 7), (300, 64, 512, 8),
                                         (5000, 1, 512, 8), (64, 64, 512, 8)])
def test_tourn_select_f32_wide_valid(cf, m, w, h, arity):
    """Random panels (gaps below 1e-3 somewhere): min(m, w) distinct rows."""
    P = inputs.uniform_pm1(m, seed=m + w, m=w)
    dP = torch.from_numpy(np.ascontiguousarray(P.T.astype(np.float32))).cuda().t()
    win = cf.tourn_select(dP, leaf_h=h, arity=arity).cpu().numpy()
    assert len(win) == min(m, w) and len(set(win.tolist())) == len(win)
    assert win.min() >= 0 and win.max() < m
    if m <= h:                       # a single leaf: GEPP; its first pivot is the column maximum
        P32 = np.abs(P[:, 0].astype(np.float32))
        assert P32[win[0]] == P32.max()


def test_tourn_select_f32_wide_ties_zeros_nan(cf):
    """The wide kernel on exact-arithmetic panels with ties, zero columns and
    a NaN (as below, at arity 5 and 8 and leaves of 100 / 512 rows)."""
    P = np.zeros((1300, 8))
    P[::3, :] = 1.0
    P[7, 0] = -1.0
    P[5, 0] = np.nan
    P[900, 3] = 2.0
    dP = torch.from_numpy(np.ascontiguousarray(P.T.astype(np.float32))).cuda().t()
    for h, arity in ((100, 5), (512, 8), (16, 8)):
        win_o, _ = oracle.tourn_select(P, h=h, arity=arity)
        win = cf.tourn_select(dP, leaf_h=h, arity=arity).cpu().numpy()
        np.testing.assert_array_equal(win, win_o)


def test_tourn_select_f32_ties_zeros_nan(cf):
    """Exact ties (ties to the smallest stacked row), zero columns and a NaN
    (ranks below every number) in FP32, with values whose elimination is
    exact, so the pivots must equal the oracle's."""
    P = np.zeros((300, 8))
    P[::3, :] = 1.0
    P[7, 0] = -1.0
    P[5, 0] = np.nan
    win_o, _ = oracle.tourn_select(P, h=16, arity=2)
    dP = torch.from_numpy(np.ascontiguousarray(P.T.astype(np.float32))).cuda().t()
    for h in (16, 256):
        win_o, _ = oracle.tourn_select(P, h=h, arity=2)
        win = cf.tourn_select(dP, leaf_h=h, arity=2).cpu().numpy()
        np.testing.assert_array_equal(win, win_o)


def test_tourn_select_f32_constructed_gepp(cf):
    """Single leaf (GEPP mode) on a constructed P^T L U: pivots are P."""
    n = 128
    A, perm, L, U = inputs.constructed_plu(n, seed=3)
    dP = torch.from_numpy(np.ascontiguousarray(A.T.astype(np.float32))).cuda().t()
    win = cf.tourn_select(dP, leaf_h=128, arity=2).cpu().numpy()
    # GEPP on the first w columns selects perm[0..w) in order
    np.testing.assert_array_equal(win, perm[:n])


@pytest.mark.parametrize("solver", ["gesv", "posv"])
def test_residual_policies(cf, solver):
    """The three residual policies of the refinement: by default every
    residual runs on the tensor cores (digit slices of A; no FP64 or pair
    product); residual_kind = 2 takes the early residuals in pair arithmetic
    and decides convergence on an FP64 one; fp64_residual = 1 takes all of
    them in FP64.  All reach eta <= 1e-14 checked on the host, and the
    answers agree to the refinement's accuracy."""
    n, nrhs = 2048, 4
    A = inputs.uniform_pm1(n, seed=2, shift=2 * np.sqrt(n)) if solver == "gesv" else inputs.spd_gram(n, seed=2)
    B = inputs.rhs_normal(n, nrhs, seed=5)
    fn = cf.gesv_mixed if solver == "gesv" else cf.posv_mixed
    out = {}
    for name, kw in (("tc", {}), ("pair", {"residual_kind": 2}), ("f64", {"fp64_residual": 1})):
        X, info, stats, st = fn(_dev(A), _dev(B), prec="f16", **kw)
        assert st == cf.CF_OK, stats.as_dict()
        out[name] = X.cpu().numpy()
        _check_solution(A, B, out[name])
        d = stats.as_dict()
        if name == "tc":
            assert d["tc_launches"] >= 1 and d["pair_launches"] == 0 and d["residual_launches"] == 0, d
        elif name == "pair":
            assert d["pair_launches"] >= 1 and d["residual_launches"] >= 1 and d["tc_launches"] == 0, d
        else:
            assert d["pair_launches"] == 0 and d["residual_launches"] >= 1 and d["tc_launches"] == 0, d
    Xs = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A, np.inf)
    for a in ("tc", "pair"):
        assert np.abs(out[a] - out["f64"]).max() / np.abs(Xs).max() <= 8 * kappa * 1e-14


@pytest.mark.parametrize("v", [None, 128])
@pytest.mark.parametrize("prec", ["f16", "bf16x3"])
def test_gesv_mixed_deep_slab(cf, prec, v):
    """Slabs of V = 2048 (the LU default from n = 16384 on) at a size the host
    check affords: two slabs, the second ragged (4500 = 2048 + 2048 + 404),
    left-looking pivot-row updates with K up to 1920, split-BF16 operands
    with three K segments of 2048."""
    n = 4500
    A = inputs.uniform_pm1(n, seed=9, shift=2 * np.sqrt(n))
    B = inputs.rhs_normal(n, 3, seed=10)
    X, info, stats, st = cf.gesv_mixed(_dev(A), _dev(B), prec=prec, outer_V=2048, v=v)
    assert st == cf.CF_OK, stats.as_dict()
    _check_solution(A, B, X.cpu().numpy())


WIDE = dict(v=64, leaf_h=512, arity=8)


@pytest.mark.parametrize("prec,n,V,shift", [("f16", 2048, 0, True), ("bf16", 1000, 256, True),
                                            ("f16", 777, 128, True), ("bf16x3", 4500, 2048, True),
                                            ("f16", 4500, 2048, True), ("bf16x3", 2048, 0, False),
                                            ("f16", 65, 64, True)])
def test_gesv_mixed_wide_tournament(cf, prec, n, V, shift):
    """The mixed LU at block size v = 64 with the wide-node tournament (leaves
    of 512 rows, arity 8): shifted and unshifted uniform matrices (the
    unshifted one hands over to GMRES-IR), deep and ragged slabs, reach
    eta <= 1e-14; A and B come back unchanged."""
    A = inputs.uniform_pm1(n, seed=n + 1, shift=2 * np.sqrt(n) if shift else 0.0)
    B = inputs.rhs_normal(n, 5, seed=6)
    dA, dB = _dev(A), _dev(B)
    X, info, stats, st = cf.gesv_mixed(dA, dB, prec=prec, outer_V=V, **WIDE)
    assert st == cf.CF_OK and int(info.item()) == 0, stats.as_dict()
    np.testing.assert_array_equal(dA.cpu().numpy(), A)
    np.testing.assert_array_equal(dB.cpu().numpy(), B)
    _check_solution(A, B, X.cpu().numpy())


@pytest.mark.parametrize("prec,n,V,v", [("f16", 2048, 0, None), ("bf16x3", 4500, 2048, None), ("f16", 3000, 1024, 128)])
def test_gesv_mixed_lookahead_identical(cf, prec, n, V, v):
    """LU-6 look-ahead in the mixed LU (the rest of each step's in-slab
    update on a second stream beside the next TournPivot) computes exactly
    what the one-stream schedule computes: the solutions agree bit for bit
    (so do the pivots and factors they come from), and reach eta <= 1e-14."""
    A = inputs.uniform_pm1(n, seed=n + 3)
    B = inputs.rhs_normal(n, 4, seed=9)
    out = {}
    for la in (0, 1):
        X, info, stats, st = cf.gesv_mixed(_dev(A), _dev(B), prec=prec, outer_V=V, v=v, lookahead=la)
        assert st == cf.CF_OK and int(info.item()) == 0, stats.as_dict()
        out[la] = (X.cpu().numpy(), stats.iterations, stats.gmres_iterations)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]
    _check_solution(A, B, out[1][0])


@pytest.mark.parametrize("prec,n,V", [("bf16x3", 2048, 0), ("f16", 3000, 1024), ("bf16", 1000, 256)])
def test_posv_mixed_lookahead_identical(cf, prec, n, V):
    """LU-6 in the mixed Cholesky (the rest of each step's in-slab update on a
    second stream beside the next A00 Cholesky) gives bit-identical solutions."""
    S = inputs.spd_gram(n, seed=n)
    B = inputs.rhs_normal(n, 3, seed=2)
    out = {}
    for la in (0, 1):
        X, info, stats, st = cf.posv_mixed(_dev(S), _dev(B), prec=prec, outer_V=V, lookahead=la)
        assert st == cf.CF_OK and int(info.item()) == 0, stats.as_dict()
        out[la] = X.cpu().numpy()
    np.testing.assert_array_equal(out[0], out[1])
    _check_solution(S, B, out[1])


def test_gesv_mixed_shape_checks(cf):
    """Tournament shapes the mixed LU cannot run are refused before any work
    (v = 128 takes arity 2 and leaves <= 256; v <= 64 takes arity * v <= 512)."""
    A = _dev(inputs.uniform_pm1(64, seed=1, shift=16.0))
    B = _dev(inputs.rhs_normal(64, 1))
    for kw in (dict(v=128, arity=3), dict(v=128, leaf_h=512), dict(v=64, arity=8, leaf_h=513),
               dict(v=96, arity=2, leaf_h=300)):
        with pytest.raises(cf.CfError) as e:
            cf.gesv_mixed(A, B, **kw)
        assert e.value.status == cf.CF_ERR_UNSUPPORTED, kw
    assert cf.gesv_mixed_workspace_size(64, 1, "f16", v=128, arity=3) == 0
    assert cf.gesv_mixed_workspace_size(64, 1, "f16", **WIDE) > 0


@pytest.mark.parametrize("solver", ["gesv", "posv"])
def test_mixed_solve_full_size(cf, solver):
    """The benchmark's systems at N = 32768 in the launch configuration it
    times (LU: A = U[-1,1] + 2 sqrt(N) I, 16 right-hand sides, FP16 updates,
    v = 64 with leaves of 512 rows and arity 8; Cholesky: A = G G^T / N + I, 8 right-hand sides,
    split-BF16 updates; alpha = lambda_max / (kappa - 1) for kappa = 1e2, as
    the benchmark sets it): the oracle's compensated residual over every row
    of a host copy gives eta <= 1e-14."""
    n = 32768
    if solver == "gesv":
        dA = inputs.uniform_pm1_torch(n, seed=0, shift=2.0 * np.sqrt(n), device="cuda")
        dB = inputs.rhs_normal_torch(n, 16, seed=3, device="cuda")
        X, info, stats, st = cf.gesv_mixed(dA, dB, prec="f16", v=64, leaf_h=512, arity=8)
    else:
        dA = inputs.spd_gram_torch(n, seed=1, alpha=0.0, device="cuda")
        inputs.shift_to_kappa_torch(dA, 1e2)
        dB = inputs.rhs_normal_torch(n, 8, seed=4, device="cuda")
        X, info, stats, st = cf.posv_mixed(dA, dB, prec="bf16x3")
    torch.cuda.synchronize()
    assert st == cf.CF_OK and int(info.item()) == 0, stats.as_dict()
    A = dA.t().cpu().numpy().T                  # column-major host copy, no second copy
    del dA
    torch.cuda.empty_cache()
    eta = oracle.backward_error(A, X.cpu().numpy(), dB.cpu().numpy()).max()
    assert eta <= 1e-14, eta
