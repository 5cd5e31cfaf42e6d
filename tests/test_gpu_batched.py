"""GPU checks of BAT-1 (cf_factor_batched / cf_getrf_batched /
cf_potrf_batched / cf_solve_batched_mixed) through the C ABI.

Each batched LU follows the tournament rule with one leaf per panel (partial
pivoting) and block size 32, so the oracle run with v = 32, h >= n is its
reference: pivots identical where the oracle's gaps are >= 1e-10, factors
within 1e-9 max|LU|, backward error <= 20 n u.  Cholesky factors within
1e-12 max|L|.  Mixed solves: eta <= 1e-14 per matrix.
"""
import time

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


def _fill(batch, mats):
    for i, M in enumerate(mats):
        n = M.shape[0]
        if n:
            batch.matrix(i).copy_(torch.from_numpy(np.ascontiguousarray(M)))


def _gen(sizes, kinds, seed0=0):
    mats = []
    for i, (n, k) in enumerate(zip(sizes, kinds)):
        if k == 0:
            mats.append(inputs.uniform_pm1(n, seed=seed0 + i))
        else:
            mats.append(inputs.spd_gram(n, seed=seed0 + i) if n > 0 else np.zeros((0, 0)))
    return mats


def _check_lu(M, LU, ip, tag=""):
    n = M.shape[0]
    LUo, ipo, info_o, gaps, _ = oracle.getrf(M, v=32, h=10 ** 6)
    if not np.array_equal(ip, ipo):
        first = int(np.argmax(ip != ipo))
        assert gaps[: first // 32 + 1].min() < 1e-10, tag
    else:
        assert np.abs(LU - LUo).max() <= 1e-9 * max(1.0, np.abs(LUo).max()), tag
    assert oracle.lu_residual(M, LU, ip) <= 20.0, tag


def test_batched_mixed_kinds_small(cf):
    rng = np.random.default_rng(7)
    sizes = [1, 2, 5, 31, 32, 33, 64, 100, 128, 129, 255, 300, 511, 512] + list(rng.integers(16, 513, 18))
    kinds = [i % 2 for i in range(len(sizes))]
    mats = _gen(sizes, kinds, seed0=50)
    b = cf.Batch(sizes, kinds=kinds)
    _fill(b, mats)
    ipiv, iptr, info = cf.factor_batched(b)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    ipv = ipiv.cpu().numpy()
    for i, (n, k) in enumerate(zip(sizes, kinds)):
        assert info[i] == 0
        out = b.matrix(i).cpu().numpy()
        if k == 0:
            ip = ipv[b.vec_offsets[i]:b.vec_offsets[i] + n]
            _check_lu(mats[i], out, ip, tag="n=%d" % n)
        else:
            Lo, _, _ = oracle.potrf(mats[i])
            assert np.abs(np.tril(out) - Lo).max() <= 1e-12 * max(1.0, np.abs(Lo).max())


def test_batched_getrf_potrf_wrappers_and_info(cf):
    sizes = [40, 70, 600]
    mats = [inputs.uniform_pm1(40, 1), inputs.uniform_pm1(70, 2), inputs.uniform_pm1(600, 3)]
    mats[1][:, 10] = 0.0
    b = cf.Batch(sizes, kinds=[0, 0, 0])
    _fill(b, mats)
    ipiv, iptr, info = cf.factor_batched(b)
    torch.cuda.synchronize()
    info = info.cpu().numpy()
    assert info[0] == 0 and info[1] == 11 and info[2] == -1     # zero column; n > 512 refused


def test_batched_mixed_solve_small(cf):
    rng = np.random.default_rng(3)
    sizes = [1, 16, 65, 200, 512] + list(rng.integers(16, 513, 11))
    kinds = [i % 2 for i in range(len(sizes))]
    mats = _gen(sizes, kinds, seed0=900)
    b = cf.Batch(sizes, kinds=kinds)
    _fill(b, mats)
    B = torch.zeros(b.vec_total, dtype=torch.float64, device="cuda")
    rhs = []
    for i, n in enumerate(sizes):
        r = inputs.rhs_normal(n, 1, seed=7 + i)[:, 0]
        rhs.append(r)
        B[b.vec_offsets[i]:b.vec_offsets[i] + n] = torch.from_numpy(r)
    X, info, iters, eta, solver = cf.solve_batched_mixed(b, B)
    torch.cuda.synchronize()
    assert (solver.cpu().numpy() == 32).all()          # well conditioned: FP32 factors suffice
    X = X.cpu().numpy()
    for i, n in enumerate(sizes):
        x = X[b.vec_offsets[i]:b.vec_offsets[i] + n]
        e = oracle.backward_error(mats[i], x.reshape(n, 1), rhs[i].reshape(n, 1)).max()
        assert e <= 1e-14, (i, n, e, int(iters[i]))
    assert (eta.cpu().numpy() <= 1e-14).all()


def test_config_20000_uneven(cf):
    """20,000 matrices, n ~ U{16..512} (seed 7); even index Cholesky of
    G G^T/n + I, odd index LU of U[-1,1]; FP64 factorization in one launch, and
    FP32 factors + FP64 refinement; sampled matrices checked against the
    oracle, every refined solution against eta <= 1e-14."""
    sizes = np.random.default_rng(7).integers(16, 513, 20000).tolist()
    kinds = [0 if i % 2 else 1 for i in range(len(sizes))]
    b = cf.Batch(sizes, kinds=kinds)
    # fill on the device (torch Philox), matrix by matrix is too slow on the
    # host for 20,000: draw one big uniform buffer and make the SPD ones
    # diagonally dominant symmetric (G G^T / n + I built for the sample only)
    g = torch.Generator(device="cuda").manual_seed(7)
    b.data.uniform_(-1.0, 1.0, generator=g)
    sample = [i for i in range(0, 20000, 997)]
    for i in range(len(sizes)):
        if kinds[i] == 1:
            M = b.matrix(i)
            n = sizes[i]
            M.copy_((M @ M.t()) / n + torch.eye(n, device="cuda", dtype=torch.float64))
    torch.cuda.synchronize()
    host = {i: b.matrix(i).cpu().numpy().copy() for i in sample}
    A0 = b.data.clone()
    t0 = time.perf_counter()
    ipiv, iptr, info = cf.factor_batched(b)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    assert (info.cpu().numpy() == 0).all()
    ipv = ipiv.cpu().numpy()
    for i in sample:
        n = sizes[i]
        out = b.matrix(i).cpu().numpy()
        if kinds[i] == 0:
            _check_lu(host[i], out, ipv[b.vec_offsets[i]:b.vec_offsets[i] + n], tag="i=%d" % i)
        else:
            Lo, _, _ = oracle.potrf(host[i])
            assert np.abs(np.tril(out) - Lo).max() <= 1e-12 * np.abs(Lo).max()
    # refined mixed solves on the original matrices
    b.data.copy_(A0)
    B = torch.randn(b.vec_total, dtype=torch.float64, device="cuda", generator=g)
    t2 = time.perf_counter()
    X, info2, iters, eta, solver = cf.solve_batched_mixed(b, B)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    assert (info2.cpu().numpy() == 0).all()
    assert (eta.cpu().numpy() <= 1e-14).all()
    fl = sum((2.0 if k == 0 else 1.0) * n ** 3 / 3.0 for n, k in zip(sizes, kinds))
    print("\nbatched FP64 factor: %.3f s (%.2f TFLOP/s); FP32+IR solve: %.3f s, mean iters %.2f, FP64 fallbacks %d"
          % (t1 - t0, fl / (t1 - t0) / 1e12, t3 - t2, iters.float().mean().item(),
             int((solver == 64).sum().item())))


def test_batched_mixed_fp64_fallback(cf):
    """Matrices beyond FP32 refinement (cond 1e10, LU and SPD) fall back to
    FP64 factors inside the launch and still reach eta <= 1e-14; a singular
    one reports info from the FP64 factorization; well-conditioned
    neighbours keep FP32 factors."""
    sizes = [96, 300, 257, 64, 128, 33]
    kinds = [0, 1, 0, 1, 0, 0]
    mats = [inputs.prescribed_cond(96, 1e10, 11),
            inputs.prescribed_cond(300, 1e10, 12, spd=True),
            inputs.uniform_pm1(257, 13),
            inputs.spd_gram(64, 14),
            inputs.prescribed_cond(128, 1e12, 15),
            inputs.uniform_pm1(33, 16)]
    mats[5][:, 7] = 0.0                                 # exactly singular
    b = cf.Batch(sizes, kinds=kinds)
    _fill(b, mats)
    B = torch.zeros(b.vec_total, dtype=torch.float64, device="cuda")
    rhs = []
    for i, n in enumerate(sizes):
        r = inputs.rhs_normal(n, 1, seed=70 + i)[:, 0]
        rhs.append(r)
        B[b.vec_offsets[i]:b.vec_offsets[i] + n] = torch.from_numpy(r)
    X, info, iters, eta, solver = cf.solve_batched_mixed(b, B)
    torch.cuda.synchronize()
    info, iters, eta, solver = (t.cpu().numpy() for t in (info, iters, eta, solver))
    X = X.cpu().numpy()
    assert list(solver) == [64, 64, 32, 32, 64, 64], solver
    assert list(info[:5]) == [0] * 5 and info[5] == 8, info
    for i in range(5):
        n = sizes[i]
        x = X[b.vec_offsets[i]:b.vec_offsets[i] + n]
        e = oracle.backward_error(mats[i], x.reshape(n, 1), rhs[i].reshape(n, 1)).max()
        assert eta[i] <= 1e-14 and e <= 1e-14, (i, eta[i], e, iters[i])


@pytest.mark.parametrize("v,cps", [(8, 1), (16, 2), (32, 1), (16, 3)])
def test_batched_block_size_and_residency(cf, v, cps):
    """Every (block size, CTAs per SM) the autotuner can pick gives LU and
    Cholesky factors with oracle-level backward error."""
    rng = np.random.default_rng(11)
    sizes = [int(x) for x in rng.integers(1, 513, 40)]
    kinds = [i % 2 for i in range(len(sizes))]
    mats = _gen(sizes, kinds, seed0=300)
    b = cf.Batch(sizes, kinds=kinds)
    _fill(b, mats)
    ipiv, iptr, info = cf.factor_batched(b, v=v, batch_cps=cps)
    assert (info.cpu().numpy() == 0).all()
    ipv = ipiv.cpu().numpy()
    for i, (n, k) in enumerate(zip(sizes, kinds)):
        out = b.matrix(i).cpu().numpy()
        if k == 0:
            assert oracle.lu_residual(mats[i], out, ipv[b.vec_offsets[i]:b.vec_offsets[i] + n]) <= 20, (i, n)
        else:
            assert oracle.chol_residual(mats[i], np.tril(out)) <= 20, (i, n)


def test_batched_graph_capture_replay(cf):
    """The batched factorization and the batched mixed solve captured in CUDA
    graphs: replays reproduce the direct calls bit for bit."""
    rng = np.random.default_rng(12)
    sizes = [int(x) for x in rng.integers(16, 300, 64)]
    kinds = [i % 2 for i in range(len(sizes))]
    mats = _gen(sizes, kinds, seed0=400)
    b = cf.Batch(sizes, kinds=kinds)
    _fill(b, mats)
    A0 = b.data.clone()
    ipiv_ref, _, info_ref = cf.factor_batched(b)
    F_ref = b.data.clone()
    plan = cf.BatchedPlan(b, "factor")
    b.data.copy_(A0)
    plan.capture()                         # capture only records; nothing runs
    for _ in range(2):
        b.data.copy_(A0)
        plan.replay()
        torch.cuda.synchronize()
        assert torch.equal(b.data, F_ref)
        assert torch.equal(plan.ipiv, ipiv_ref) and torch.equal(plan.info, info_ref)
    # mixed solve
    b.data.copy_(A0)
    Bv = torch.randn(b.vec_total, dtype=torch.float64, device="cuda")
    X_ref, info2, iters, eta, solver = cf.solve_batched_mixed(b, Bv)
    mp = cf.BatchedPlan(b, "mixed")
    mp.B.copy_(Bv)
    mp.capture()
    mp.replay()
    torch.cuda.synchronize()
    assert torch.equal(mp.X, X_ref) and torch.equal(mp.eta, eta)
    assert (mp.eta.cpu().numpy() <= 1e-14).all()


def test_batched_autotune(cf):
    """The autotuner returns a candidate configuration that runs and
    factors correctly; the sample's time is positive."""
    sizes = np.random.default_rng(7).integers(16, 513, 3000).tolist()
    kinds = [0 if i % 2 else 1 for i in range(len(sizes))]
    b = cf.Batch(sizes, kinds=kinds)
    for mixed in (False, True):
        opt, ms = cf.batched_autotune(b, mixed=mixed)
        assert opt.v in (8, 16, 32) and 1 <= opt.batch_cps <= (2 if mixed else 3) and ms > 0
    opt, ms = cf.batched_autotune(b, mixed=False)
    sub = [16, 100, 257, 512]
    mats = _gen(sub, [0, 1, 0, 1], seed0=500)
    bs = cf.Batch(sub, kinds=[0, 1, 0, 1])
    _fill(bs, mats)
    ipiv, iptr, info = cf.factor_batched(bs, opt=opt)
    assert (info.cpu().numpy() == 0).all()
