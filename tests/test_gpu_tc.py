"""GPU checks of the tensor-core Schur update C -= A B^T (tcgen05, TMA,
TMEM) through cf_schur_update_lp.

Reference: the same BF16/FP16 operands widened to FP64 on the host, C - A B^T
in FP64 (a plain definition of the operation).  Bound per entry: the FP32
accumulation of k products and the final FP32 subtraction,
|err| <= 2 (k + 2) 2^-24 (|A| |B|^T + |C|).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    assert torch.cuda.is_available()
    from paper_2108_09337_gb300 import cf as _cf
    return _cf


def _run(cf, m, n, k, dtype, lower=False, ldc_pad=0, seed=0):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn((m, k), generator=g).to(dtype)
    B = torch.randn((n, k), generator=g).to(dtype)
    C = torch.randn((m, n), generator=g, dtype=torch.float32)
    dC = torch.zeros((n, m + ldc_pad), dtype=torch.float32)
    dC[:, :m] = C.t()
    dC = dC.cuda().t()[:m, :]
    cf.schur_update_lp(A.cuda(), B.cuda(), dC, lower=lower)
    assert cf.device_status() == 0
    got = dC.cpu().double().numpy()
    Ad, Bd, Cd = A.double().numpy(), B.double().numpy(), C.double().numpy()
    ref = Cd - Ad @ Bd.T
    bound = 2 * (k + 2) * 2.0 ** -24 * (np.abs(Ad) @ np.abs(Bd).T + np.abs(Cd))
    if lower:
        il = np.tril(np.ones((m, n), dtype=bool))
        assert np.all(np.abs(got - ref)[il] <= bound[il])
        assert np.array_equal(got[~il], Cd[~il])      # upper part untouched
    else:
        assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (128, 256, 128), (256, 512, 64), (300, 500, 192),
                                   (1, 1, 64), (129, 257, 64), (1000, 700, 1024), (4096, 4096, 128)])
def test_schur_update_bf16(cf, m, n, k):
    _run(cf, m, n, k, torch.bfloat16, seed=m + n + k)


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (333, 777, 256)])
def test_schur_update_fp16(cf, m, n, k):
    _run(cf, m, n, k, torch.float16, seed=k)


@pytest.mark.parametrize("m,k", [(128, 64), (600, 128), (1000, 256)])
def test_schur_update_lower(cf, m, k):
    _run(cf, m, m, k, torch.bfloat16, lower=True, seed=m)


def test_schur_update_ldc(cf):
    _run(cf, 200, 300, 128, torch.bfloat16, ldc_pad=40)


def test_schur_update_many_tiles_persistent(cf):
    """More tiles than SMs: every CTA walks several tiles and reuses both
    TMEM accumulators."""
    _run(cf, 2048, 8192, 128, torch.bfloat16, seed=5)


def test_schur_update_slab_depth(cf):
    """The mixed LU's K = V slab update at its timed depth, M = N = 8192,
    K = 2048 (FP16 operands, 0.6 GB with C): 4096 sampled entries against the
    FP64 product of the same operands, within the FP32-accumulation bound."""
    m = n = 8192
    k = 2048
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn((m, k), generator=g, device="cuda").to(torch.float16)
    B = torch.randn((n, k), generator=g, device="cuda").to(torch.float16)
    C0 = torch.randn((n, m), generator=g, device="cuda", dtype=torch.float32).t()
    C = C0.clone().t().contiguous().t()
    cf.schur_update_lp(A, B, C)
    assert cf.device_status() == 0
    rng = np.random.default_rng(3)
    ii, jj = rng.integers(0, m, 4096), rng.integers(0, n, 4096)
    Ad = A[torch.from_numpy(ii).cuda()].double().cpu().numpy()
    Bd = B[torch.from_numpy(jj).cuda()].double().cpu().numpy()
    c0 = C0[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].double().cpu().numpy()
    got = C[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].double().cpu().numpy()
    ref = c0 - np.einsum("ik,ik->i", Ad, Bd)
    bound = 2 * (k + 2) * 2.0 ** -24 * (np.einsum("ik,ik->i", np.abs(Ad), np.abs(Bd)) + np.abs(c0))
    assert np.all(np.abs(got - ref) <= bound)


def _run_splitk(cf, m, n, k, ksplit, lower=False, seed=0):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn((m, k), generator=g).to(torch.bfloat16)
    B = torch.randn((n, k), generator=g).to(torch.bfloat16)
    C = torch.randn((m, n), generator=g, dtype=torch.float32)
    outs = []
    for _ in range(2):
        dC = C.t().contiguous().cuda().t()
        cf.schur_update_lp_splitk(A.cuda(), B.cuda(), dC, ksplit, lower=lower)
        assert cf.device_status() == 0
        outs.append(dC.cpu().double().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])             # deterministic
    got = outs[0]
    Ad, Bd, Cd = A.double().numpy(), B.double().numpy(), C.double().numpy()
    ref = Cd - Ad @ Bd.T
    # ksplit FP32 partial sums of k / ksplit products, added in FP32, then subtracted
    bound = 2 * (k + ksplit + 2) * 2.0 ** -24 * (np.abs(Ad) @ np.abs(Bd).T + np.abs(Cd))
    if lower:
        il = np.tril(np.ones((m, n), dtype=bool))
        assert np.all(np.abs(got - ref)[il] <= bound[il])
        assert np.array_equal(got[~il], Cd[~il])
    else:
        assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("m,n,k,ksplit,lower", [(256, 256, 2048, 4, False), (300, 500, 1024, 3, False),
                                                (1000, 700, 4096, 8, False), (129, 257, 640, 16, False),
                                                (512, 512, 2048, 6, True), (1000, 1000, 1024, 2, True),
                                                (64, 64, 128, 1, False)])
def test_schur_update_splitk(cf, m, n, k, ksplit, lower):
    """Split-K (K cut into ksplit ranges run as separate work units, partials
    added in range order): within the FP32 bound of the FP64 product,
    bit-identical over two calls, the strict upper triangle untouched in the
    lower form; more ranges than K blocks are merged (640 = 10 blocks, 16
    ranges asked)."""
    _run_splitk(cf, m, n, k, ksplit, lower=lower, seed=m + k)
