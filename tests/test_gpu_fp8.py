"""GPU checks of the FP8 e4m3 building blocks (cf_quantize_e4m3,
cf_schur_update_fp8) through the C ABI.

Quantization: per 128 x 128 tile the scale equals amax / 448 computed in
FP32, and every code equals torch's round-to-nearest-even float8_e4m3fn
conversion of x * (448 / amax) (an implementation independent of ours);
decoded codes times the scale reproduce x within the e4m3 unit roundoff
2^-4 (relative) or the smallest subnormal step.
Update: against the FP64 sum over K-blocks of sA sB (decoded qA)(decoded qB)^T,
with the FP32 accumulation bound (k + 2) 2^-24 (|A||B|^T + |C|) per entry.
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


def _colmajor(x):
    return x.t().contiguous().t()


def _decode(q):
    return q.view(torch.float8_e4m3fn).to(torch.float64)


@pytest.mark.parametrize("rows,k", [(128, 128), (300, 200), (1, 5), (1000, 384)])
def test_quantize_matches_torch_e4m3(cf, rows, k):
    g = torch.Generator(device="cuda").manual_seed(rows + k)
    src = _colmajor(torch.randn(rows, k, device="cuda", generator=g, dtype=torch.float32) *
                    torch.logspace(-3, 2, k, device="cuda"))
    src[0, 0] = 0.0
    q, sc = cf.quantize_e4m3(src)
    torch.cuda.synchronize()
    kpad = q.shape[1]
    assert (q[:, k:] == 0).all()
    for rb in range((rows + 127) // 128):
        for kb in range(kpad // 128):
            t = src[rb * 128:(rb + 1) * 128, kb * 128:min((kb + 1) * 128, k)]
            if t.numel() == 0:
                continue
            # IEEE FP32 arithmetic on the host (numpy), conversion by torch on the CPU
            th = t.cpu().numpy().astype(np.float32)
            amax = np.float32(np.abs(th).max())
            exp_scale = amax / np.float32(448.0) if amax > 0 else np.float32(1.0)
            assert np.float32(sc[rb, kb].item()) == exp_scale
            inv = np.float32(448.0) / amax if amax > 0 else np.float32(1.0)
            ref = torch.from_numpy((th * inv).astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8)
            got = q[rb * 128:(rb + 1) * 128, kb * 128:kb * 128 + t.shape[1]].cpu()
            assert torch.equal(got, ref)
            dec = _decode(got) * float(sc[rb, kb])
            err = (dec - torch.from_numpy(th).double()).abs()
            assert (err <= 2.0 ** -4 * torch.from_numpy(th).double().abs() + 2.0 ** -9 * float(sc[rb, kb])).all()


@pytest.mark.parametrize("m,n,k,lower", [(128, 256, 128, False), (300, 520, 384, False), (1000, 777, 1024, False),
                                         (640, 640, 256, True), (129, 129, 128, True)])
def test_schur_update_fp8_against_fp64(cf, m, n, k, lower):
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n + k)
    A = _colmajor(torch.randn(m, k, device="cuda", generator=g) * (1.0 + torch.arange(k, device="cuda") / 64.0))
    B = A if lower and m == n else _colmajor(torch.randn(n, k, device="cuda", generator=g))
    qA, sA = cf.quantize_e4m3(A)
    qB, sB = (qA, sA) if B is A else cf.quantize_e4m3(B)
    C0 = _colmajor(torch.randn(m, n, device="cuda", generator=g))
    C = C0.clone()
    C = _colmajor(C)
    cf.schur_update_fp8(qA, sA, qB, sB, C, lower=lower)
    assert cf.device_status() == cf.CF_OK
    # FP64 reference from the same codes and scales
    rowsA = torch.arange(m, device="cuda") // 128
    rowsB = torch.arange(n, device="cuda") // 128
    Ad = torch.zeros(m, k, dtype=torch.float64, device="cuda")
    Bd = torch.zeros(n, k, dtype=torch.float64, device="cuda")
    ref = C0.double().clone()
    bound = C0.double().abs().clone()
    for kb in range(k // 128):
        sl = slice(kb * 128, (kb + 1) * 128)
        a = _decode(qA[:, sl]) * sA[rowsA, kb].double()[:, None]
        b = _decode(qB[:, sl]) * sB[rowsB, kb].double()[:, None]
        ref -= a @ b.t()
        bound += a.abs() @ b.abs().t()
    tol = (k + 2) * 2.0 ** -24 * bound
    got = C.double()
    diff = (got - ref).abs()
    if lower:
        mask = torch.ones(m, n, dtype=torch.bool, device="cuda").tril()
        assert (diff[mask] <= tol[mask]).all(), diff.max()
        assert torch.equal(got[~mask], C0.double()[~mask])     # strictly upper untouched
    else:
        assert (diff <= tol).all(), (diff / tol).max()
