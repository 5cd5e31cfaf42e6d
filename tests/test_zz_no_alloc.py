"""cf_getrf_noalloc: the LU for callers that cannot allocate device memory
(for example code running under stream capture, or a plugin inside a
framework that owns all device memory).  It keeps its tournament scratch in
a fixed array inside the library, so these tests check, through the C ABI,
that it returns what cf_getrf returns with a caller-provided work buffer, on
two calls in a row (the second call reuses the array the first one left
behind), that both agree with the CPU oracle's LU, that a call captured
into a CUDA graph and replayed gives the same factors and pivots, and that
a request too large for the array is refused.

Tolerance: the same as the other LU parity tests (pivots identical to the
oracle's except after a step where the oracle logged an argmax gap below
1e-10, factors within 1e-9 max|LU|, ||PA - LU||_1 / (n u ||A||_1) <= 20);
the two entry points run the same kernels in the same order, so against each
other the results are bit-identical.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2108_09337_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


@pytest.fixture(scope="module")
def cf():
    assert torch.cuda.is_available()
    from paper_2108_09337_gb300 import cf as _cf
    return _cf


@pytest.mark.parametrize("call", [0, 1])
def test_noalloc_matches_getrf_two_calls(cf, call):
    results = []
    for n, seed in ((700, 11), (1029, 12)):       # two calls in a row
        A = inputs.uniform_pm1(n, seed=seed + call)
        dA_ref = _dev(A)
        ipiv_ref, info_ref = cf.getrf(dA_ref)
        dA = _dev(A)
        ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        cf.getrf_noalloc(dA, ipiv=ipiv, info=info)
        torch.cuda.synchronize()
        ip = ipiv.cpu().numpy()
        np.testing.assert_array_equal(ip, ipiv_ref.cpu().numpy())
        assert int(info.item()) == int(info_ref.item()) == 0
        LU, LUr = dA.cpu().numpy(), dA_ref.cpu().numpy()
        np.testing.assert_array_equal(LU, LUr)
        # against the oracle (same v, leaf height and arity as the defaults)
        LUo, ipo, info_o, gaps, _ = oracle.getrf(A, v=128, h=128, arity=8)   # the FP64 defaults
        assert info_o == 0
        div = np.nonzero(ip != ipo)[0]
        if div.size:
            assert gaps[div[0] // 128] < 1e-10, "pivots differ from the oracle at row %d" % div[0]
        else:
            assert np.abs(LU - LUo).max() <= 1e-9 * np.abs(LUo).max()
        assert oracle.lu_residual(A, LU, ip) <= 20.0
        results.append(n)
    assert results == [700, 1029]


def test_noalloc_captured_in_cuda_graph(cf):
    """The case the entry point exists for: one warm-up call, then the call
    captured into a CUDA graph (stream capture refuses device allocations)
    and replayed twice on fresh copies of A; each replay's pivots, info and
    factors equal cf_getrf's with a work buffer."""
    n = 700
    A = inputs.uniform_pm1(n, seed=21)
    dA_ref = _dev(A)
    ipiv_ref, info_ref = cf.getrf(dA_ref)
    A0 = _dev(A)
    dA = _dev(A)
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    cf.getrf_noalloc(dA, ipiv=ipiv, info=info)           # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cf.getrf_noalloc(dA, ipiv=ipiv, info=info)
    torch.cuda.synchronize()
    for _ in range(2):
        dA.copy_(A0)
        ipiv.fill_(-1)
        info.fill_(-1)                                   # the call itself resets info to 0
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ipiv.cpu().numpy(), ipiv_ref.cpu().numpy())
        assert int(info.item()) == int(info_ref.item()) == 0
        np.testing.assert_array_equal(dA.cpu().numpy(), dA_ref.cpu().numpy())


def test_noalloc_rejects_oversized_request(cf):
    n = 1 << 20                                   # needs far more than the fixed array
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    ip = torch.zeros(4, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    opt = cf.options()
    st = cf.lib().cf_getrf_noalloc(n, ctypes.c_void_p(dummy.data_ptr()), n, ctypes.c_void_p(ip.data_ptr()),
                                   ctypes.c_void_p(info.data_ptr()), ctypes.byref(opt),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == cf.CF_ERR_WORKSPACE
