"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function include/cf.h declares, and its host-side logic (options, status
strings, workspace sizes, argument validation) behaves without a GPU.  No
call here reaches a kernel."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_09337_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _header_functions():
    import re
    txt = open(os.path.join(ROOT, "include", "cf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cf_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_function(lib):
    names = _header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_default_options_and_status_strings(lib):
    from paper_2108_09337_gb300 import cf
    o = cf.options()
    # v, leaf_h and arity are left 0: each routine takes its own default
    assert (o.v, o.leaf_h, o.arity, o.lookahead, o.max_iter) == (0, 0, 0, 1, 30)
    assert o.tol == 1e-14
    lib.cf_status_string.restype = ctypes.c_char_p
    assert lib.cf_status_string(0) == b"ok"
    assert b"workspace" in lib.cf_status_string(-101)
    assert b"invalid" in lib.cf_status_string(-3)


def test_workspace_sizes_are_host_only(lib):
    from paper_2108_09337_gb300 import cf
    L = cf.lib()
    o = cf.options()
    s1 = L.cf_getrf_workspace_size(2048, ctypes.byref(o))
    s2 = L.cf_getrf_workspace_size(32768, ctypes.byref(o))
    assert 0 < s1 < s2 < 64 << 20
    assert L.cf_getrs_workspace_size(1000, 4) >= 1000 * 4 * 8 + 4000
    bad = cf.options(v=200)
    assert L.cf_getrf_workspace_size(100, ctypes.byref(bad)) == 0


def test_noalloc_scratch_limit(lib):
    """cf_getrf_noalloc keeps the tournament scratch in a fixed 2 MiB array:
    the sizes include/cf.h promises fit (n up to 393216 with leaf_h = 128 and
    arity 8, 196608 with leaf_h = 64; 131072 and 65536 with arity 2), the
    scratch grows with n, and a far larger request does not fit (the entry
    point refuses it with CF_ERR_WORKSPACE)."""
    from paper_2108_09337_gb300 import cf
    L = cf.lib()
    L.cf_getrf_workspace_size.restype = ctypes.c_size_t
    limit = 2 << 20
    for leaf_h, arity, n_max in ((128, 8, 393216), (64, 8, 196608), (128, 2, 131072), (64, 2, 65536)):
        o = cf.options(leaf_h=leaf_h, arity=arity)
        sizes = [L.cf_getrf_workspace_size(n, ctypes.byref(o)) for n in (1024, n_max // 4, n_max)]
        assert 0 < sizes[0] <= sizes[1] <= sizes[2] <= limit, (leaf_h, arity, sizes)
        assert L.cf_getrf_workspace_size(4 * n_max, ctypes.byref(o)) > limit


def test_argument_validation_returns_before_any_cuda_call(lib):
    from paper_2108_09337_gb300 import cf
    L = cf.lib()
    null = ctypes.c_void_p(0)
    # negative n -> -1 ; lda too small -> -3
    assert L.cf_getrf(-1, null, 1, null, null, null, 0, None, null) == -1
    assert L.cf_getrf(10, ctypes.c_void_p(16), 5, ctypes.c_void_p(16), ctypes.c_void_p(16), null, 0,
                      None, null) == -3
    assert L.cf_potrf(-2, null, 1, null, null, 0, None, null) == -1
    assert L.cf_tourn_select(10, 200, ctypes.c_void_p(16), 10, 128, 2, null, null, 0, null) == -2
    assert L.cf_tourn_select(10, 4, ctypes.c_void_p(16), 10, 0, 2, null, null, 0, null) == -5
    assert L.cf_tourn_select(10, 4, ctypes.c_void_p(16), 10, 8, 9, null, null, 0, null) == -6
    assert L.cf_residual(-1, 1, 1, null, 1, null, 1, null, 1, null, 1, null) == -1
    assert L.cf_getrs(4, 1, ctypes.c_void_p(16), 2, null, null, 4, null, 0, null) == -4


def test_mixed_options_and_workspace(lib):
    """The refinement options and workspace queries of the mixed solvers:
    fp64_residual takes 0 or 1 and residual_kind 0 or 2 (anything else is
    refused by the size query, which returns 0); by default the residuals run
    on the tensor cores, whose digit slices of A (8 n^2 BF16) the workspace
    holds, and fp64_residual = 1 or residual_kind = 2 drop them; deeper
    slabs from n = 16384 make the workspace grow, and the pair-residual query
    is host-only and linear in m + n."""
    from paper_2108_09337_gb300 import cf
    L = cf.lib()
    o = cf.options()
    assert o.fp64_residual == 0 and o.residual_kind == 0
    n = 4096
    tc = cf.gesv_mixed_workspace_size(n, 4, "f16")
    ok = cf.gesv_mixed_workspace_size(n, 4, "f16", residual_kind=2)
    assert ok > 0 and tc - ok >= 16 * n * n
    assert cf.gesv_mixed_workspace_size(n, 4, "f16", fp64_residual=1) == ok
    assert cf.gesv_mixed_workspace_size(n, 4, "f16", fp64_residual=2) == 0
    assert cf.gesv_mixed_workspace_size(n, 4, "f16", residual_kind=1) == 0
    assert cf.posv_mixed_workspace_size(n, 4, "f16", fp64_residual=-1) == 0
    kw = dict(residual_kind=2)
    for fn in (cf.gesv_mixed_workspace_size, cf.posv_mixed_workspace_size):
        # slabs of V = 2048 from n = 16384 (Lb / Ub hold 3 V columns of each row)
        deep = fn(16384, 16, "f16", **kw)
        assert deep == fn(16384, 16, "f16", outer_V=2048, **kw)
        assert deep - fn(16384, 16, "f16", outer_V=1024, **kw) >= 2 * 3 * 1024 * 16384 * 2
    p1 = L.cf_residual_pair_workspace_size(1000, 1000, 16)
    p2 = L.cf_residual_pair_workspace_size(2000, 2000, 16)
    assert 0 < p1 < p2 <= 2 * p1 + 4096


def test_generic_workspace_query_matches_each_call(lib):
    """cf_workspace_size(op, ...) equals the per-call queries."""
    from paper_2108_09337_gb300 import cf
    L = cf.lib()
    o = cf.options()
    ob = ctypes.byref(o)
    W = cf.workspace_size
    assert W("getrf", 4096) == L.cf_getrf_workspace_size(4096, ob) > 0
    assert W("getrf", 4096, leaf_h=64) == L.cf_getrf_workspace_size(4096, ctypes.byref(cf.options(leaf_h=64)))
    assert W("potrf", 4096) == L.cf_potrf_workspace_size(4096, ob)
    assert W("getrs", 1000, 4) == L.cf_getrs_workspace_size(1000, 4) > 0
    assert W("potrs", 1000, 4) == 0
    for prec in ("bf16", "f16", "bf16x3"):
        assert W("gesv_mixed", 4096, 16, prec) == cf.gesv_mixed_workspace_size(4096, 16, prec) > 0
        assert W("posv_mixed", 4096, 8, prec) == cf.posv_mixed_workspace_size(4096, 8, prec) > 0
    assert W("posv_mixed", 8192, 8, "fp8") == cf.posv_mixed_workspace_size(8192, 8, "fp8") > 0
    assert W("getrf_batched", 2000) == L.cf_getrf_batched_workspace_size(2000, ob) > 0
    assert W("potrf_batched", 2000) == L.cf_potrf_batched_workspace_size(2000, ob)
    assert W("factor_batched", 2000) == L.cf_factor_batched_workspace_size(2000, ob)
    assert W("solve_batched_mixed", 2000) == L.cf_solve_batched_mixed_workspace_size(2000, ob) > 0
    assert W("residual_pair", 3000, 16) == L.cf_residual_pair_workspace_size(3000, 3000, 16) > 0
    assert W("tourn_select", 5000, 128) == L.cf_tourn_workspace_size(5000, 128, 128, 8) > 0   # default arity 8
    assert L.cf_workspace_size(99, 100, 1, 0, None) == 0
    assert L.cf_workspace_size(0, -1, 0, 0, None) == 0
    assert W("getrf", 100, v=200) == 0


def test_noalloc_scratch_limit_matches_documented_sizes(lib):
    """cf_getrf_noalloc keeps its scratch in a fixed 2 MiB array and needs
    exactly cf_getrf's workspace: with the default arity 8, n = 393216 fits
    with leaf_h = 128 and 196608 with leaf_h = 64, 524288 and 262144 do not;
    with arity 2, 131072 (leaf_h = 128) and 65536 (leaf_h = 64) fit and twice
    those sizes do not."""
    from paper_2108_09337_gb300 import cf
    lib.cf_getrf_workspace_size.restype = ctypes.c_size_t
    lib.cf_getrf_workspace_size.argtypes = [ctypes.c_int, ctypes.c_void_p]
    limit = 2 << 20

    def need(n, h, arity=None):
        o = cf.options(leaf_h=h, arity=arity)
        return lib.cf_getrf_workspace_size(n, ctypes.cast(ctypes.byref(o), ctypes.c_void_p))

    assert 0 < need(393216, 128) <= limit
    assert need(524288, 128) > limit
    assert 0 < need(196608, 64) <= limit
    assert need(262144, 64) > limit
    assert 0 < need(131072, 128, 2) <= limit
    assert need(262144, 128, 2) > limit
    assert 0 < need(65536, 64, 2) <= limit
    assert need(131072, 64, 2) > limit
