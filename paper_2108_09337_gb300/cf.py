"""ctypes binding of libcf (include/cf.h): argument marshalling only.

Every computation happens in libcf's CUDA kernels; torch provides device
memory and the current stream.  Matrices are column-major torch tensors:
an m x n matrix is a tensor of shape (m, n) with stride (1, ld), ld >= m
(e.g. ``fortran_empty(m, n)`` or ``t.t().contiguous().t()``).

Importing this module loads libcf.so and raises if it is missing: there is no
CPU or PyTorch fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcf.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "cf.h")

if not os.path.exists(LIB_PATH):
    raise ImportError("libcf.so is not built (run __graft_entry__.build() or "
                      "python -m paper_2108_09337_gb300.build)")
_lib = ctypes.CDLL(LIB_PATH)

CF_OK = 0
CF_ERR_CUDA = -100
CF_ERR_WORKSPACE = -101
CF_ERR_NOT_CONVERGED = -102
CF_ERR_TIMEOUT = -103
CF_ERR_UNSUPPORTED = -104
CF_F64, CF_F32, CF_BF16, CF_F16, CF_FP8E4M3, CF_BF16X3 = range(6)
PREC = {"f64": CF_F64, "f32": CF_F32, "bf16": CF_BF16, "f16": CF_F16,
        "fp8": CF_FP8E4M3, "fp8e4m3": CF_FP8E4M3, "bf16x3": CF_BF16X3}


class Options(ctypes.Structure):
    _fields_ = [("v", ctypes.c_int), ("leaf_h", ctypes.c_int), ("arity", ctypes.c_int),
                ("outer_V", ctypes.c_int), ("lookahead", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("gmres_restart", ctypes.c_int), ("batch_cps", ctypes.c_int),
                ("fp64_residual", ctypes.c_int), ("residual_kind", ctypes.c_int)]


class RefineStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("solver", ctypes.c_int), ("converged", ctypes.c_int),
                ("info", ctypes.c_int), ("eta", ctypes.c_double), ("eta0", ctypes.c_double),
                ("shift", ctypes.c_double), ("factor_ms", ctypes.c_double),
                ("refine_ms", ctypes.c_double), ("residual_ms", ctypes.c_double),
                ("update_ms", ctypes.c_double), ("update_flops", ctypes.c_double),
                ("residual_launches", ctypes.c_int), ("update_launches", ctypes.c_int),
                ("gmres_iterations", ctypes.c_int), ("escalated", ctypes.c_int),
                ("pair_ms", ctypes.c_double), ("pair_launches", ctypes.c_int),
                ("tourn_ms", ctypes.c_double), ("tourn_launches", ctypes.c_int), ("tourn_flops", ctypes.c_double),
                ("tc_ms", ctypes.c_double), ("tc_launches", ctypes.c_int), ("tc_prep_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_I, _P, _S, _D = ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_double
_OPT = ctypes.POINTER(Options)
_SIG = {
    "cf_default_options": (None, [_OPT]),
    "cf_status_string": (ctypes.c_char_p, [_I]),
    "cf_workspace_size": (_S, [_I, _I, _I, _I, _OPT]),
    "cf_last_cuda_error": (_I, []),
    "cf_kernel_launches": (ctypes.c_longlong, []),
    "cf_tourn_workspace_size": (_S, [_I, _I, _I, _I]),
    "cf_tourn_select": (_I, [_I, _I, _P, _I, _I, _I, _P, _P, _S, _P]),
    "cf_tourn_select_f32": (_I, [_I, _I, _P, _I, _I, _I, _P, _P, _S, _P]),
    "cf_getrf_workspace_size": (_S, [_I, _OPT]),
    "cf_getrf": (_I, [_I, _P, _I, _P, _P, _P, _S, _OPT, _P]),
    "cf_getrf_noalloc": (_I, [_I, _P, _I, _P, _P, _OPT, _P]),
    "cf_potrf_workspace_size": (_S, [_I, _OPT]),
    "cf_potrf": (_I, [_I, _P, _I, _P, _P, _S, _OPT, _P]),
    "cf_getrs_workspace_size": (_S, [_I, _I]),
    "cf_getrs": (_I, [_I, _I, _P, _I, _P, _P, _I, _P, _S, _P]),
    "cf_potrs": (_I, [_I, _I, _P, _I, _P, _I, _P]),
    "cf_residual": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P]),
    "cf_residual_pair_workspace_size": (_S, [_I, _I, _I]),
    "cf_residual_tc_workspace_size": (_S, [_I, _I, _I]),
    "cf_residual_tc": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _S, _P]),
    "cf_residual_pair": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _S, _P]),
    "cf_schur_update_lp": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _I, _I, _P]),
    "cf_schur_update_lp_splitk_workspace_size": (_S, [_I, _I, _I, _I]),
    "cf_schur_update_lp_splitk": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _I, _I, _I, _P, _S, _P]),
    "cf_device_status": (_I, [_P]),
    "cf_trsv_f32_workspace_size": (_S, [_I]),
    "cf_trsv_f32": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _S, _P]),
    "cf_trsv_f32_withheld": (_I, [_I, _I, _I, _P, _I, _P, _I, ctypes.c_longlong, _P, _S, _P]),
    "cf_factor_batched_workspace_size": (_S, [_I, _OPT]),
    "cf_factor_batched": (_I, [_I, _P, _I, _P, _P, _P, _P, _P, _P, _S, _OPT, _P]),
    "cf_getrf_batched_workspace_size": (_S, [_I, _OPT]),
    "cf_getrf_batched": (_I, [_I, _P, _P, _P, _P, _P, _P, _S, _OPT, _P]),
    "cf_potrf_batched_workspace_size": (_S, [_I, _OPT]),
    "cf_potrf_batched": (_I, [_I, _P, _P, _P, _P, _P, _S, _OPT, _P]),
    "cf_solve_batched_mixed_workspace_size": (_S, [_I, _OPT]),
    "cf_batched_autotune_workspace_size": (_S, [_I, _P, _P, _I, _I]),
    "cf_batched_autotune": (_I, [_I, _P, _P, _I, _I, _P, _S, _OPT, ctypes.POINTER(ctypes.c_float), _P]),
    "cf_solve_batched_mixed": (_I, [_I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _S, _OPT, _P]),
    "cf_quantize_e4m3": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _P]),
    "cf_schur_update_fp8": (_I, [_I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _I, _I, _P]),
    "cf_gesv_mixed_workspace_size": (_S, [_I, _I, _I, _OPT]),
    "cf_gesv_mixed": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _I, _P, ctypes.POINTER(RefineStats),
                           _P, _S, _OPT, _P]),
    "cf_posv_mixed_workspace_size": (_S, [_I, _I, _I, _OPT]),
    "cf_posv_mixed": (_I, [_I, _I, _P, _I, _P, _I, _P, _I, _I, _P, ctypes.POINTER(RefineStats),
                           _P, _S, _OPT, _P]),
}
for _name, (_res, _args) in _SIG.items():
    if hasattr(_lib, _name):
        _f = getattr(_lib, _name)
        _f.restype = _res
        _f.argtypes = _args


def header_functions(path: str = HEADER):
    """Names of the functions include/cf.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cf_[a-z0-9_]+)\s*\(", txt)))


class CfError(RuntimeError):
    def __init__(self, fn, status):
        msg = _lib.cf_status_string(status).decode()
        if status == CF_ERR_CUDA:
            msg += " (cudaError %d)" % _lib.cf_last_cuda_error()
        super().__init__("%s returned %d: %s" % (fn, status, msg))
        self.status = status


def _check(fn, st):
    if st != CF_OK:
        raise CfError(fn, st)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _ld(t: torch.Tensor, name: str) -> int:
    """Leading dimension of a column-major CUDA tensor (checked)."""
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dim() == 1:
        if t.shape[0] > 1 and t.stride(0) != 1:
            raise ValueError("%s must be contiguous" % name)
        return max(t.shape[0], 1)
    if t.dim() != 2:
        raise ValueError("%s must be 1-D or 2-D" % name)
    m, n = t.shape
    if m > 1 and t.stride(0) != 1:
        raise ValueError("%s must be column-major (stride (1, ld))" % name)
    if n > 1:
        if t.stride(1) < m:
            raise ValueError("%s: leading dimension below the row count" % name)
        return max(t.stride(1), 1)
    return max(m, 1)


def fortran_empty(m: int, n: int, dtype=torch.float64, device="cuda"):
    return torch.empty((n, m), dtype=dtype, device=device).t()


def to_fortran(t: torch.Tensor) -> torch.Tensor:
    return t.t().contiguous().t()


def options(**kw) -> Options:
    o = Options()
    _lib.cf_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


OPS = {name: i for i, name in enumerate(
    ["getrf", "potrf", "getrs", "potrs", "gesv_mixed", "posv_mixed", "getrf_batched", "potrf_batched",
     "factor_batched", "solve_batched_mixed", "residual_pair", "tourn_select"])}


def workspace_size(op: str, n: int, nrhs: int = 0, prec="f64", **opt_kw) -> int:
    """cf_workspace_size: bytes of work the call `op` needs (n = order, or
    batch size for the batched calls, or panel rows for tourn_select; nrhs =
    right-hand sides, or the panel width for tourn_select)."""
    opt = options(**opt_kw)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    return _lib.cf_workspace_size(OPS[op], n, nrhs, p, ctypes.byref(opt))


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# --------------------------------------------------------------------------
def tourn_select(panel: torch.Tensor, leaf_h: int = 128, arity: int = 2) -> torch.Tensor:
    """TournPivot on a column-major FP64 (cf_tourn_select) or FP32
    (cf_tourn_select_f32) panel; returns the winners' row indices."""
    assert panel.dtype in (torch.float64, torch.float32)
    m, w = panel.shape
    ld = _ld(panel, "panel")
    win = torch.empty(max(min(m, w), 1), dtype=torch.int32, device=panel.device)
    ws = _workspace(_lib.cf_tourn_workspace_size(m, w, leaf_h, arity), panel.device)
    fn, name = ((_lib.cf_tourn_select, "cf_tourn_select") if panel.dtype == torch.float64
                else (_lib.cf_tourn_select_f32, "cf_tourn_select_f32"))
    _check(name, fn(m, w, _ptr(panel), ld, leaf_h, arity, _ptr(win), _ptr(ws), ws.numel(), _stream()))
    return win[:min(m, w)]


def getrf(A: torch.Tensor, v=None, leaf_h=None, arity=None, work=None, lookahead=None):
    """In-place LU with tournament pivoting.  Returns (ipiv, info) device
    int32 tensors (ipiv 1-based).  lookahead: 1 (default) overlaps step
    t+1's TournPivot with step t's trailing update, 0 keeps one stream."""
    assert A.dtype == torch.float64
    n = A.shape[0]
    assert A.shape == (n, n)
    lda = _ld(A, "A")
    opt = options(v=v, leaf_h=leaf_h, arity=arity, lookahead=lookahead)
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    need = _lib.cf_getrf_workspace_size(n, ctypes.byref(opt))
    ws = work if work is not None else _workspace(need, A.device)
    _check("cf_getrf", _lib.cf_getrf(n, _ptr(A), lda, _ptr(ipiv), _ptr(info), _ptr(ws), ws.numel(),
                                     ctypes.byref(opt), _stream()))
    return ipiv[:n], info


def getrf_noalloc(A: torch.Tensor, v=None, leaf_h=None, arity=None, ipiv=None, info=None):
    """cf_getrf_noalloc: the LU of getrf with the library's fixed scratch
    instead of a work buffer (see include/cf.h).  ipiv and info may be passed
    in so that the call itself allocates nothing."""
    assert A.dtype == torch.float64
    n = A.shape[0]
    assert A.shape == (n, n)
    lda = _ld(A, "A")
    opt = options(v=v, leaf_h=leaf_h, arity=arity)
    if ipiv is None:
        ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
    # the C ABI writes n int32 pivots and one int32 info through these
    assert ipiv.dtype == torch.int32 and ipiv.device == A.device and ipiv.is_contiguous() and ipiv.numel() >= n
    assert info.dtype == torch.int32 and info.device == A.device and info.numel() >= 1
    _check("cf_getrf_noalloc", _lib.cf_getrf_noalloc(n, _ptr(A), lda, _ptr(ipiv), _ptr(info),
                                                     ctypes.byref(opt), _stream()))
    return ipiv[:n], info


def potrf(A: torch.Tensor, v=None, lookahead=None):
    """In-place lower Cholesky.  Returns info (device int32).  lookahead as
    in getrf."""
    assert A.dtype == torch.float64
    n = A.shape[0]
    lda = _ld(A, "A")
    opt = options(v=v, lookahead=lookahead)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    ws = _workspace(_lib.cf_potrf_workspace_size(n, ctypes.byref(opt)), A.device)
    _check("cf_potrf", _lib.cf_potrf(n, _ptr(A), lda, _ptr(info), _ptr(ws), ws.numel(),
                                     ctypes.byref(opt), _stream()))
    return info


def getrs(LU: torch.Tensor, ipiv: torch.Tensor, B: torch.Tensor):
    n = LU.shape[0]
    nrhs = B.shape[1] if B.dim() == 2 else 1
    ws = _workspace(_lib.cf_getrs_workspace_size(n, nrhs), LU.device)
    _check("cf_getrs", _lib.cf_getrs(n, nrhs, _ptr(LU), _ld(LU, "LU"), _ptr(ipiv), _ptr(B), _ld(B, "B"),
                                     _ptr(ws), ws.numel(), _stream()))
    return B


def potrs(L: torch.Tensor, B: torch.Tensor):
    n = L.shape[0]
    nrhs = B.shape[1] if B.dim() == 2 else 1
    _check("cf_potrs", _lib.cf_potrs(n, nrhs, _ptr(L), _ld(L, "L"), _ptr(B), _ld(B, "B"), _stream()))
    return B


def residual(A: torch.Tensor, X: torch.Tensor, B: torch.Tensor, R: torch.Tensor | None = None):
    m, n = A.shape
    nrhs = X.shape[1] if X.dim() == 2 else 1
    if R is None:
        R = fortran_empty(m, nrhs, device=A.device)
    _check("cf_residual", _lib.cf_residual(m, n, nrhs, _ptr(A), _ld(A, "A"), _ptr(X), _ld(X, "X"),
                                           _ptr(B), _ld(B, "B"), _ptr(R), _ld(R, "R"), _stream()))
    return R


def residual_tc(A: torch.Tensor, X: torch.Tensor, B: torch.Tensor, R: torch.Tensor | None = None):
    """R = B - A X at FP64 accuracy on the tensor cores (cf_residual_tc)."""
    m, n = A.shape
    nrhs = X.shape[1] if X.dim() == 2 else 1
    if R is None:
        R = fortran_empty(m, nrhs, device=A.device)
    ws = _workspace(_lib.cf_residual_tc_workspace_size(m, n, nrhs), A.device)
    _check("cf_residual_tc", _lib.cf_residual_tc(m, n, nrhs, _ptr(A), _ld(A, "A"), _ptr(X), _ld(X, "X"),
                                                 _ptr(B), _ld(B, "B"), _ptr(R), _ld(R, "R"), _ptr(ws), ws.numel(),
                                                 _stream()))
    return R


def residual_pair(A: torch.Tensor, X: torch.Tensor, B: torch.Tensor, R: torch.Tensor | None = None):
    """R = B - A X on the FP32 pipes at FP64 accuracy (cf_residual_pair)."""
    m, n = A.shape
    nrhs = X.shape[1] if X.dim() == 2 else 1
    if R is None:
        R = fortran_empty(m, nrhs, device=A.device)
    ws = _workspace(_lib.cf_residual_pair_workspace_size(m, n, nrhs), A.device)
    _check("cf_residual_pair", _lib.cf_residual_pair(m, n, nrhs, _ptr(A), _ld(A, "A"), _ptr(X), _ld(X, "X"),
                                                     _ptr(B), _ld(B, "B"), _ptr(R), _ld(R, "R"), _ptr(ws),
                                                     ws.numel(), _stream()))
    return R


def schur_update_lp(A_lp: torch.Tensor, B_lp: torch.Tensor, C: torch.Tensor, lower: bool = False):
    """C -= A_lp @ B_lp^T on the tensor cores; A_lp (m x k) and B_lp (n x k)
    row-major (K-major) bf16/fp16 tensors, C float32 column-major."""
    m, k = A_lp.shape
    n = B_lp.shape[0]
    prec = {torch.bfloat16: CF_BF16, torch.float16: CF_F16}[A_lp.dtype]
    _check("cf_schur_update_lp", _lib.cf_schur_update_lp(m, n, k, _ptr(A_lp), A_lp.stride(0), _ptr(B_lp),
                                                         B_lp.stride(0), _ptr(C), _ld(C, "C"), prec,
                                                         int(lower), _stream()))
    return C


def schur_update_lp_splitk(A_lp: torch.Tensor, B_lp: torch.Tensor, C: torch.Tensor, ksplit: int,
                           lower: bool = False):
    """cf_schur_update_lp_splitk: the update with K cut into ksplit ranges."""
    m, k = A_lp.shape
    n = B_lp.shape[0]
    prec = {torch.bfloat16: CF_BF16, torch.float16: CF_F16}[A_lp.dtype]
    ws = _workspace(_lib.cf_schur_update_lp_splitk_workspace_size(m, n, k, ksplit), C.device)
    _check("cf_schur_update_lp_splitk",
           _lib.cf_schur_update_lp_splitk(m, n, k, _ptr(A_lp), A_lp.stride(0), _ptr(B_lp), B_lp.stride(0), _ptr(C),
                                          _ld(C, "C"), prec, int(lower), ksplit, _ptr(ws), ws.numel(), _stream()))
    return C


def quantize_e4m3(src: torch.Tensor):
    """Per-128x128-tile e4m3 quantization of a column-major float32 block
    (cf_quantize_e4m3).  Returns (q uint8 rows x kpad K-major, scales float32
    ceil(rows/128) x kpad/128)."""
    rows, k = src.shape
    kpad = (k + 127) // 128 * 128
    q = torch.empty((rows, kpad), dtype=torch.uint8, device=src.device)
    sc = torch.empty((max((rows + 127) // 128, 1), kpad // 128), dtype=torch.float32, device=src.device)
    _check("cf_quantize_e4m3", _lib.cf_quantize_e4m3(rows, k, _ptr(src), _ld(src, "src"), _ptr(q), kpad, _ptr(sc),
                                                     kpad // 128, _stream()))
    return q, sc


def schur_update_fp8(qA, sA, qB, sB, C: torch.Tensor, lower: bool = False):
    """C -= sum_kb sA sB (qA qB^T)_kb on the tensor cores (cf_schur_update_fp8);
    qA (m x k), qB (n x k) uint8 e4m3 codes, K-major; sA, sB tile scales."""
    m, k = qA.shape
    n = qB.shape[0]
    _check("cf_schur_update_fp8", _lib.cf_schur_update_fp8(m, n, k, _ptr(qA), qA.stride(0), _ptr(sA), sA.stride(0),
                                                           _ptr(qB), qB.stride(0), _ptr(sB), sB.stride(0), _ptr(C),
                                                           _ld(C, "C"), int(lower), _stream()))
    return C


def trsv_f32(T: torch.Tensor, X: torch.Tensor, mode: int):
    """cf_trsv_f32: X <- M^-1 X in place with the FP32 factor T (mode 0: unit
    lower, 1: upper, 2: lower, 3: lower transposed); nrhs <= 16."""
    assert T.dtype == torch.float32 and X.dtype == torch.float32
    n = T.shape[0]
    nrhs = X.shape[1] if X.dim() == 2 else 1
    ws = _workspace(_lib.cf_trsv_f32_workspace_size(n), T.device)
    _check("cf_trsv_f32", _lib.cf_trsv_f32(mode, n, nrhs, _ptr(T), _ld(T, "T"), _ptr(X), _ld(X, "X"), _ptr(ws),
                                           ws.numel(), _stream()))
    return X


def trsv_f32_withheld(T: torch.Tensor, X: torch.Tensor, mode: int, spin_limit: int = 0):
    """cf_trsv_f32_withheld: the same solve with its first block withheld, so
    that every wait for it runs out (failure-detection test; X comes back
    wrong and cf_device_status reports CF_ERR_TIMEOUT)."""
    assert T.dtype == torch.float32 and X.dtype == torch.float32
    n = T.shape[0]
    nrhs = X.shape[1] if X.dim() == 2 else 1
    ws = _workspace(_lib.cf_trsv_f32_workspace_size(n), T.device)
    _check("cf_trsv_f32_withheld", _lib.cf_trsv_f32_withheld(mode, n, nrhs, _ptr(T), _ld(T, "T"), _ptr(X),
                                                             _ld(X, "X"), spin_limit, _ptr(ws), ws.numel(),
                                                             _stream()))
    return X


def device_status() -> int:
    """Synchronises the current stream; CF_OK or CF_ERR_TIMEOUT (then cleared)."""
    return _lib.cf_device_status(_stream())


def _mixed(fn, wsfn, A, B, prec, opt_kw, work=None):
    n = A.shape[0]
    nrhs = B.shape[1] if B.dim() == 2 else 1
    X = fortran_empty(n, nrhs, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    opt = options(**opt_kw)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    need = wsfn(n, nrhs, p, ctypes.byref(opt))
    ws = work if work is not None else _workspace(need, A.device)
    stats = RefineStats()
    st = fn(n, nrhs, _ptr(A), _ld(A, "A"), _ptr(B), _ld(B, "B"), _ptr(X), _ld(X, "X"), p, _ptr(info),
            ctypes.byref(stats), _ptr(ws), ws.numel(), ctypes.byref(opt), _stream())
    if st not in (CF_OK, CF_ERR_NOT_CONVERGED):
        raise CfError(fn.__name__, st)
    return X, info, stats, st


def gesv_mixed(A, B, prec="bf16", work=None, **opt_kw):
    """Mixed-precision LU solve with FP64 refinement; A, B unchanged.
    Returns (X, info, stats, status)."""
    return _mixed(_lib.cf_gesv_mixed, _lib.cf_gesv_mixed_workspace_size, A, B, prec, opt_kw, work)


def posv_mixed(A, B, prec="bf16", work=None, **opt_kw):
    """Mixed-precision Cholesky solve with FP64 refinement."""
    return _mixed(_lib.cf_posv_mixed, _lib.cf_posv_mixed_workspace_size, A, B, prec, opt_kw, work)


def gesv_mixed_workspace_size(n, nrhs, prec="bf16", **opt_kw):
    opt = options(**opt_kw)
    return _lib.cf_gesv_mixed_workspace_size(n, nrhs, PREC[prec], ctypes.byref(opt))


def posv_mixed_workspace_size(n, nrhs, prec="bf16", **opt_kw):
    opt = options(**opt_kw)
    return _lib.cf_posv_mixed_workspace_size(n, nrhs, PREC[prec], ctypes.byref(opt))


class Batch:
    """A batch of column-major matrices packed in one device buffer, with the
    device pointer / size arrays the batched C entry points take."""

    def __init__(self, sizes, device="cuda", dtype=torch.float64, kinds=None):
        self.sizes = [int(x) for x in sizes]
        offs, o = [], 0
        for n in self.sizes:
            offs.append(o)
            o += max(n * n, 1)
            o = (o + 31) // 32 * 32          # 256-byte alignment of every matrix
        self.offsets = offs
        self.data = torch.zeros(max(o, 1), dtype=dtype, device=device)
        el = self.data.element_size()
        base = self.data.data_ptr()
        self.n = torch.tensor(self.sizes, dtype=torch.int32, device=device)
        self.lda = torch.tensor([max(n, 1) for n in self.sizes], dtype=torch.int32, device=device)
        self.ptrs = torch.tensor([base + el * q for q in offs], dtype=torch.int64, device=device)
        self.kind = None if kinds is None else torch.tensor(list(kinds), dtype=torch.int32, device=device)
        po, p = [], 0
        for n in self.sizes:
            po.append(p)
            p += max(n, 1)
        self.vec_offsets = po
        self.vec_total = max(p, 1)

    def matrix(self, i):
        n = self.sizes[i]
        return self.data[self.offsets[i]:self.offsets[i] + n * n].view(n, n).t()

    def vec_ptrs(self, buf):
        el = buf.element_size()
        return torch.tensor([buf.data_ptr() + el * q for q in self.vec_offsets], dtype=torch.int64,
                            device=buf.device)


def factor_batched(batch: "Batch", default_kind=0, v=None, work=None, batch_cps=None, opt=None):
    """In-place FP64 LU / Cholesky of every matrix (cf_factor_batched).
    Returns (ipiv buffer, ipiv pointer array, info)."""
    nb = len(batch.sizes)
    ipiv = torch.zeros(batch.vec_total, dtype=torch.int32, device=batch.data.device)
    iptr = batch.vec_ptrs(ipiv)
    info = torch.zeros(max(nb, 1), dtype=torch.int32, device=batch.data.device)
    opt = opt if opt is not None else options(v=v, batch_cps=batch_cps)
    ws = work if work is not None else _workspace(_lib.cf_factor_batched_workspace_size(nb, ctypes.byref(opt)),
                                                  batch.data.device)
    kind = _ptr(batch.kind) if batch.kind is not None else ctypes.c_void_p(0)
    _check("cf_factor_batched", _lib.cf_factor_batched(nb, kind, default_kind, _ptr(batch.n), _ptr(batch.ptrs),
                                                       _ptr(batch.lda), _ptr(iptr), _ptr(info), _ptr(ws),
                                                       ws.numel(), ctypes.byref(opt), _stream()))
    torch.cuda.current_stream().synchronize()     # iptr is freed on return
    return ipiv, iptr, info


def solve_batched_mixed(batch: "Batch", B: torch.Tensor, default_kind=0, tol=None, max_iter=None, work=None,
                        v=None, batch_cps=None, opt=None):
    """FP32 factors + FP64 refinement for every A_i x_i = b_i
    (cf_solve_batched_mixed); B packed like batch.vec_offsets.  Returns
    (X, info, iters, eta, solver), solver[i] = 32 or 64 (the precision of
    the factors that produced x_i)."""
    nb = len(batch.sizes)
    dev = batch.data.device
    X = torch.zeros(batch.vec_total, dtype=torch.float64, device=dev)
    info = torch.zeros(max(nb, 1), dtype=torch.int32, device=dev)
    iters = torch.zeros(max(nb, 1), dtype=torch.int32, device=dev)
    eta = torch.zeros(max(nb, 1), dtype=torch.float64, device=dev)
    solver = torch.zeros(max(nb, 1), dtype=torch.int32, device=dev)
    opt = opt if opt is not None else options(tol=tol, max_iter=max_iter, v=v, batch_cps=batch_cps)
    ws = work if work is not None else _workspace(_lib.cf_solve_batched_mixed_workspace_size(nb, ctypes.byref(opt)),
                                                  dev)
    kind = _ptr(batch.kind) if batch.kind is not None else ctypes.c_void_p(0)
    bptr = batch.vec_ptrs(B)      # keep the pointer arrays alive across the call
    xptr = batch.vec_ptrs(X)
    _check("cf_solve_batched_mixed",
           _lib.cf_solve_batched_mixed(nb, kind, default_kind, _ptr(batch.n), _ptr(batch.ptrs), _ptr(batch.lda),
                                       _ptr(bptr), _ptr(xptr), _ptr(info), _ptr(iters), _ptr(eta), _ptr(solver),
                                       _ptr(ws), ws.numel(), ctypes.byref(opt), _stream()))
    torch.cuda.current_stream().synchronize()
    return X, info, iters, eta, solver


def batched_autotune(batch: "Batch", mixed=False, default_kind=0, **opt_kw):
    """cf_batched_autotune: times the candidate (v, batch_cps) pairs on a
    synthetic sample with the batch's sizes and kinds; returns (Options with
    the fastest, sample milliseconds)."""
    nb = len(batch.sizes)
    hn = (ctypes.c_int * nb)(*batch.sizes)
    hk = None
    if batch.kind is not None:
        hk = (ctypes.c_int * nb)(*[int(x) for x in batch.kind.cpu().tolist()])
    kptr = ctypes.cast(hk, ctypes.c_void_p) if hk is not None else ctypes.c_void_p(0)
    nptr = ctypes.cast(hn, ctypes.c_void_p)
    need = _lib.cf_batched_autotune_workspace_size(nb, nptr, kptr, default_kind, int(mixed))
    ws = _workspace(need, batch.data.device)
    opt = options(**opt_kw)
    ms = ctypes.c_float(0.0)
    _check("cf_batched_autotune", _lib.cf_batched_autotune(nb, nptr, kptr, default_kind, int(mixed), _ptr(ws),
                                                           ws.numel(), ctypes.byref(opt), ctypes.byref(ms),
                                                           _stream()))
    return opt, ms.value


class BatchedPlan:
    """Everything a batched call needs, allocated once, so that the call
    itself only enqueues work: run() on the current stream, or capture() into
    a CUDA graph and replay() it (BAT-1 "one persistent launch captured in a
    CUDA graph").  kind: "factor" (in-place FP64 LU / Cholesky) or "mixed"
    (FP32 factors + FP64 refinement; set the right-hand sides in .B)."""

    def __init__(self, batch: "Batch", kind="factor", default_kind=0, opt=None):
        self.batch, self.kind_name, self.default_kind = batch, kind, default_kind
        self.opt = opt if opt is not None else options()
        dev = batch.data.device
        nb = len(batch.sizes)
        self.nb = nb
        self.info = torch.zeros(max(nb, 1), dtype=torch.int32, device=dev)
        if kind == "factor":
            self.ipiv = torch.zeros(batch.vec_total, dtype=torch.int32, device=dev)
            self.iptr = batch.vec_ptrs(self.ipiv)
            need = _lib.cf_factor_batched_workspace_size(nb, ctypes.byref(self.opt))
        else:
            self.B = torch.zeros(batch.vec_total, dtype=torch.float64, device=dev)
            self.X = torch.zeros(batch.vec_total, dtype=torch.float64, device=dev)
            self.bptr, self.xptr = batch.vec_ptrs(self.B), batch.vec_ptrs(self.X)
            self.iters = torch.zeros(max(nb, 1), dtype=torch.int32, device=dev)
            self.eta = torch.zeros(max(nb, 1), dtype=torch.float64, device=dev)
            self.solver = torch.zeros(max(nb, 1), dtype=torch.int32, device=dev)
            need = _lib.cf_solve_batched_mixed_workspace_size(nb, ctypes.byref(self.opt))
        self.ws = _workspace(need, dev)
        self.graph = None
        torch.cuda.synchronize()

    def run(self):
        b = self.batch
        kind = _ptr(b.kind) if b.kind is not None else ctypes.c_void_p(0)
        if self.kind_name == "factor":
            _check("cf_factor_batched", _lib.cf_factor_batched(
                self.nb, kind, self.default_kind, _ptr(b.n), _ptr(b.ptrs), _ptr(b.lda), _ptr(self.iptr),
                _ptr(self.info), _ptr(self.ws), self.ws.numel(), ctypes.byref(self.opt), _stream()))
        else:
            _check("cf_solve_batched_mixed", _lib.cf_solve_batched_mixed(
                self.nb, kind, self.default_kind, _ptr(b.n), _ptr(b.ptrs), _ptr(b.lda), _ptr(self.bptr),
                _ptr(self.xptr), _ptr(self.info), _ptr(self.iters), _ptr(self.eta), _ptr(self.solver),
                _ptr(self.ws), self.ws.numel(), ctypes.byref(self.opt), _stream()))

    def capture(self):
        """Capture one run() into a CUDA graph (on a side stream, as torch
        requires); replay() then launches it."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(self.graph, stream=s):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        return self.graph

    def replay(self):
        self.graph.replay()


def kernel_launches() -> int:
    """Kernel launches libcf has enqueued in this process so far."""
    return int(_lib.cf_kernel_launches())


def lib():
    return _lib
