"""FP64 CPU oracle for the COnfLUX / COnfCHOX hot path (arXiv 2108.09337).

TEST INFRASTRUCTURE ONLY.  The product library never imports this package;
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path: the arithmetic lives in ``cf_oracle.c`` (plain C, compiled with
``-O2 -ffp-contract=off``); this module only marshals numpy arrays and writes
out the plain definitions of the error measures.

Functions and the passages they follow:

* :func:`tourn_select` -- TournPivot (Alg. 1; Sec. 7.3 "Tournament
  Pivoting" and "Pivoting in COnfLUX"; the pivot selection in the I/O-cost proof).
* :func:`getrf` -- COnfLUX LU (Alg. 1, Sec. 7.2 routines, Table 2; the
  in-place LU of Fig. "prog_rep").
* :func:`potrf` -- COnfCHOX's factorization, Listing "Cholesky Factorization"
  (Sec. 6.2), lower triangle.
* :func:`getrs`, :func:`potrs` -- substitution with the factors (paper
  silent; textbook definition).
* :func:`residual` -- R = B - A X with the compensated dot product Dot2
  (Ogita, Rump, Oishi 2005).
* :func:`lu_flops`, :func:`chol_flops`, :func:`io_lower_bound_lu`,
  :func:`io_lower_bound_chol`, :func:`io_conflux` -- closed forms of Sec. 6.1,
  6.2 and Sec. 7.4 (Lemma on the I/O cost of COnfLUX).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cf_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

EPS = float(np.finfo(np.float64).eps) / 2.0  # unit roundoff u = 2^-53


def build(force: bool = False) -> str:
    """Compile cf_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.or_tourn_select.argtypes = [I, I, P, I, I, I, P, P]
            lib.or_getrf.argtypes = [I, P, I, I, I, I, P, P, P, P]
            lib.or_potrf.argtypes = [I, P, I, P, P]
            lib.or_getrs.argtypes = [I, I, P, I, P, P, I]
            lib.or_potrs.argtypes = [I, I, P, I, P, I]
            lib.or_residual.argtypes = [I, I, I, P, I, P, I, P, I, P, I]
            for f in (lib.or_tourn_select, lib.or_getrf, lib.or_potrf,
                      lib.or_getrs, lib.or_potrs, lib.or_residual):
                f.restype = I
            _lib = lib
    return _lib


def _fortran(a: np.ndarray) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def tourn_select(panel: np.ndarray, h: int = 128, arity: int = 2):
    """TournPivot on an m x w panel.  Returns (winners, min_gap): 0-based panel
    row indices of the min(m, w) pivots in pivot order, and the smallest
    argmax gap seen at any column of any node."""
    P = _fortran(panel)
    m, w = P.shape
    win = np.zeros(max(min(m, w), 1), dtype=np.int32)
    gap = ctypes.c_double(1.0)
    ld = max(m, 1)
    np_ = _load().or_tourn_select(m, w, _ptr(P), ld, int(h), int(arity),
                                  _ptr(win), ctypes.byref(gap))
    return win[:np_].copy(), gap.value


def getrf(A: np.ndarray, v: int = 128, h: int = 128, arity: int = 2):
    """COnfLUX LU with tournament pivoting.  Returns (LU, ipiv, info, gaps,
    n_upd): the in-place factors, 1-based LAPACK ipiv, info, the smallest
    tournament gap of each step and the number of updates
    A[i,j] -= A[i,k] A[k,j] executed.
    h >= n gives Gaussian elimination with partial pivoting."""
    LU = _fortran(A).copy(order="F")
    n = LU.shape[0]
    assert LU.shape == (n, n)
    ipiv = np.zeros(max(n, 1), dtype=np.int32)
    info = ctypes.c_int(0)
    nsteps = max((n + v - 1) // v, 1)
    gaps = np.ones(nsteps, dtype=np.float64)
    nupd = ctypes.c_longlong(0)
    rc = _load().or_getrf(n, _ptr(LU), max(n, 1), int(v), int(h), int(arity),
                          _ptr(ipiv), ctypes.byref(info), _ptr(gaps),
                          ctypes.byref(nupd))
    if rc != 0:
        raise ValueError("or_getrf: bad argument")
    return LU, ipiv[:n].copy(), info.value, gaps[:(n + v - 1) // v], nupd.value


def potrf(A: np.ndarray):
    """Cholesky (lower).  Returns (L, info, n_upd); the strict upper triangle
    of L is zeroed."""
    L = _fortran(A).copy(order="F")
    n = L.shape[0]
    info = ctypes.c_int(0)
    nupd = ctypes.c_longlong(0)
    rc = _load().or_potrf(n, _ptr(L), max(n, 1), ctypes.byref(info),
                          ctypes.byref(nupd))
    if rc != 0:
        raise ValueError("or_potrf: bad argument")
    L = np.tril(L)
    return np.asfortranarray(L), info.value, nupd.value


def getrs(LU: np.ndarray, ipiv: np.ndarray, B: np.ndarray) -> np.ndarray:
    LU = _fortran(LU)
    X = _fortran(B.reshape(B.shape[0], -1)).copy(order="F")
    n, nrhs = X.shape
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _load().or_getrs(n, nrhs, _ptr(LU), max(n, 1), _ptr(piv), _ptr(X),
                     max(n, 1))
    return X.reshape(B.shape)


def potrs(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    L = _fortran(L)
    X = _fortran(B.reshape(B.shape[0], -1)).copy(order="F")
    n, nrhs = X.shape
    _load().or_potrs(n, nrhs, _ptr(L), max(n, 1), _ptr(X), max(n, 1))
    return X.reshape(B.shape)


def residual(A: np.ndarray, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    """R = B - A X, compensated (about twice FP64 accuracy)."""
    A = _fortran(A)
    Xf = _fortran(X.reshape(X.shape[0], -1))
    Bf = _fortran(B.reshape(B.shape[0], -1))
    m, n = A.shape
    nrhs = Xf.shape[1]
    R = np.zeros((m, nrhs), dtype=np.float64, order="F")
    _load().or_residual(m, n, nrhs, _ptr(A), max(m, 1), _ptr(Xf), max(n, 1),
                        _ptr(Bf), max(m, 1), _ptr(R), max(m, 1))
    return R.reshape(B.shape)


# --------------------------------------------------------------------------
# Plain definitions built on the factors.
# --------------------------------------------------------------------------
def perm_from_ipiv(ipiv: np.ndarray, n: int) -> np.ndarray:
    """Row order p such that (P A)[i] = A[p[i]], from 1-based interchanges."""
    p = np.arange(n)
    for i in range(len(ipiv)):
        j = int(ipiv[i]) - 1
        if j != i:
            p[i], p[j] = p[j], p[i]
    return p


def split_lu(LU: np.ndarray):
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    return L, U


def lu_residual(A: np.ndarray, LU: np.ndarray, ipiv: np.ndarray) -> float:
    """||P A - L U||_1 / (n * u * ||A||_1), u = 2^-53."""
    n = A.shape[0]
    if n == 0:
        return 0.0
    L, U = split_lu(LU)
    p = perm_from_ipiv(ipiv, n)
    R = A[p, :] - L @ U
    na = np.linalg.norm(A, 1)
    return float(np.linalg.norm(R, 1) / (n * EPS * na)) if na > 0 else 0.0


def chol_residual(A: np.ndarray, L: np.ndarray) -> float:
    """||A - L L^T||_1 / (n * u * ||A||_1) over the full symmetric A."""
    n = A.shape[0]
    if n == 0:
        return 0.0
    L = np.tril(L)
    R = A - L @ L.T
    na = np.linalg.norm(A, 1)
    return float(np.linalg.norm(R, 1) / (n * EPS * na)) if na > 0 else 0.0


def backward_error(A: np.ndarray, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Per-column eta_j = ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf)
    with the compensated residual."""
    R = residual(A, X, B).reshape(A.shape[0], -1)
    Xc = X.reshape(X.shape[0], -1)
    Bc = B.reshape(B.shape[0], -1)
    na = np.linalg.norm(A, np.inf)
    num = np.abs(R).max(axis=0)
    den = na * np.abs(Xc).max(axis=0) + np.abs(Bc).max(axis=0)
    return num / den


def lu_random_projection_error(apply_pa, apply_l, apply_u, n, norm_a,
                               nvec: int = 4, seed: int = 0) -> float:
    """Probabilistic form of the factorization residual for large n:
    max over nvec random z of ||P A z - L (U z)||_2 / (||A||_F ||z||_2),
    given callables that apply P A, L and U to a vector block."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, nvec))
    R = apply_pa(Z) - apply_l(apply_u(Z))
    return float(np.max(np.linalg.norm(R, axis=0) /
                        (norm_a * np.linalg.norm(Z, axis=0))))


# --------------------------------------------------------------------------
# Closed forms.
# --------------------------------------------------------------------------
def lu_update_count(n: int) -> int:
    """Executions of the update A[i,j] -= A[i,k] A[k,j] in the in-place LU of
    Fig. "prog_rep":
    sum_k (n-k-1)^2 = (n-1) n (2n-1) / 6."""
    return (n - 1) * n * (2 * n - 1) // 6


def chol_update_count(n: int) -> int:
    """Executions of the trailing update A[i,j] -= A[i,k] A[j,k] (j <= i) in
    the Cholesky listing: sum_k (n-k-1)(n-k)/2."""
    return (n - 1) * n * (n + 1) // 6


def lu_flops(n: int) -> float:
    """Flop convention of the metric: 2 n^3 / 3 (leading term of twice the update count)."""
    return 2.0 * n ** 3 / 3.0


def chol_flops(n: int) -> float:
    """n^3 / 3 (leading term of twice the update count)."""
    return n ** 3 / 3.0


def io_lower_bound_lu(N: float, P: float, M: float) -> float:
    """Sec. 6.1: Q >= (2N^3 - 6N^2 + 4N) / (3 P sqrt(M)) + N(N-1)/(2P)."""
    return (2 * N ** 3 - 6 * N ** 2 + 4 * N) / (3 * P * np.sqrt(M)) + \
        N * (N - 1) / (2 * P)


def io_lower_bound_chol(N: float, P: float, M: float) -> float:
    """Sec. 6.2: Q >= N^3 / (3 P sqrt(M)) + N^2 / (2P) + N / P."""
    return N ** 3 / (3 * P * np.sqrt(M)) + N ** 2 / (2 * P) + N / P


def io_conflux(N: float, P: float, M: float) -> float:
    """Leading term of the COnfLUX I/O cost (Sec. 7.4): N^3 / (P sqrt(M))."""
    return N ** 3 / (P * np.sqrt(M))
