"""Seeded synthetic inputs for the factorizations.

This module holds only random-matrix recipes; none of the factorization
arithmetic lives here.  Both the CUDA path's tests and benchmarks and the CPU
oracle's tests draw their inputs from it, so the two sides always see the
same bytes.  All matrices are returned column-major (Fortran order) float64.

Recipes (the paper measures synthetic dense matrices only, Sec. 9):

* ``uniform_pm1``  -- a_ij = 2u - 1, u ~ U[0, 1), optional diagonal shift s.
* ``spd_gram``     -- A = G G^T / n + alpha I, G_ij ~ N(0, 1), symmetrised.
* ``rhs_normal``   -- right-hand sides, i.i.d. N(0, 1).
* ``constructed_plu`` -- A = P^T L U with unit lower L, |L_ij| <= 1 - gap and
  |U_ii| in [1, 2]: Gaussian elimination with partial pivoting must return
  exactly P, with every argmax separated by at least ``gap`` (relative),
  and exactly ``gap`` at one row per column.
* ``dyadic_plu``   -- the same with L in {0, +-1/4, +-1/2, +-3/4} and U small
  integers with U_ii in {+-1, +-2}: A is exact in binary64 and elimination
  recovers L and U exactly.
* ``integer_l0``   -- lower L0 with small integer entries and power-of-two
  diagonal, A = L0 L0^T exact in binary64.
* ``small_int``    -- integer entries in [lo, hi].

For sizes where host generation is slow the ``*_torch`` variants draw on the
device with torch's Philox generator; the oracle side then receives a copy of
exactly those bytes.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def uniform_pm1(n: int, seed: int = 0, shift: float = 0.0, m: int | None = None
                ) -> np.ndarray:
    m = n if m is None else m
    A = 2.0 * _rng(seed).random((n, m)) - 1.0
    A = np.asfortranarray(A)
    if shift:
        k = min(n, m)
        A[np.arange(k), np.arange(k)] += shift
    return A


def spd_gram(n: int, seed: int = 1, alpha: float = 1.0) -> np.ndarray:
    G = _rng(seed).standard_normal((n, n))
    A = (G @ G.T) / n
    A = 0.5 * (A + A.T)
    A[np.arange(n), np.arange(n)] += alpha
    return np.asfortranarray(A)


def rhs_normal(n: int, nrhs: int = 1, seed: int = 2) -> np.ndarray:
    return np.asfortranarray(_rng(seed).standard_normal((n, nrhs)))


def small_int(n: int, seed: int, lo: int = -5, hi: int = 5) -> np.ndarray:
    return np.asfortranarray(
        _rng(seed).integers(lo, hi + 1, size=(n, n)).astype(np.float64))


def constructed_plu(n: int, seed: int, gap: float = 1e-3,
                    lscale: float = 0.2, uscale: float = 0.2):
    """Returns (A, perm, L, U) with A[perm[i]] = (L U)[i] (so P A = L U for
    the row order perm).  Off-diagonal L entries are U(-lscale, lscale) plus
    one entry per column of magnitude exactly 1 - gap (so the smallest argmax
    separation is gap); off-diagonal U entries are U(-uscale, uscale).  The
    small scales keep L and U well conditioned, so that floating-point
    elimination stays close enough to the exact one for the pivots to be
    the constructed ones up to n of about a thousand."""
    rng = _rng(seed)
    L = np.tril(rng.uniform(-lscale, lscale, (n, n)), -1)
    for j in range(n - 1):
        L[rng.integers(j + 1, n), j] = (1.0 - gap) * rng.choice([-1.0, 1.0])
    L += np.eye(n)
    U = np.triu(rng.uniform(-uscale, uscale, (n, n)), 1)
    d = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    U[np.arange(n), np.arange(n)] = d
    perm = rng.permutation(n)
    LUm = L @ U
    A = np.empty_like(LUm)
    A[perm, :] = LUm
    return np.asfortranarray(A), perm, L, U


def dyadic_plu(n: int, seed: int):
    """Exact variant of constructed_plu (n <= 64 keeps every value exact)."""
    rng = _rng(seed)
    L = np.tril(rng.integers(-3, 4, (n, n)) / 4.0, -1) + np.eye(n)
    U = np.triu(rng.integers(-3, 4, (n, n)).astype(np.float64), 1)
    d = rng.choice([1.0, 2.0], n) * rng.choice([-1.0, 1.0], n)
    U[np.arange(n), np.arange(n)] = d
    perm = rng.permutation(n)
    LUm = L @ U
    A = np.empty_like(LUm)
    A[perm, :] = LUm
    return np.asfortranarray(A), perm, L, U


def integer_l0(n: int, seed: int):
    """Returns (A, L0) with A = L0 L0^T exact in binary64 (n <= 64)."""
    rng = _rng(seed)
    L0 = np.tril(rng.integers(-3, 4, (n, n)).astype(np.float64), -1)
    L0[np.arange(n), np.arange(n)] = rng.choice([1.0, 2.0, 4.0], n)
    A = L0 @ L0.T
    return np.asfortranarray(A), L0


# --------------------------------------------------------------------------
# Device-side variants for large n (torch Philox; torch is plumbing here).
# --------------------------------------------------------------------------
def prescribed_cond(n: int, cond: float, seed: int, spd: bool = False) -> np.ndarray:
    """Q1 diag(s) Q2^T with Q1, Q2 Haar-random orthogonal (QR of Gaussian
    matrices, sign-fixed) and s geometric from 1 down to 1/cond; spd=True
    takes Q2 = Q1 (symmetric positive definite, condition number cond)."""
    g = _rng(seed)
    def haar():
        q, r = np.linalg.qr(g.standard_normal((n, n)))
        return q * np.sign(np.diag(r))
    q1 = haar()
    q2 = q1 if spd else haar()
    s = np.geomspace(1.0, 1.0 / cond, n) if n > 1 else np.ones(1)
    A = (q1 * s) @ q2.T
    if spd:
        A = 0.5 * (A + A.T)
    return np.asfortranarray(A)


def typed_panel(m: int, w: int, seed: int, eps: float = 1e-4, ratio: float = 1.004) -> np.ndarray:
    """An m x w panel (m a multiple of w) on which every argmax of tournament
    pivoting is separated by about ratio - 1 (relative), whatever the leaf
    height (a multiple of w) and the arity.  Each block of w consecutive rows
    holds one row of every "type" j < w (in shuffled order); a row of type j
    has one entry of magnitude in [1, ratio^(m/w)) at column j (random sign;
    the values of a type are distinct powers of ratio, shuffled) and entries
    of magnitude <= eps elsewhere.  Eliminating with a pivot of type j' moves
    the other rows' entries by O(eps) at most, so column j of every leaf or
    playoff node picks its largest row of type j, which beats the next one by
    a factor ratio and every other row by about 1/eps.  Entries are rounded
    to float32 (exact in both precisions)."""
    assert m % w == 0
    rng = _rng(seed)
    P = eps * (2.0 * rng.random((m, w)) - 1.0)
    nper = m // w
    types = np.concatenate([rng.permutation(w) for _ in range(nper)])
    mags = np.empty(m)
    for j in range(w):
        rows = np.nonzero(types == j)[0]
        mags[rows] = ratio ** rng.permutation(nper)
    sign = np.where(rng.random(m) < 0.5, -1.0, 1.0)
    P[np.arange(m), types] = sign * mags
    return np.asfortranarray(P.astype(np.float32).astype(np.float64))


def uniform_pm1_torch(n: int, seed: int = 0, shift: float = 0.0,
                      device="cuda", dtype=None):
    import torch
    dtype = dtype or torch.float64
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    # Column-major n x n: allocate the transpose contiguous and view it.
    At = torch.rand((n, n), generator=g, device=device, dtype=dtype)
    At.mul_(2.0).sub_(1.0)
    if shift:
        At.diagonal().add_(shift)
    return At.t()  # column-major view, stride (1, n)


def spd_gram_torch(n: int, seed: int = 1, alpha: float = 1.0, device="cuda"):
    """A = fl32(G G^T) / n symmetrised in float64, + alpha I.  The Gram product
    is formed in float32 on the device (an FP64 product at n = 32768 would
    take about a minute on this part); symmetrising and the shift are FP64."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn((n, n), generator=g, device=device, dtype=torch.float32)
    C = torch.empty((n, n), device=device, dtype=torch.float64)
    blk = 8192
    for i in range(0, n, blk):
        Ci = (G[i:i + blk] @ G.t()).to(torch.float64)
        C[i:i + blk] = Ci
    del G
    C.div_(n)
    # Symmetrise blockwise: C = (C + C^T) / 2
    for i in range(0, n, blk):
        for j in range(i, n, blk):
            a = C[i:i + blk, j:j + blk]
            b = C[j:j + blk, i:i + blk]
            s = 0.5 * (a + b.t())
            C[i:i + blk, j:j + blk] = s
            C[j:j + blk, i:i + blk] = s.t()
    C.diagonal().add_(alpha)
    return C.t()  # symmetric: the column-major view holds the same matrix


def shift_to_kappa_torch(A, kappa: float, iters: int = 30, seed: int = 5):
    """Adds alpha I to the symmetric positive semi-definite A (in place) with
    alpha = lambda_max / (kappa - 1), lambda_max estimated by ``iters`` power
    iterations from a seeded N(0, 1) start, so that A + alpha I has condition
    number about kappa when lambda_min(A) ~ 0 (the Gram matrix of a square G).
    Returns (alpha, lambda_max estimate)."""
    import torch
    n = A.shape[0]
    g = torch.Generator(device=A.device)
    g.manual_seed(seed)
    x = torch.randn(n, 1, generator=g, device=A.device, dtype=torch.float64)
    lam = 0.0
    for _ in range(iters):
        y = A @ x
        lam = float(torch.linalg.vector_norm(y) / torch.linalg.vector_norm(x))
        x = y / torch.linalg.vector_norm(y)
    alpha = lam / (kappa - 1.0)
    A.diagonal().add_(alpha)
    return alpha, lam


def rhs_normal_torch(n: int, nrhs: int, seed: int = 2, device="cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    Bt = torch.randn((nrhs, n), generator=g, device=device,
                     dtype=torch.float64)
    return Bt.t()  # column-major n x nrhs
