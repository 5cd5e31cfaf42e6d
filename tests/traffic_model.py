"""Bytes moved by the mixed-precision factorizations' schedule, per
factorization, for comparison with the paper's I/O lower bounds recast for
one GPU (Sec. 6.1 LU, Sec. 6.2 Cholesky).  A model of the launch sequence of
the library's mixed LU and Cholesky (steps of v = 128 columns inside slabs of
V columns, every slab's update of the rest one K = V contraction), counting
per launch:

* loads into the SMs: what the kernels bring into shared memory, TMEM or
  registers, from L2 or HBM.  The tensor-core update loads a 128-row A tile
  and a 256-row B tile of K x 2 bytes per segment for each 128 x 256 C tile
  and reads + writes that C tile in FP32; a panel kernel loads its operands
  once;
* HBM: every FP32 C element read and written once per update launch, each
  operand once (the tiles shared by neighbouring CTAs come from L2).

Row swaps are left out: they depend on the matrix (none when the pivots sit
on the diagonal)."""
import math

BM, BN = 128, 256


def schur(M, N, K, lower=False, S=1):
    """(loads, hbm) bytes of one tensor-core update C[M x N] -= A B^T of
    depth K with S operand segments (split BF16: S = 3); lower: the tiles on
    or below the diagonal only."""
    if M <= 0 or N <= 0 or K <= 0:
        return 0.0, 0.0
    tm, tn = math.ceil(M / BM), math.ceil(N / BN)
    if lower:
        tiles = sum(min(tn, (i * BM + BM - 1) // BN + 1) for i in range(tm))
    else:
        tiles = tm * tn
    loads = tiles * ((BM + BN) * S * K * 2 + BM * BN * 8)
    area = M * N / 2 if lower else M * N
    return float(loads), float(area * 8 + (M + N) * S * K * 2)


def mixed_lu(n, V, v=128, S=1):
    """Per-part (loads, hbm) of the mixed LU (FP16/BF16: S = 1)."""
    parts = {}

    def add(k, a, b):
        p = parts.setdefault(k, [0.0, 0.0])
        p[0] += a
        p[1] += b
    for J0 in range(0, n, V):
        JE = min(J0 + V, n)
        for k0 in range(J0, JE, v):
            wd, m = min(v, JE - k0), n - k0
            leaves = math.ceil(m / 256)
            node_rows = (leaves - 1) * 256 * wd * 4 + (leaves * min(256, m) * wd * 4 if leaves > 1 else 0)
            add("tournament", m * wd * 4 + node_rows, m * wd * 4)
            add("A00", wd * wd * 8, 0)
            below, right, off, nout = m - wd, n - k0 - wd, k0 - J0, n - JE
            if off > 0 and nout > 0:
                a, b = schur(wd, nout, off, S=S)
                add("pivot-row update", a + wd * off * 6, b)
            add("LU-4", wd * right * (8 + 2 * S), wd * right * (8 + 2 * S))
            if nout > 0:
                add("operands", wd * nout * (4 + 2 * S), wd * nout * (4 + 2 * S))
            add("LU-3", below * wd * (8 + 2 * S), below * wd * (8 + 2 * S))
            nslab = JE - (k0 + wd)
            if below > 0 and nslab > 0:
                add("in-slab update", *schur(below, nslab, wd, S=S))
        if JE < n:
            mr, Vs = n - JE, JE - J0
            add("operands", mr * Vs * (4 + 2 * S), mr * Vs * (4 + 2 * S))
            add("K=V update", *schur(mr, mr, Vs, S=S))
    return parts


def mixed_chol(n, V, v=128, S=3):
    """Per-part (loads, hbm) of the mixed Cholesky (split BF16: S = 3)."""
    parts = {}

    def add(k, a, b):
        p = parts.setdefault(k, [0.0, 0.0])
        p[0] += a
        p[1] += b
    for J0 in range(0, n, V):
        JE = min(J0 + V, n)
        for k0 in range(J0, JE, v):
            wd, m = min(v, JE - k0), n - k0
            add("A00", wd * wd * 8, wd * wd * 8)
            below = m - wd
            add("CH-2", below * wd * (8 + 4 * S), below * wd * (8 + 4 * S))
            nslab = JE - (k0 + wd)
            if below > 0 and nslab > 0:
                add("in-slab update", *schur(below, nslab, wd, S=S))
        if JE < n:
            mr, Vs = n - JE, JE - J0
            add("operands", mr * Vs * (4 + 4 * S), mr * Vs * (4 + 4 * S))
            add("K=V update", *schur(mr, mr, Vs, lower=True, S=S))
    return parts


def totals(parts):
    return sum(p[0] for p in parts.values()), sum(p[1] for p in parts.values())
