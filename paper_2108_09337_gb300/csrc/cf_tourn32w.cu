// cf_tourn32w.cu -- LU-1 (TournPivot, Alg. 1; Sec. 7.3) for the FP32
// panels of the mixed-precision LU at block size v <= 64: few, wide tree
// levels.
//
// A panel's tournament is a chain of (tree levels + 1) partial-pivoting
// eliminations, each a chain of v column steps whose latency (a barrier, a
// CTA-wide argmax and the row updates) does not shrink with the number of
// rows.  A row of v <= 64 FP32 values takes 64 registers, so one CTA of 512
// threads holds 512 candidate rows, one per thread: leaves of up to 512 rows
// and playoff nodes that stack the winners of up to 8 children (8 x 64 rows).
// At m = 32768, h = 512 and arity 8 a panel needs 3 eliminations of 64
// columns (64 leaves -> 8 nodes -> root), against 8 of 128 columns for
// v = 128 with 256-row leaves and a binary tree.
//
// Same selection rule as the FP64 tournament and the oracle (leaves of h
// consecutive rows of the current panel, playoff nodes on the original panel
// values of their children's winners stacked in child order, ties to the
// smallest stacked position, a group with one child passes its winners up),
// and the same per-node elimination as the v = 128 FP32 kernel: per column a
// warp maximum of integer keys (redux.sync), each warp's candidate
// publishes its in-block values before the column's only barrier, every
// thread takes the CTA maximum from the warp keys, the in-block columns are
// updated per column and the rest of each row once per block of 8 columns
// with the algebraically identical rank-8 form a -= sum_U c_U a^_U,
// c^T (I + L) = l^T.  Pivot rows are not updated once chosen (only the
// selection is used; the factors are recomputed from the original rows).
#include <climits>
#include <vector>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_regrow.cuh"

namespace cf {

namespace tw {

constexpr int kW = 64;                 // row width: columns of a panel, at most
constexpr int kWP = kW / 2;            // float2 pairs per row
constexpr int kMaxArity = 8;

// NT threads hold RPT rows each: stacked row p = q * NT + thread (q < RPT),
// so the smallest stacked position is the smallest q, then the smallest
// thread.
template <int NT, int RPT>
struct Smem {
    static constexpr int NW = NT / 32;
    // column U of the current block of 8: each warp's candidate (its eight
    // in-block values), key, 1 / its value and stacked position
    float4 slot[kBlk][NW][2];
    alignas(16) unsigned wkey[kBlk][NW];
    alignas(16) float wrinv[kBlk][NW];
    alignas(16) unsigned wpos[kBlk][NW];
    // block end: pivot U's row at the block start (columns 8 on, relative to
    // the block; padded stride against bank conflicts) and its multipliers
    // with respect to pivots 0..U-1 of the block
    float4 prow[kBlk][kW / 4 + 1];
    float lmat[kBlk][kBlk];
    int order[kW];
    int rows[NT * RPT];
    int ccnt[kMaxArity];
    int nrows;
    int cont;
    int lab_at[2 * kW];
    int where_[2 * kW];
};

__device__ __forceinline__ unsigned key32u(float a, bool used) {
    const float x = fabsf(a);
    return used ? 0u : ((x != x) ? 1u : __float_as_uint(x) + 2u);
}

__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int U>
__device__ __forceinline__ float elem(const float2 (&a)[kWP]) {
    return (U & 1) ? a[U >> 1].y : a[U >> 1].x;
}

// Shift the row left by one block of 8 columns; 32-column chunks beyond the
// live width `lim` (relative to the new block start) are left alone.
__device__ __forceinline__ void shift_row(float2 (&a)[kWP], int lim) {
#pragma unroll
    for (int c = 0; c < kW / 32; ++c) {
        if (c * 32 < lim) {
#pragma unroll
            for (int p = c * 16; p < c * 16 + 16; ++p)
                if (p + kBlk / 2 < kWP) a[p] = a[p + kBlk / 2];
        }
    }
}

template <int NT, int RPT>
struct BlockStep {
    static constexpr int NW = NT / 32;
    Smem<NT, RPT> &s;
    float2 (&a)[RPT][kWP];
    float (&lb)[RPT][kBlk];
    bool (&used)[RPT];
    int (&pidx)[RPT];
    int w, tid, lane, warp;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int j = j0 + U;
        float aj[RPT];
        unsigned k[RPT];
        unsigned kk = 0u;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            aj[q] = elem<U>(a[q]);
            k[q] = key32u(aj[q], used[q]);
            kk = k[q] > kk ? k[q] : kk;
        }
        // warp maximum; its smallest stacked position: the first q, then lane
        const unsigned m = __reduce_max_sync(0xffffffffu, kk);
        int wq = 0;
        unsigned bal = __ballot_sync(0xffffffffu, k[0] == m);
#pragma unroll
        for (int q = 1; q < RPT; ++q) {
            const unsigned b = __ballot_sync(0xffffffffu, k[q] == m);
            if (bal == 0u) { bal = b; wq = q; }
        }
        const int wl = __ffs(bal) - 1;
        if (lane == wl) {
#pragma unroll
            for (int q = 0; q < RPT; ++q)
                if (q == wq) {
                    s.slot[U][warp][0] = make_float4(a[q][0].x, a[q][0].y, a[q][1].x, a[q][1].y);
                    s.slot[U][warp][1] = make_float4(a[q][2].x, a[q][2].y, a[q][3].x, a[q][3].y);
                    s.wrinv[U][warp] = aj[q] != 0.f ? rcp_fast(aj[q]) : 0.f;   // zero pivot: no elimination
                }
            s.wkey[U][warp] = m;
            s.wpos[U][warp] = (unsigned)(wq * NT + tid);
        }
        __syncthreads();
        // CTA maximum over the warp keys (lane i reads warp i's), then the
        // smallest stacked position among the warps that hold it (with one
        // row per thread, the smallest such warp)
        const unsigned wk = lane < NW ? s.wkey[U][lane] : 0u;
        const unsigned M = __reduce_max_sync(0xffffffffu, wk);
        unsigned P;
        int wb;
        if constexpr (RPT == 1) {
            // the winning warp is the first that holds M: its position, 1 /
            // pivot and in-block values are loaded together
            wb = __ffs(__ballot_sync(0xffffffffu, wk == M)) - 1;
            P = s.wpos[U][wb];
        } else {
            const unsigned cand = (lane < NW && wk == M) ? s.wpos[U][lane] : 0xffffffffu;
            P = __reduce_min_sync(0xffffffffu, cand);
            wb = (int)(P % NT) >> 5;
        }
        const float ri = s.wrinv[U][wb];
        const float4 u0 = s.slot[U][wb][0], u1 = s.slot[U][wb][1];
        const int pt = (int)(P % NT), pq = (int)(P / NT);
        if (tid == pt) {
            s.order[j] = (int)P;
#pragma unroll
            for (int q = 0; q < RPT; ++q)
                if (q == pq) { used[q] = true; pidx[q] = U; }
        }
        if (ri != 0.f) {
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                if (used[q]) continue;
                const float l = aj[q] * ri;
                lb[q][U] = l;
                const float2 nl = make_float2(-l, -l);
                if (1 > U) a[q][0] = __ffma2_rn(nl, make_float2(u0.x, u0.y), a[q][0]);
                if (3 > U) a[q][1] = __ffma2_rn(nl, make_float2(u0.z, u0.w), a[q][1]);
                if (5 > U) a[q][2] = __ffma2_rn(nl, make_float2(u1.x, u1.y), a[q][2]);
                if (7 > U) a[q][3] = __ffma2_rn(nl, make_float2(u1.z, u1.w), a[q][3]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < RPT; ++q)
                if (!used[q]) lb[q][U] = 0.f;
        }
    }
    // Deferred update of the columns past the block (relative 8 .. w - j0).
    __device__ __forceinline__ void block_end(int j0) {
        const int lim = w - j0;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            if (pidx[q] < 0) continue;
            const int pu = pidx[q];
#pragma unroll
            for (int t = 0; t < kBlk - 1; ++t)
                if (t < pu) s.lmat[pu][t] = lb[q][t];
            float4 *dst = s.prow[pu];
#pragma unroll
            for (int c = 0; c < kW / 32; ++c)
                if (c * 32 < lim) {
#pragma unroll
                    for (int g = c * 8; g < c * 8 + 8; ++g)
                        if (g >= 2)
                            dst[g] = make_float4(a[q][2 * g].x, a[q][2 * g].y, a[q][2 * g + 1].x, a[q][2 * g + 1].y);
                }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            if (used[q]) continue;
            float c[kBlk];
#pragma unroll
            for (int u = kBlk - 1; u >= 0; --u) {
                float t = lb[q][u];
#pragma unroll
                for (int u2 = u + 1; u2 < kBlk; ++u2) t = fmaf(-c[u2], s.lmat[u2][u], t);
                c[u] = t;
            }
#pragma unroll
            for (int u = 0; u < kBlk; ++u) {
                const float2 nc = make_float2(-c[u], -c[u]);
#pragma unroll
                for (int ch = 0; ch < kW / 32; ++ch)
                    if (ch * 32 < lim) {
#pragma unroll
                        for (int g = ch * 8; g < ch * 8 + 8; ++g) {
                            if (g < 2) continue;
                            const float4 p = s.prow[u][g];
                            a[q][2 * g] = __ffma2_rn(nc, make_float2(p.x, p.y), a[q][2 * g]);
                            a[q][2 * g + 1] = __ffma2_rn(nc, make_float2(p.z, p.w), a[q][2 * g + 1]);
                        }
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
#pragma unroll
            for (int u = 0; u < kBlk; ++u) lb[q][u] = 0.f;
            pidx[q] = -1;
        }
    }
};

// Masked partial-pivoting selection of npiv pivots among the rows held by
// this CTA (stacked row p lives in thread p % NT as its row p / NT, valid if
// p < s.nrows); s.order[0..npiv) receives the stacked indices of the pivots
// in pivot order.
template <int NT, int RPT>
__device__ void gepp_select(Smem<NT, RPT> &s, float2 (&a)[RPT][kWP], int w, int npiv) {
    const int tid = threadIdx.x;
    float lb[RPT][kBlk];
    bool used[RPT];
    int pidx[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
#pragma unroll
        for (int u = 0; u < kBlk; ++u) lb[q][u] = 0.f;
        used[q] = !(q * NT + tid < s.nrows);
        pidx[q] = -1;
    }
    BlockStep<NT, RPT> body{s, a, lb, used, pidx, w, tid, tid & 31, tid >> 5};
    for (int j0 = 0; j0 < npiv; j0 += kBlk) {
        body.template step<0>(j0);
        if (j0 + 1 < npiv) body.template step<1>(j0);
        if (j0 + 2 < npiv) body.template step<2>(j0);
        if (j0 + 3 < npiv) body.template step<3>(j0);
        if (j0 + 4 < npiv) body.template step<4>(j0);
        if (j0 + 5 < npiv) body.template step<5>(j0);
        if (j0 + 6 < npiv) body.template step<6>(j0);
        if (j0 + 7 < npiv) body.template step<7>(j0);
        if (j0 + kBlk >= npiv) break;              // no selection left: skip the update
        body.block_end(j0);
#pragma unroll
        for (int q = 0; q < RPT; ++q) shift_row(a[q], w - j0 - kBlk);
    }
    __syncthreads();
}

// LAPACK interchanges and the list of moved rows, from the root's winners
// (panel rows in pivot order): winner j moves from its current position to
// k0 + j.  Positions 0..w-1 are the pivot block, w + j stands for winner j's
// original row when that row lies below the block.
template <int NT, int RPT>
__device__ void root_epilogue(Smem<NT, RPT> &s, const int *win, int np, const TournEpilogue &ep) {
    if (ep.ipiv == nullptr || threadIdx.x != 0) return;
    const int w = np;
    for (int q = 0; q < 2 * w; ++q) { s.lab_at[q] = q; s.where_[q] = q; }
    for (int j = 0; j < w; ++j) {
        const int hj = win[j] < w ? win[j] : w + j;
        const int ps = s.where_[hj];
        const int p = ps < w ? ps : win[ps - w];
        ep.ipiv[ep.k0 + j] = ep.k0 + p + 1;
        if (ps != j) {
            const int hx = s.lab_at[j];
            s.lab_at[j] = hj; s.where_[hj] = j;
            s.lab_at[ps] = hx; s.where_[hx] = ps;
        }
    }
    int cnt = 0;
    for (int q = 0; q < 2 * w; ++q) {
        if (s.lab_at[q] == q) continue;
        const int hq = s.lab_at[q];
        ep.swap_dst[cnt] = q < w ? q : win[q - w];
        ep.swap_src[cnt] = hq < w ? hq : win[hq - w];
        ++cnt;
    }
    *ep.swap_cnt = cnt;
}

__device__ __forceinline__ void load_row64(float2 (&a)[kWP], const float *__restrict__ P, int ldp, size_t row, int w,
                                           bool valid) {
#pragma unroll
    for (int k = 0; k < kWP; ++k) {
        const float x = (valid && 2 * k < w) ? P[row + (size_t)(2 * k) * ldp] : 0.f;
        const float y = (valid && 2 * k + 1 < w) ? P[row + (size_t)(2 * k + 1) * ldp] : 0.f;
        a[k] = make_float2(x, y);
    }
}

template <int NT, int RPT>
__global__ void __launch_bounds__(NT, 1)
k_tourn32w(const float *__restrict__ P, int ldp, TournPlan plan, TournWS ws, TournEpilogue ep) {
    __shared__ Smem<NT, RPT> s;
    const int tid = threadIdx.x;
    const int w = plan.w;
    const int ar = plan.arity;
    float2 a[RPT][kWP];

    // ---- leaf: h consecutive rows of the panel
    const int leaf = blockIdx.x;
    {
        const int row0 = leaf * plan.h;
        const int nr = min(plan.h, plan.m - row0);
        if (tid == 0) s.nrows = nr;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int p = q * NT + tid;
            const bool valid = p < nr;
            s.rows[p] = row0 + p;
            const size_t rr = valid ? (size_t)(row0 + p) : 0;
            load_row64(a[q], P, ldp, rr, w, valid);
            if (ws.rows32 != nullptr && valid && plan.nlevels > 1) {   // original rows for the playoff nodes
                float4 *dst = reinterpret_cast<float4 *>(ws.rows32 + rr * kW);
#pragma unroll
                for (int g = 0; g < kW / 4; ++g)
                    dst[g] = make_float4(a[q][2 * g].x, a[q][2 * g].y, a[q][2 * g + 1].x, a[q][2 * g + 1].y);
            }
        }
        __syncthreads();
        const int np = min(nr, w);
        gepp_select<NT, RPT>(s, a, w, np);
        int *dst = ws.node_win + (size_t)(plan.off[0] + leaf) * kMaxV;
        if (tid < np) dst[tid] = s.rows[s.order[tid]];
        if (tid == 0) ws.node_cnt[plan.off[0] + leaf] = np;
        if (plan.nlevels == 1) {
            __syncthreads();
            if (tid < np) ws.root_win[tid] = dst[tid];
            __syncthreads();
            root_epilogue<NT, RPT>(s, dst, np, ep);
            return;
        }
    }
    // ---- playoff nodes: the last of a group's children to finish climbs
    int level = 0, g = leaf;
    while (true) {
        const int parent = g / ar;
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const int pnode = plan.off[level + 1] + parent;
            const int pch = min(ar, plan.cnt[level] - parent * ar);
            const int old = atomicAdd(ws.counter + pnode, 1);
            const int cont = (old == pch - 1);
            if (cont) ws.counter[pnode] = 0;     // leave the counter clean
            s.cont = cont;
        }
        __syncthreads();
        if (!s.cont) return;
        __threadfence();
        ++level;
        g = parent;
        const int child0 = g * ar;
        const int nchild = min(ar, plan.cnt[level - 1] - child0);
        const int node = plan.off[level] + g;
        const int s0 = plan.off[level - 1] + child0;
        int *dst = ws.node_win + (size_t)node * kMaxV;
        int np;
        if (nchild == 1) {
            np = __ldcg(ws.node_cnt + s0);
            if (tid < np) dst[tid] = __ldcg(ws.node_win + (size_t)s0 * kMaxV + tid);
            if (tid == 0) ws.node_cnt[node] = np;
        } else {
            if (tid < nchild) s.ccnt[tid] = __ldcg(ws.node_cnt + s0 + tid);
            __syncthreads();
            // stacked row p: child c, position p - (counts of children < c)
            int nr = 0, mine[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q) mine[q] = -1;
            for (int c = 0; c < nchild; ++c) {
                const int cc = s.ccnt[c];
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    const int p = q * NT + tid;
                    if (mine[q] < 0 && p < nr + cc)
                        mine[q] = __ldcg(ws.node_win + (size_t)(s0 + c) * kMaxV + (p - nr));
                }
                nr += cc;
            }
            np = min(nr, w);
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int p = q * NT + tid;
                const bool valid = p < nr;
                if (valid) s.rows[p] = mine[q];
                if (ws.rows32 != nullptr) {            // contiguous original rows (the leaves' copy)
                    const float4 *src = reinterpret_cast<const float4 *>(ws.rows32 + (size_t)(valid ? mine[q] : 0) * kW);
#pragma unroll
                    for (int g2 = 0; g2 < kW / 4; ++g2) {
                        const float4 v = valid ? __ldcg(src + g2) : make_float4(0.f, 0.f, 0.f, 0.f);
                        a[q][2 * g2] = make_float2(v.x, v.y);
                        a[q][2 * g2 + 1] = make_float2(v.z, v.w);
                    }
                } else {
                    load_row64(a[q], P, ldp, valid ? (size_t)mine[q] : 0, w, valid);
                }
            }
            if (tid == 0) s.nrows = nr;
            __syncthreads();
            gepp_select<NT, RPT>(s, a, w, np);
            if (tid < np) dst[tid] = s.rows[s.order[tid]];
            if (tid == 0) ws.node_cnt[node] = np;
        }
        if (level == plan.nlevels - 1) {
            __syncthreads();
            if (tid < np) ws.root_win[tid] = dst[tid];
            __syncthreads();
            root_epilogue<NT, RPT>(s, dst, np, ep);
            return;
        }
    }
}

}  // namespace tw

// The shapes this kernel takes: w <= 64, leaves of up to 512 rows, arity up
// to 8 with arity * w <= 512 (every node's candidates fit one CTA).
bool tourn32w_supported(int w, int h, int arity) {
    return w >= 0 && w <= tw::kW && h >= 1 && h <= 512 && arity >= 2 && arity <= tw::kMaxArity &&
           arity * (w > 0 ? w : 1) <= 512;
}

int launch_tourn32w(const float *P, int ldp, int m, int w, int h, int arity, const TournWS &ws,
                    const TournEpilogue &ep, cudaStream_t st) {
    if (!tourn32w_supported(w, h, arity) || m < 0) return CF_ERR_UNSUPPORTED;
    if (m == 0 || w == 0) return CF_OK;
    TournPlan plan{};
    int rc = make_tourn_plan(m, w, h, arity, &plan);
    if (rc != CF_OK) return rc;
    // one candidate row per thread: 256 threads when no leaf or node holds
    // more than 256 rows, else 512 (two rows per thread on 256 threads, with
    // half the warps in each barrier and reduction, measured 9% slower: the
    // column chain is latency-bound, not issue-bound)
    const bool small = h <= 256 && (plan.nlevels == 1 || arity * w <= 256);
    if (small)
        tw::k_tourn32w<256, 1><<<plan.nleaves, 256, 0, st>>>(P, ldp, plan, ws, ep);
    else
        tw::k_tourn32w<512, 1><<<plan.nleaves, 512, 0, st>>>(P, ldp, plan, ws, ep);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

}  // namespace cf
