// cf_tourn32w.cu -- LU-1 (TournPivot, Alg. 1 step 2; Sec. 7.3) for the FP32
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

template <int NT>
struct Smem {
    static constexpr int NW = NT / 32;
    // column U of the current block of 8: each warp's candidate (its eight
    // in-block values), key and 1 / its value
    float4 slot[kBlk][NW][2];
    alignas(16) unsigned wkey[kBlk][NW];
    alignas(16) float wrinv[kBlk][NW];
    // block end: pivot U's row at the block start (columns 8 on, relative to
    // the block; padded stride against bank conflicts) and its multipliers
    // with respect to pivots 0..U-1 of the block
    float4 prow[kBlk][kW / 4 + 1];
    float lmat[kBlk][kBlk];
    int order[kW];
    int rows[NT];
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

// The largest of the NW warp keys (smallest warp on ties) and the reciprocal
// published with it, computed by every warp alike: lane i reads warp i's key,
// one redux.sync gives the maximum and a ballot its smallest warp, whose
// reciprocal is one broadcast load.
template <int NW>
__device__ __forceinline__ int warp_argmax(const unsigned (&wk)[NW], const float (&wr)[NW], int lane, float &rinv) {
    const unsigned k = lane < NW ? wk[lane] : 0u;
    const unsigned mx = __reduce_max_sync(0xffffffffu, k);
    const int wb = __ffs(__ballot_sync(0xffffffffu, k == mx)) - 1;
    rinv = wr[wb];
    return wb;
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

template <int NT>
struct BlockStep {
    static constexpr int NW = NT / 32;
    Smem<NT> &s;
    float2 (&a)[kWP];
    float (&lb)[kBlk];
    int w, r, lane, warp, pidx;
    bool used;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int j = j0 + U;
        const float aj = elem<U>(a);
        const unsigned k = key32u(aj, used);
        const unsigned m = __reduce_max_sync(0xffffffffu, k);
        const int wl = __ffs(__ballot_sync(0xffffffffu, k == m)) - 1;
        if (lane == wl) {
            s.slot[U][warp][0] = make_float4(a[0].x, a[0].y, a[1].x, a[1].y);
            s.slot[U][warp][1] = make_float4(a[2].x, a[2].y, a[3].x, a[3].y);
            s.wkey[U][warp] = m;
            s.wrinv[U][warp] = aj != 0.f ? rcp_fast(aj) : 0.f;   // zero pivot: no elimination
        }
        __syncthreads();
        float ri;
        const int wb = warp_argmax<NW>(s.wkey[U], s.wrinv[U], lane, ri);
        if (warp == wb && lane == wl) {
            s.order[j] = r;
            used = true;
            pidx = U;
        }
        if (!used) {
            const float l = ri != 0.f ? aj * ri : 0.f;
            lb[U] = l;
            if (ri != 0.f) {
                const float2 nl = make_float2(-l, -l);
                const float4 u0 = s.slot[U][wb][0], u1 = s.slot[U][wb][1];
                if (1 > U) a[0] = __ffma2_rn(nl, make_float2(u0.x, u0.y), a[0]);
                if (3 > U) a[1] = __ffma2_rn(nl, make_float2(u0.z, u0.w), a[1]);
                if (5 > U) a[2] = __ffma2_rn(nl, make_float2(u1.x, u1.y), a[2]);
                if (7 > U) a[3] = __ffma2_rn(nl, make_float2(u1.z, u1.w), a[3]);
            }
        }
    }
    // Deferred update of the columns past the block (relative 8 .. w - j0).
    __device__ __forceinline__ void block_end(int j0) {
        const int lim = w - j0;
        if (pidx >= 0) {
#pragma unroll
            for (int t = 0; t < kBlk - 1; ++t)
                if (t < pidx) s.lmat[pidx][t] = lb[t];
            float4 *dst = s.prow[pidx];
#pragma unroll
            for (int c = 0; c < kW / 32; ++c)
                if (c * 32 < lim) {
#pragma unroll
                    for (int q = c * 8; q < c * 8 + 8; ++q)
                        if (q >= 2) dst[q] = make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y);
                }
        }
        __syncthreads();
        if (!used) {
            float c[kBlk];
#pragma unroll
            for (int u = kBlk - 1; u >= 0; --u) {
                float t = lb[u];
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
                        for (int q = ch * 8; q < ch * 8 + 8; ++q) {
                            if (q < 2) continue;
                            const float4 p = s.prow[u][q];
                            a[2 * q] = __ffma2_rn(nc, make_float2(p.x, p.y), a[2 * q]);
                            a[2 * q + 1] = __ffma2_rn(nc, make_float2(p.z, p.w), a[2 * q + 1]);
                        }
                    }
            }
        }
#pragma unroll
        for (int u = 0; u < kBlk; ++u) lb[u] = 0.f;
        pidx = -1;
    }
};

// Masked partial-pivoting selection of npiv pivots among the rows held by
// this CTA (thread r holds stacked row r if r < s.nrows); s.order[0..npiv)
// receives the stacked indices of the pivots in pivot order.
template <int NT>
__device__ void gepp_select(Smem<NT> &s, float2 (&a)[kWP], int w, int npiv) {
    const int r = threadIdx.x;
    float lb[kBlk];
#pragma unroll
    for (int u = 0; u < kBlk; ++u) lb[u] = 0.f;
    BlockStep<NT> body{s, a, lb, w, r, r & 31, r >> 5, -1, !(r < s.nrows)};
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
        shift_row(a, w - j0 - kBlk);
    }
    __syncthreads();
}

// LAPACK interchanges and the list of moved rows, from the root's winners
// (panel rows in pivot order): winner j moves from its current position to
// k0 + j.  Positions 0..w-1 are the pivot block, w + j stands for winner j's
// original row when that row lies below the block.
template <int NT>
__device__ void root_epilogue(Smem<NT> &s, const int *win, int np, const TournEpilogue &ep) {
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

template <int NT>
__global__ void __launch_bounds__(NT, 1)
k_tourn32w(const float *__restrict__ P, int ldp, TournPlan plan, TournWS ws, TournEpilogue ep) {
    __shared__ Smem<NT> s;
    const int tid = threadIdx.x;
    const int w = plan.w;
    const int ar = plan.arity;
    float2 a[kWP];

    // ---- leaf: h consecutive rows of the panel
    const int leaf = blockIdx.x;
    {
        const int row0 = leaf * plan.h;
        const int nr = min(plan.h, plan.m - row0);
        const bool valid = tid < nr;
        if (tid == 0) s.nrows = nr;
        s.rows[tid] = row0 + tid;
        const size_t rr = valid ? (size_t)(row0 + tid) : 0;
#pragma unroll
        for (int k = 0; k < kWP; ++k) {
            const float x = (valid && 2 * k < w) ? P[rr + (size_t)(2 * k) * ldp] : 0.f;
            const float y = (valid && 2 * k + 1 < w) ? P[rr + (size_t)(2 * k + 1) * ldp] : 0.f;
            a[k] = make_float2(x, y);
        }
        if (ws.rows32 != nullptr && valid && plan.nlevels > 1) {   // original rows for the playoff nodes
            float4 *dst = reinterpret_cast<float4 *>(ws.rows32 + rr * kW);
#pragma unroll
            for (int q = 0; q < kW / 4; ++q)
                dst[q] = make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y);
        }
        __syncthreads();
        const int np = min(nr, w);
        gepp_select<NT>(s, a, w, np);
        int *dst = ws.node_win + (size_t)(plan.off[0] + leaf) * kMaxV;
        if (tid < np) dst[tid] = s.rows[s.order[tid]];
        if (tid == 0) ws.node_cnt[plan.off[0] + leaf] = np;
        if (plan.nlevels == 1) {
            __syncthreads();
            if (tid < np) ws.root_win[tid] = dst[tid];
            __syncthreads();
            root_epilogue<NT>(s, dst, np, ep);
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
            // stacked row tid: child c, position tid - (counts of children < c)
            int nr = 0, mine = -1;
            for (int c = 0; c < nchild; ++c) {
                const int cc = s.ccnt[c];
                if (mine < 0 && tid < nr + cc) mine = __ldcg(ws.node_win + (size_t)(s0 + c) * kMaxV + (tid - nr));
                nr += cc;
            }
            np = min(nr, w);
            if (tid < nr) s.rows[tid] = mine;
            if (tid == 0) s.nrows = nr;
            if (ws.rows32 != nullptr) {            // contiguous original rows (the leaves' copy)
                const float4 *src = reinterpret_cast<const float4 *>(ws.rows32 + (size_t)(tid < nr ? mine : 0) * kW);
#pragma unroll
                for (int q = 0; q < kW / 4; ++q) {
                    const float4 v = tid < nr ? __ldcg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                    a[2 * q] = make_float2(v.x, v.y);
                    a[2 * q + 1] = make_float2(v.z, v.w);
                }
            } else {
                const bool valid = tid < nr;
                const size_t rr = valid ? (size_t)mine : 0;
#pragma unroll
                for (int k = 0; k < kWP; ++k) {
                    const float x = (valid && 2 * k < w) ? P[rr + (size_t)(2 * k) * ldp] : 0.f;
                    const float y = (valid && 2 * k + 1 < w) ? P[rr + (size_t)(2 * k + 1) * ldp] : 0.f;
                    a[k] = make_float2(x, y);
                }
            }
            __syncthreads();
            gepp_select<NT>(s, a, w, np);
            if (tid < np) dst[tid] = s.rows[s.order[tid]];
            if (tid == 0) ws.node_cnt[node] = np;
        }
        if (level == plan.nlevels - 1) {
            __syncthreads();
            if (tid < np) ws.root_win[tid] = dst[tid];
            __syncthreads();
            root_epilogue<NT>(s, dst, np, ep);
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
    // one thread per candidate row: 256 threads when no leaf or node holds
    // more than 256 rows
    const bool small = h <= 256 && (plan.nlevels == 1 || arity * w <= 256);
    if (small)
        tw::k_tourn32w<256><<<plan.nleaves, 256, 0, st>>>(P, ldp, plan, ws, ep);
    else
        tw::k_tourn32w<512><<<plan.nleaves, 512, 0, st>>>(P, ldp, plan, ws, ep);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

}  // namespace cf
