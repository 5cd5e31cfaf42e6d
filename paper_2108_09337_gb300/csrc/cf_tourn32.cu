// cf_tourn32.cu -- LU-1 (TournPivot, Alg. 1; Sec. 7.3) for the FP32
// panels of the mixed-precision path.
//
// Same rule as the FP64 tournament (leaves of h consecutive rows, binary
// playoff nodes on the original panel values of the stacked candidates, ties
// to the smallest stacked position), built for latency:
//   * one CTA of 256 threads is a whole leaf (h <= 256) or a whole node
//     (2 x 128 candidates); each thread holds one row in registers, indexed
//     relative to the current block of 8 columns (cf_regrow.cuh), so all
//     register indices are compile-time constants;
//   * per column: a warp maximum of integer keys (one redux.sync and a
//     ballot); each warp's candidate publishes its row before the column's
//     only barrier, so the winner's row is readable right after it;
//   * the CTA that finishes a node second climbs to the parent (atomic
//     counter), so no CTA waits for another;
//   * with a rows32 workspace the leaves also write their rows' original
//     values row-major, so a playoff node reads each candidate row as 32
//     contiguous 16-byte loads instead of 128 loads from a scattered row of
//     the column-major panel (an eighth of the L2 sectors).
// FP32 with FMA: the mixed path's pivots are reported, not held to bit
// equality with the FP64 oracle.
#include <climits>
#include <vector>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_regrow.cuh"

namespace cf {

constexpr int kT2 = 256;                 // rows per unit = threads per CTA
constexpr int kT2Warps = kT2 / 32;

struct T2Smem {
    // Column U of the current block of 8: each warp's candidate (its in-block
    // values, key and 1 / its value).
    float4 slot[kBlk][kT2Warps][2];
    alignas(16) unsigned wkey[kBlk][kT2Warps];
    alignas(16) float wrinv[kBlk][kT2Warps];
    // Block end: pivot U's row at the block start (relative to the block,
    // columns 8 on; stride padded against bank conflicts) and its
    // multipliers with respect to pivots 0..U-1 of the block.
    float4 prow[kBlk][kMaxV / 4 + 1];
    float lmat[kBlk][kBlk];
    int order[kMaxV];
    int rows[kT2];
    int nrows;
    int cont;
    int lab_at[2 * kMaxV];
    int where_[2 * kMaxV];
};

// Candidate key as an unsigned integer with the selection order
// used < NaN < |a| (non-negative floats order like their bit patterns), so a
// maximum is one redux.sync.
__device__ __forceinline__ unsigned key32u(float a, bool used) {
    const float x = fabsf(a);
    return used ? 0u : ((x != x) ? 1u : __float_as_uint(x) + 2u);
}

// Fast reciprocal (MUFU, relative error ~2^-23): the multipliers only steer
// the selection, whose factors are recomputed from the original rows.
__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The largest of eight warp keys (smallest index on ties) and the reciprocal
// published with it, from four broadcast loads and a three-level comparison
// tree in registers.
__device__ __forceinline__ int warp_argmax8(const unsigned (&wk)[kT2Warps], const float (&wr)[kT2Warps], float &rinv) {
    const uint4 k0 = *reinterpret_cast<const uint4 *>(&wk[0]);
    const uint4 k1 = *reinterpret_cast<const uint4 *>(&wk[4]);
    const float4 r0 = *reinterpret_cast<const float4 *>(&wr[0]);
    const float4 r1 = *reinterpret_cast<const float4 *>(&wr[4]);
    const bool c01 = k0.y > k0.x, c23 = k0.w > k0.z, c45 = k1.y > k1.x, c67 = k1.w > k1.z;
    const unsigned a01 = c01 ? k0.y : k0.x, a23 = c23 ? k0.w : k0.z;
    const unsigned a45 = c45 ? k1.y : k1.x, a67 = c67 ? k1.w : k1.z;
    const float f01 = c01 ? r0.y : r0.x, f23 = c23 ? r0.w : r0.z, f45 = c45 ? r1.y : r1.x, f67 = c67 ? r1.w : r1.z;
    const int i01 = c01 ? 1 : 0, i23 = c23 ? 3 : 2, i45 = c45 ? 5 : 4, i67 = c67 ? 7 : 6;
    const bool d0 = a23 > a01, d1 = a67 > a45;
    const unsigned b0 = d0 ? a23 : a01, b1 = d1 ? a67 : a45;
    const float g0 = d0 ? f23 : f01, g1 = d1 ? f67 : f45;
    const int j0 = d0 ? i23 : i01, j1 = d1 ? i67 : i45;
    const bool e = b1 > b0;
    rinv = e ? g1 : g0;
    return e ? j1 : j0;
}

// Masked partial-pivoting selection on the rows held by this CTA's threads
// (thread r holds stacked row r if r < s.nrows).  s.order[0..npiv) = stacked
// indices of the pivots.  Blocked by 8 columns (a right-looking blocked GEPP
// whose trailing update is deferred to the block end):
//   column U of the block: warp maximum of the keys (redux.sync) and its
//   smallest lane (ballot); that lane publishes its 8 in-block values, key
//   and 1 / value in its warp's slot; barrier; every thread takes the
//   largest of the eight warp keys (smallest warp on ties; within the warp
//   the smallest lane won), so ties go to the smallest stacked row; every remaining row takes l_U = a * (1 / pivot) and updates only its
//   in-block columns.  One barrier and 32 bytes per candidate per column;
//   1 / value is the MUFU approximation (the multipliers only steer the
//   selection).
//   block end (if pivots remain): the eight pivots publish the rest of their
//   rows as they were at the block start, â_U, and their multipliers L with
//   respect to the block's earlier pivots; barrier; every remaining row
//   applies a -= sum_U c_U â_U with c^T (I + L) = l^T, which equals the
//   eight rank-1 updates of unblocked elimination (the pivot rows' own
//   updates u_U = â_U - sum_{U' < U} L(U, U') u_U' folded into c).
// Pivot rows are not updated once chosen: only the selection is used (the
// factors are recomputed from the original rows).
struct TournBlockStep {
    T2Smem &s;
    float2 (&a)[kPairs];
    float (&lb)[kBlk];
    int w, r, lane, warp, pidx;
    bool used;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int j = j0 + U;
        const float aj = pair_elem<U>(a);
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
        const int wb = warp_argmax8(s.wkey[U], s.wrinv[U], ri);
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
            for (int c = 0; c < 4; ++c)
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
            // pivot by pivot, so consecutive FMAs on one element are a row apart
#pragma unroll
            for (int u = 0; u < kBlk; ++u) {
                const float2 nc = make_float2(-c[u], -c[u]);
#pragma unroll
                for (int ch = 0; ch < 4; ++ch)
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

__device__ void gepp_select_t2(T2Smem &s, float2 (&a)[kPairs], int w, int npiv) {
    const int r = threadIdx.x;
    float lb[kBlk];
#pragma unroll
    for (int u = 0; u < kBlk; ++u) lb[u] = 0.f;
    TournBlockStep body{s, a, lb, w, r, r & 31, r >> 5, -1, !(r < s.nrows)};
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
        shift_pairs(a, w - j0 - kBlk);
    }
    __syncthreads();
}

__device__ __forceinline__ void load_row32(float2 (&a)[kPairs], const float *__restrict__ P, int ldp, int row, int w,
                                           bool valid) {
#pragma unroll
    for (int k = 0; k < kPairs; ++k) {
        const float x = (valid && 2 * k < w) ? P[(size_t)row + (size_t)(2 * k) * ldp] : 0.f;
        const float y = (valid && 2 * k + 1 < w) ? P[(size_t)row + (size_t)(2 * k + 1) * ldp] : 0.f;
        a[k] = make_float2(x, y);
    }
}

__device__ void root_epilogue_t2(T2Smem &s, const int *win, int np, const TournEpilogue &ep) {
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

__global__ void __launch_bounds__(kT2, 1)
k_tourn32(const float *__restrict__ P, int ldp, TournPlan plan, TournWS ws, TournEpilogue ep) {
    __shared__ T2Smem s;
    const int tid = threadIdx.x;
    const int w = plan.w;
    float2 a[kPairs];

    // ---- leaf
    const int leaf = blockIdx.x;
    {
        const int row0 = leaf * plan.h;
        const int nr = min(plan.h, plan.m - row0);
        if (tid == 0) s.nrows = nr;
        s.rows[tid] = row0 + tid;
        load_row32(a, P, ldp, row0 + tid, w, tid < nr);
        if (ws.rows32 != nullptr && tid < nr && plan.nlevels > 1) {   // original rows for the playoff nodes
            float4 *dst = reinterpret_cast<float4 *>(ws.rows32 + (size_t)(row0 + tid) * kMaxV);
#pragma unroll
            for (int q = 0; q < kMaxV / 4; ++q)
                dst[q] = make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y);
        }
        __syncthreads();
        const int np = min(nr, w);
        gepp_select_t2(s, a, w, np);
        int *dst = ws.node_win + (size_t)(plan.off[0] + leaf) * kMaxV;
        if (tid < np) dst[tid] = s.rows[s.order[tid]];
        if (tid == 0) ws.node_cnt[plan.off[0] + leaf] = np;
        if (plan.nlevels == 1) {
            __syncthreads();
            if (tid < np) ws.root_win[tid] = dst[tid];
            __syncthreads();
            root_epilogue_t2(s, dst, np, ep);
            return;
        }
    }
    // ---- playoff nodes: the second of two siblings to finish climbs
    int level = 0, g = leaf;
    while (true) {
        const int parent = g >> 1;
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const int pnode = plan.off[level + 1] + parent;
            const int pch = min(2, plan.cnt[level] - parent * 2);
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
        const int child0 = g * 2;
        const int nchild = min(2, plan.cnt[level - 1] - child0);
        const int node = plan.off[level] + g;
        int *dst = ws.node_win + (size_t)node * kMaxV;
        int np;
        if (nchild == 1) {
            const int src = plan.off[level - 1] + child0;
            np = __ldcg(ws.node_cnt + src);
            if (tid < np) dst[tid] = __ldcg(ws.node_win + (size_t)src * kMaxV + tid);
            if (tid == 0) ws.node_cnt[node] = np;
        } else {
            const int s0 = plan.off[level - 1] + child0;
            const int c0 = __ldcg(ws.node_cnt + s0), c1 = __ldcg(ws.node_cnt + s0 + 1);
            const int nr = c0 + c1;
            np = min(nr, w);
            if (tid < c0) s.rows[tid] = __ldcg(ws.node_win + (size_t)s0 * kMaxV + tid);
            else if (tid < nr) s.rows[tid] = __ldcg(ws.node_win + (size_t)(s0 + 1) * kMaxV + (tid - c0));
            if (tid == 0) s.nrows = nr;
            __syncthreads();
            if (ws.rows32 != nullptr) {            // contiguous original rows (the leaves' copy)
                const float4 *src = reinterpret_cast<const float4 *>(ws.rows32 + (size_t)s.rows[tid < nr ? tid : 0] * kMaxV);
#pragma unroll
                for (int q = 0; q < kMaxV / 4; ++q) {
                    const float4 v = tid < nr ? __ldcg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                    a[2 * q] = make_float2(v.x, v.y);
                    a[2 * q + 1] = make_float2(v.z, v.w);
                }
            } else {
                load_row32(a, P, ldp, tid < nr ? s.rows[tid] : 0, w, tid < nr);
            }
            __syncthreads();
            gepp_select_t2(s, a, w, np);
            if (tid < np) dst[tid] = s.rows[s.order[tid]];
            if (tid == 0) ws.node_cnt[node] = np;
        }
        if (level == plan.nlevels - 1) {
            __syncthreads();
            if (tid < np) ws.root_win[tid] = dst[tid];
            __syncthreads();
            root_epilogue_t2(s, dst, np, ep);
            return;
        }
    }
}

// Elimination flops of one FP32 tournament (m x w panel, leaves of h rows,
// `arity` children per playoff node): per GEPP on r rows x w columns,
// sum_j (r-j-1)(2(w-j-1) + 1) for j < min(r, w); nodes with one child pass
// their winners through.
double tourn32_flops(int m, int w, int h, int arity) {
    auto gepp = [w](int r) {
        double f = 0.0;
        const int p = r < w ? r : w;
        for (int j = 0; j < p; ++j) f += (double)(r - j - 1) * (2.0 * (w - j - 1) + 1.0);
        return f;
    };
    if (m <= 0 || w <= 0 || h <= 0) return 0.0;
    std::vector<int> cnt;
    double f = 0.0;
    for (int r0 = 0; r0 < m; r0 += h) {
        const int r = m - r0 < h ? m - r0 : h;
        f += gepp(r);
        cnt.push_back(r < w ? r : w);
    }
    if (arity < 2) arity = 2;
    while (cnt.size() > 1) {
        std::vector<int> up;
        for (size_t i = 0; i < cnt.size(); i += arity) {
            const size_t e = i + arity < cnt.size() ? i + arity : cnt.size();
            if (e - i == 1) { up.push_back(cnt[i]); continue; }
            int r = 0;
            for (size_t c = i; c < e; ++c) r += cnt[c];
            f += gepp(r);
            up.push_back(r < w ? r : w);
        }
        cnt.swap(up);
    }
    return f;
}

bool tourn32_shape_ok(int v, int h, int arity) {
    if (v <= 64) return tourn32w_supported(v, h, arity);
    return v <= kMaxV && h >= 1 && h <= kT2 && arity == 2;
}

int launch_tourn32_any(const float *P, int ldp, int m, int w, int h, int arity, const TournWS &ws,
                       const TournEpilogue &ep, cudaStream_t st) {
    if (w <= 64 && tourn32w_supported(w, h, arity)) return launch_tourn32w(P, ldp, m, w, h, arity, ws, ep, st);
    return launch_tourn32(P, ldp, m, w, h, arity, ws, ep, st);
}

int launch_tourn32(const float *P, int ldp, int m, int w, int h, int arity, const TournWS &ws, const TournEpilogue &ep,
                   cudaStream_t st) {
    if (arity != 2 || h < 1 || h > kT2 || w < 0 || w > kMaxV || m < 0) return CF_ERR_UNSUPPORTED;
    if (m == 0 || w == 0) return CF_OK;
    TournPlan plan{};
    plan.m = m; plan.w = w; plan.h = h; plan.arity = 2;
    plan.nleaves = ceil_div(m, h);
    int c = plan.nleaves, lv = 0, off = 0;
    while (true) {
        if (lv >= kMaxLevels) return CF_ERR_UNSUPPORTED;
        plan.cnt[lv] = c; plan.off[lv] = off; off += c; ++lv;
        if (c <= 1) break;
        c = (c + 1) / 2;
    }
    plan.nlevels = lv;
    plan.total_nodes = off;
    k_tourn32<<<plan.nleaves, kT2, 0, st>>>(P, ldp, plan, ws, ep);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

}  // namespace cf

extern "C" int cf_tourn_select_f32(int m, int w, const float *panel, int ldp, int leaf_h, int arity, int *winners,
                                   void *work, size_t lwork, cudaStream_t stream) {
    using namespace cf;
    if (m < 0) return -1;
    if (w < 0 || w > kMaxV) return -2;
    if (m > 0 && w > 0 && panel == nullptr) return -3;
    if (ldp < (m > 1 ? m : 1)) return -4;
    if (leaf_h < 1 || leaf_h > (w <= 64 ? 512 : kT2)) return -5;
    if (arity < 2 || arity > (w <= 64 ? 8 : 2) || (w <= 64 && !tourn32w_supported(w, leaf_h, arity))) return -6;
    if (m == 0 || w == 0) return CF_OK;
    if (winners == nullptr) return -7;
    if (lwork < cf_tourn_workspace_size(m, w, 1, arity) || work == nullptr) return CF_ERR_WORKSPACE;
    TournWS ws{};
    TournEpilogue ep{};
    int rc = tourn_ws_carve(work, m, 1, arity, &ws, &ep);
    if (rc != CF_OK) return rc;
    ep.ipiv = nullptr;
    CF_CUDA_TRY(cudaMemsetAsync(ws.counter, 0, ws.counter_bytes, stream));
    ws.root_win = winners;
    return launch_tourn32_any(panel, ldp, m, w, leaf_h, arity, ws, ep, stream);
}
