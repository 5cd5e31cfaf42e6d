// cf_tourn32.cu -- LU-1 (TournPivot, Alg. 1 step 2; Sec. 7.3) for the FP32
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
//     ballot), eight packed 64-bit warp keys in shared memory, and only the
//     winning row is written to shared memory (its live part), so the
//     shared-memory traffic per column is one row, not one per warp;
//   * the CTA that finishes a node second climbs to the parent (atomic
//     counter), so no CTA waits for another.
// FP32 with FMA: the mixed path's pivots are reported, not held to bit
// equality with the FP64 oracle.
#include <climits>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_regrow.cuh"

namespace cf {

constexpr int kT2 = 256;                 // rows per unit = threads per CTA
constexpr int kT2Warps = kT2 / 32;

struct T2Smem {
    float4 prow[kMaxV / 4];               // the current pivot row (relative to the block start)
    unsigned wkey[kT2Warps];              // each warp's largest key
    float rinv;                           // 1 / pivot
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

// Masked partial-pivoting selection on the rows held by this CTA's threads
// (thread r holds stacked row r if r < s.nrows).  s.order[0..npiv) = stacked
// indices of the pivots.  Per column:
//   warp maximum of the keys (redux.sync) and its smallest lane (ballot);
//   barrier; every warp takes the maximum of the eight warp keys the same
//   way (lane q reads warp q's key), so ties go to the smallest warp, then
//   the smallest lane: the smallest stacked row;
//   the winner publishes the live part of its row and 1 / pivot; barrier;
//   every remaining row applies the rank-1 update with l = a * (1 / pivot)
//   (FP32 selection only: the factors are recomputed from the original rows).
struct TournStep {
    T2Smem &s;
    float2 (&a)[kPairs];
    int w, r, lane, warp;
    bool used;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int j = j0 + U;
        const float aj = pair_elem<U>(a);
        const unsigned k = key32u(aj, used);
        const unsigned m = __reduce_max_sync(0xffffffffu, k);
        const int wl = __ffs(__ballot_sync(0xffffffffu, k == m)) - 1;
        if (lane == 0) s.wkey[warp] = m;
        __syncthreads();
        const unsigned kk = s.wkey[lane & (kT2Warps - 1)];
        const unsigned gm = __reduce_max_sync(0xffffffffu, kk);
        const int wb = __ffs(__ballot_sync(0xffffffffu, kk == gm)) - 1;
        if (warp == wb && lane == wl) {
            store_live_pairs<U>(s.prow, a, w - j0);
            s.rinv = aj != 0.f ? 1.0f / aj : 0.f;      // zero pivot: no elimination
            s.order[j] = r;
            used = true;
        }
        __syncthreads();
        if (!used) {
            const float ri = s.rinv;
            if (ri != 0.f) rank1_pairs<U>(a, aj * ri, s.prow, w - j0);
        }
    }
};

__device__ void gepp_select_t2(T2Smem &s, float2 (&a)[kPairs], int w, int npiv) {
    const int r = threadIdx.x;
    TournStep body{s, a, w, r, r & 31, r >> 5, !(r < s.nrows)};
    for_blocks_pairs(a, npiv, w, body);
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
            load_row32(a, P, ldp, tid < nr ? s.rows[tid] : 0, w, tid < nr);
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
    if (leaf_h < 1 || leaf_h > 256) return -5;
    if (arity != 2) return -6;
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
    return launch_tourn32(panel, ldp, m, w, leaf_h, arity, ws, ep, stream);
}
