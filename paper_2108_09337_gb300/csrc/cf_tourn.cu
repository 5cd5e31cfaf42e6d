// cf_tourn.cu -- LU-1: TournPivot (Alg. 1; Sec. 7.3 "Tournament
// Pivoting" and "Pivoting in COnfLUX"; the pivot selection in the I/O-cost proof) and
// LU-2: the row interchanges that bring the winners to the top.
//
// GPU design.  One launch runs a whole tournament.  A thread-block cluster of
// `arity` CTAs is the unit of work: in the leaf phase each CTA eliminates its
// own leaf (h consecutive panel rows) in shared memory; in a playoff node the
// cluster's CTAs each hold one child's candidate rows (original panel values)
// and eliminate them together, exchanging the per-column argmax through
// distributed shared memory (one cluster barrier per column).  The cluster
// that finishes a node last (atomic counter, no spinning) climbs to the
// parent, so no CTA ever waits for another; the root cluster writes the
// winners, the LAPACK ipiv and the list of moved rows.
//
// Every elimination step uses separately rounded multiply and subtract and
// an IEEE division, in the same order as the FP64 oracle, so a tournament on
// the same panel bytes picks the same pivots bit for bit.
#include <cooperative_groups.h>

#include <climits>

#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cg = cooperative_groups;

namespace cf {

constexpr int kTournThreads = 256;

template <typename T>
struct TournSmem {
    T tile[kMaxV * kMaxV];      // column-major, ld kMaxV: tile[k*kMaxV + r]
    T prow[kMaxV];              // pivot row of the current column
    T redv[kTournThreads / 32];
    int redi[kTournThreads / 32];
    T slotv[2];                 // this CTA's argmax, by column parity
    int sloti[2];
    int used[kMaxV];
    int order[kMaxV];
    int rows[kMaxV];            // panel row of each tile row
    int nrows;
    int cont;
    int lab_at[2 * kMaxV];      // root epilogue: swap simulation
    int where_[2 * kMaxV];
};

// Key of the argmax: |a|, with NaN ranked below every number but above "no
// candidate" (-1), exactly as the oracle ranks it.
template <typename T>
__device__ __forceinline__ T piv_key(T a) {
    T x = fabs(a);
    return (x != x) ? T(-0.5) : x;
}

template <typename T>
__device__ __forceinline__ void better(T &bv, int &bi, T ov, int oi) {
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
}

// Masked partial-pivoting selection on the stacked rows held by the CTAs of
// the cluster (CLUSTERED) or by this CTA alone.  Stacked index of a row =
// rank * kMaxV + tile row (clustered) or tile row.  Leaves s.order[0..npiv)
// identical in every participating CTA.
template <typename T, bool CLUSTERED, int CL>
__device__ void gepp_select(TournSmem<T> &s, int w, int npiv, int rank) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int base = CLUSTERED ? rank * kMaxV : 0;
    const int r = tid & (kMaxV - 1);
    const int half = tid / kMaxV;      // 0 or 1
    cg::cluster_group cl = cg::this_cluster();
    for (int j = 0; j < npiv; ++j) {
        // (1) local argmax of column j over the unused rows.
        T bv = T(-1);
        int bi = INT_MAX;
        if (tid < kMaxV && tid < s.nrows && !s.used[tid]) {
            bv = piv_key(s.tile[j * kMaxV + tid]);
            bi = base + tid;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            better(bv, bi, ov, oi);
        }
        if (lane == 0) { s.redv[warp] = bv; s.redi[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            T v = s.redv[0];
            int i = s.redi[0];
#pragma unroll
            for (int q = 1; q < kMaxV / 32; ++q) better(v, i, s.redv[q], s.redi[q]);
            s.slotv[j & 1] = v;
            s.sloti[j & 1] = i;
        }
        if (CLUSTERED) cl.sync(); else __syncthreads();
        // (2) winner over the cluster (same comparison order everywhere).
        T gv = T(-1);
        int gi = INT_MAX;
        if (CLUSTERED) {
#pragma unroll
            for (int q = 0; q < CL; ++q) {
                TournSmem<T> *rs = cl.map_shared_rank(&s, q);
                better(gv, gi, rs->slotv[j & 1], rs->sloti[j & 1]);
            }
        } else {
            gv = s.slotv[j & 1];
            gi = s.sloti[j & 1];
        }
        const int owner = CLUSTERED ? gi / kMaxV : rank;
        const int lrow = CLUSTERED ? gi % kMaxV : gi;
        // (3) pivot row into local prow; the owner marks the row used.  The
        // owner's row is final (used rows are never updated again).
        {
            TournSmem<T> *os = CLUSTERED ? cl.map_shared_rank(&s, owner) : &s;
            for (int k = j + tid; k < w; k += kTournThreads) s.prow[k] = os->tile[k * kMaxV + lrow];
        }
        if (tid == 0) {
            s.order[j] = gi;
            if (owner == rank) s.used[lrow] = 1;
        }
        __syncthreads();
        // (4) eliminate column j from the unused rows.  Column j+1 of row r is
        // updated by thread r itself (half 0), which is also the thread that
        // reads it in the next argmax, so no barrier is needed here.
        const T piv = s.prow[j];
        if (piv != T(0) && r < s.nrows && !s.used[r]) {
            const T l = div_rn(s.tile[j * kMaxV + r], piv);
            for (int k = j + 1 + half; k < w; k += 2)
                s.tile[k * kMaxV + r] = sub_rn(s.tile[k * kMaxV + r], mul_rn(l, s.prow[k]));
        }
    }
    if (CLUSTERED) cl.sync(); else __syncthreads();
}

template <typename T>
__device__ void load_rows(TournSmem<T> &s, const T *__restrict__ P, int ldp, int w, int nrows) {
    for (int idx = threadIdx.x; idx < kMaxV * w; idx += kTournThreads) {
        const int k = idx / kMaxV, i = idx % kMaxV;
        if (i < nrows) s.tile[k * kMaxV + i] = P[(size_t)s.rows[i] + (size_t)k * ldp];
    }
    for (int i = threadIdx.x; i < kMaxV; i += kTournThreads) s.used[i] = (i < nrows) ? 0 : 1;
}

// Root epilogue: LAPACK ipiv and the list of moved rows (relative positions)
// for bringing the winners, in pivot order, to positions 0..w-1.
template <typename T>
__device__ void root_epilogue(TournSmem<T> &s, const int *win, int np, const TournEpilogue &ep) {
    if (ep.ipiv == nullptr) return;
    if (threadIdx.x != 0) return;
    const int w = np;
    // Home slot of a label: labels < w live in slot == label; the label of
    // a winner j with win[j] >= w lives in slot w + j.
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

template <typename T, int CL>
__global__ void __launch_bounds__(kTournThreads, 1)
k_tourn(const T *__restrict__ P, int ldp, TournPlan plan, TournWS ws, TournEpilogue ep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TournSmem<T> &s = *reinterpret_cast<TournSmem<T> *>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (CL > 1) ? (int)cl.block_rank() : 0;
    const int c = blockIdx.x / CL;
    const int tid = threadIdx.x;
    const int w = plan.w;

    // ---- leaves
    const int leaf = c * CL + rank;
    if (leaf < plan.nleaves) {
        const int row0 = leaf * plan.h;
        const int nr = min(plan.h, plan.m - row0);
        for (int i = tid; i < kMaxV; i += kTournThreads) s.rows[i] = row0 + i;
        if (tid == 0) s.nrows = nr;
        __syncthreads();
        load_rows(s, P, ldp, w, nr);
        __syncthreads();
        const int np = min(nr, w);
        gepp_select<T, false, CL>(s, w, np, rank);
        int *dst = ws.node_win + (size_t)(plan.off[0] + leaf) * kMaxV;
        for (int j = tid; j < np; j += kTournThreads) dst[j] = s.rows[s.order[j]];
        if (tid == 0) ws.node_cnt[plan.off[0] + leaf] = np;
        if (plan.nlevels == 1) {          // a single leaf is the root
            __syncthreads();
            for (int j = tid; j < np; j += kTournThreads) ws.root_win[j] = dst[j];
            __threadfence();
            __syncthreads();
            root_epilogue(s, dst, np, ep);
        }
    }
    if (plan.nlevels == 1) {
        if (CL > 1) cl.sync();
        return;
    }
    __threadfence();
    if (CL > 1) cl.sync(); else __syncthreads();

    // ---- playoff nodes: level 1 node c has exactly this cluster's leaves.
    int level = 1, g = c;
    while (true) {
        const int child0 = g * CL;
        const int nchild = min(CL, plan.cnt[level - 1] - child0);
        const int node = plan.off[level] + g;
        int *dst = ws.node_win + (size_t)node * kMaxV;
        int np;
        if (nchild == 1) {                // pass-through
            const int src = plan.off[level - 1] + child0;
            np = __ldcg(ws.node_cnt + src);
            if (rank == 0) {
                for (int j = tid; j < np; j += kTournThreads) dst[j] = __ldcg(ws.node_win + (size_t)src * kMaxV + j);
                if (tid == 0) ws.node_cnt[node] = np;
            }
        } else {
            int total = 0;
            for (int q = 0; q < nchild; ++q) total += __ldcg(ws.node_cnt + plan.off[level - 1] + child0 + q);
            np = min(total, w);
            int nr = 0;
            if (rank < nchild) {
                const int src = plan.off[level - 1] + child0 + rank;
                nr = __ldcg(ws.node_cnt + src);
                for (int i = tid; i < nr; i += kTournThreads) s.rows[i] = __ldcg(ws.node_win + (size_t)src * kMaxV + i);
            }
            if (tid == 0) s.nrows = nr;
            __syncthreads();
            load_rows(s, P, ldp, w, nr);
            __syncthreads();
            if (CL > 1) gepp_select<T, true, CL>(s, w, np, rank);
            else gepp_select<T, false, CL>(s, w, np, rank);
            if (rank == 0) {
                for (int j = tid; j < np; j += kTournThreads) {
                    const int gi = s.order[j];
                    const int owner = (CL > 1) ? gi / kMaxV : 0;
                    const int lr = (CL > 1) ? gi % kMaxV : gi;
                    const TournSmem<T> *os = (CL > 1) ? cl.map_shared_rank(&s, owner) : &s;
                    dst[j] = os->rows[lr];
                }
                if (tid == 0) ws.node_cnt[node] = np;
            }
        }
        __threadfence();
        if (CL > 1) cl.sync(); else __syncthreads();
        if (level == plan.nlevels - 1) {  // root
            if (rank == 0) {
                for (int j = tid; j < np; j += kTournThreads) ws.root_win[j] = dst[j];
                __syncthreads();
                root_epilogue(s, dst, np, ep);
            }
            break;
        }
        // Climb: the last child to finish continues with the parent.
        const int parent = g / CL;
        if (rank == 0 && tid == 0) {
            const int pnode = plan.off[level + 1] + parent;
            const int pch = min(CL, plan.cnt[level] - parent * CL);
            const int old = atomicAdd(ws.counter + pnode, 1);
            const int cont = (old == pch - 1);
            if (cont) ws.counter[pnode] = 0;   // leave the counter clean
            __threadfence();
            if (CL > 1) {
                for (int q = 0; q < CL; ++q) cl.map_shared_rank(&s, q)->cont = cont;
            } else {
                s.cont = cont;
            }
        }
        if (CL > 1) cl.sync(); else __syncthreads();
        if (!s.cont) break;
        __threadfence();
        ++level;
        g = parent;
    }
    if (CL > 1) cl.sync();
}

// LU-2: gather the moved rows of every column (one warp per column) and the
// row order.  Reads all sources before writing any destination.
template <typename T>
__global__ void __launch_bounds__(256)
k_apply_swaps(T *__restrict__ A, int lda, int ncols, int k0, const int *swap_cnt, const int *swap_dst,
              const int *swap_src, int *perm) {
    __shared__ int sd[2 * kMaxV], ss[2 * kMaxV];
    const int cnt = *swap_cnt;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) { sd[e] = swap_dst[e]; ss[e] = swap_src[e]; }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = blockIdx.x * (blockDim.x >> 5) + warp;
    if (col < ncols) {
        T *c = A + (size_t)col * lda + k0;
        T v[2 * kMaxV / 32];
#pragma unroll
        for (int q = 0; q < 2 * kMaxV / 32; ++q) {
            const int e = lane + 32 * q;
            if (e < cnt) v[q] = c[ss[e]];
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2 * kMaxV / 32; ++q) {
            const int e = lane + 32 * q;
            if (e < cnt) c[sd[e]] = v[q];
        }
    } else if (col == ncols && perm != nullptr) {
        int *c = perm + k0;
        int v[2 * kMaxV / 32];
#pragma unroll
        for (int q = 0; q < 2 * kMaxV / 32; ++q) {
            const int e = lane + 32 * q;
            if (e < cnt) v[q] = c[ss[e]];
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2 * kMaxV / 32; ++q) {
            const int e = lane + 32 * q;
            if (e < cnt) c[sd[e]] = v[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int make_tourn_plan(int m, int w, int h, int arity, TournPlan *plan) {
    if (m < 0 || w < 0 || w > kMaxV || h < 1 || h > 4 * kMaxV || arity < 2 || arity > 8) return CF_ERR_UNSUPPORTED;
    TournPlan p{};
    p.m = m; p.w = w; p.h = h; p.arity = arity;
    p.nleaves = m > 0 ? ceil_div(m, h) : 0;
    int c = p.nleaves, lv = 0, off = 0;
    while (true) {
        if (lv >= kMaxLevels) return CF_ERR_UNSUPPORTED;
        p.cnt[lv] = c; p.off[lv] = off; off += c; ++lv;
        if (c <= 1) break;
        c = (c + arity - 1) / arity;
    }
    p.nlevels = lv;
    p.total_nodes = off;
    *plan = p;
    return CF_OK;
}

size_t tourn_ws_bytes(int m, int h, int arity) {
    TournPlan p{};
    if (make_tourn_plan(m, 1, h, arity, &p) != CF_OK) return 0;
    Carver cv(nullptr);
    cv.take<int>((size_t)p.total_nodes * kMaxV);
    cv.take<int>(p.total_nodes);
    cv.take<int>(p.total_nodes);
    cv.take<int>(kMaxV);
    cv.take<int>(1);
    cv.take<int>(2 * kMaxV);
    cv.take<int>(2 * kMaxV);
    return cv.size();
}

// Counters must be zero before the first tournament; the tournament leaves
// them zero.
int tourn_ws_carve(void *work, int m, int h, int arity, TournWS *ws, TournEpilogue *ep) {
    TournPlan p{};
    int st = make_tourn_plan(m, 1, h, arity, &p);
    if (st != CF_OK) return st;
    Carver cv(work);
    ws->node_win = cv.take<int>((size_t)p.total_nodes * kMaxV);
    ws->node_cnt = cv.take<int>(p.total_nodes);
    ws->counter = cv.take<int>(p.total_nodes);
    ws->root_win = cv.take<int>(kMaxV);
    ws->counter_bytes = sizeof(int) * (size_t)p.total_nodes;
    ep->swap_cnt = cv.take<int>(1);
    ep->swap_dst = cv.take<int>(2 * kMaxV);
    ep->swap_src = cv.take<int>(2 * kMaxV);
    return CF_OK;
}

template <typename T, int CL>
static int launch_tourn_cl(const T *P, int ldp, const TournPlan &plan, const TournWS &ws, const TournEpilogue &ep,
                           cudaStream_t st) {
    const size_t smem = sizeof(TournSmem<T>);
    // The attribute belongs to the current device: set it on every call (a
    // flag kept per process would skip it on the second device).
    CF_CUDA_TRY(cudaFuncSetAttribute(k_tourn<T, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nclusters = ceil_div(plan.nleaves, CL);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nclusters * CL);
    cfg.blockDim = dim3(kTournThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tourn<T, CL>, P, ldp, plan, ws, ep));
    count_launches(1);
    return CF_OK;
}

template <typename T>
int launch_tourn(const T *P, int ldp, int m, int w, int h, int arity, const TournWS &ws, const TournEpilogue &ep,
                 cudaStream_t st) {
    if (h > kMaxV) return CF_ERR_UNSUPPORTED;      // a leaf is one tile of kMaxV rows at most
    TournPlan plan{};
    int rc = make_tourn_plan(m, w, h, arity, &plan);
    if (rc != CF_OK) return rc;
    if (m == 0 || w == 0) return CF_OK;
    switch (arity) {
        case 2: return launch_tourn_cl<T, 2>(P, ldp, plan, ws, ep, st);
        case 3: return launch_tourn_cl<T, 3>(P, ldp, plan, ws, ep, st);
        case 4: return launch_tourn_cl<T, 4>(P, ldp, plan, ws, ep, st);
        case 5: return launch_tourn_cl<T, 5>(P, ldp, plan, ws, ep, st);
        case 6: return launch_tourn_cl<T, 6>(P, ldp, plan, ws, ep, st);
        case 7: return launch_tourn_cl<T, 7>(P, ldp, plan, ws, ep, st);
        case 8: return launch_tourn_cl<T, 8>(P, ldp, plan, ws, ep, st);
        default: return CF_ERR_UNSUPPORTED;
    }
}

template <typename T>
int launch_apply_swaps(T *A, int lda, int ncols, int k0, const TournEpilogue &ep, int *perm, cudaStream_t st) {
    const int cols = ncols + (perm ? 1 : 0);
    if (cols == 0) return CF_OK;
    k_apply_swaps<T><<<ceil_div(cols, 8), 256, 0, st>>>(A, lda, ncols, k0, ep.swap_cnt, ep.swap_dst, ep.swap_src,
                                                          perm);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template int launch_tourn<double>(const double *, int, int, int, int, int, const TournWS &, const TournEpilogue &,
                                  cudaStream_t);
template int launch_tourn<float>(const float *, int, int, int, int, int, const TournWS &, const TournEpilogue &,
                                 cudaStream_t);
template int launch_apply_swaps<double>(double *, int, int, int, const TournEpilogue &, int *, cudaStream_t);
template int launch_apply_swaps<float>(float *, int, int, int, const TournEpilogue &, int *, cudaStream_t);

}  // namespace cf

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" size_t cf_tourn_workspace_size(int m, int w, int leaf_h, int arity) {
    (void)w;
    (void)leaf_h;   // sized for the most leaves (h = 1), valid for every leaf height
    if (arity > 8) return 0;
    return cf::tourn_ws_bytes(m > 0 ? m : 1, 1, arity < 2 ? 2 : arity);
}

extern "C" int cf_tourn_select(int m, int w, const double *panel, int ldp, int leaf_h, int arity, int *winners,
                               void *work, size_t lwork, cudaStream_t stream) {
    using namespace cf;
    if (m < 0) return -1;
    if (w < 0 || w > kMaxV) return -2;
    if (m > 0 && w > 0 && panel == nullptr) return -3;
    if (ldp < (m > 1 ? m : 1)) return -4;
    if (leaf_h < 1 || leaf_h > kMaxV) return -5;
    if (arity < 2 || arity > 8) return -6;
    if (m == 0 || w == 0) return CF_OK;
    if (winners == nullptr) return -7;
    if (lwork < cf_tourn_workspace_size(m, w, leaf_h, arity) || work == nullptr) return CF_ERR_WORKSPACE;
    TournWS ws{};
    TournEpilogue ep{};
    int rc = tourn_ws_carve(work, m, 1, arity, &ws, &ep);
    if (rc != CF_OK) return rc;
    ep.ipiv = nullptr;
    CF_CUDA_TRY(cudaMemsetAsync(ws.counter, 0, ws.counter_bytes, stream));
    ws.root_win = winners;
    return launch_tourn<double>(panel, ldp, m, w, leaf_h, arity, ws, ep, stream);
}
