// Hot-path kernels of the SLR apply (Eq. 4.1 with S~^{-1} of Eq. 4.7) and of
// the setup Lanczos on H (Eq. 3.2, Section 5.1), written for sm_103a.
//
//  K1  band solve      t = B^{-1} f, p independent banded Cholesky solves
//  K2  coupling SpMVs  g' = g - E^T t,  b = E y
//  K3  C solves        L^{-1} and L^{-T} with a supernodal, level-scheduled factor
//                      in unit block form (one dependent step per level)
//  K4  low rank        w' = w/(1-theta) + U_k (d o U_k^T w)
//  K5  PCG             A p, dots, axpys, scalar updates (FP64)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <type_traits>
#include <vector>

#include "slr_device.h"

namespace slr {

std::atomic<int64_t> g_kernel_launches{0};
thread_local int64_t t_kernel_launches = 0;

void count_launches(int64_t n) {
    g_kernel_launches.fetch_add(n, std::memory_order_relaxed);
    t_kernel_launches += n;
}
int64_t thread_launches() { return t_kernel_launches; }

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The warp sums of N values (N a power of two up to 32) at once: at each of the
// first log2 N butterfly steps a lane keeps half of its values and adds its
// partner's copies of them (own + partner, as warp_sum does), the remaining steps
// add whole; every sum is formed by warp_sum's tree, bit for bit, with N - 1 +
// 5 - log2 N shuffles instead of 5 N.  Lane l returns the sum of value
// rs_index<N>(l); lanes that differ only in the low 5 - log2 N bits hold the same.
template <typename T, int N>
__device__ __forceinline__ T reduce_scatter(T (&v)[N], int lane) {
    static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "a power of two up to 32");
    int o = 16;
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    T r = v[0];
    for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}
template <int N>
__device__ __forceinline__ int rs_index(int lane) {
    int k = 0, o = 16;
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2, o >>= 1)
        if (lane & o) k += h;
    return k;
}
// a lane that writes its reduce_scatter<N> sum (one per distinct sum)
template <int N>
__device__ __forceinline__ bool rs_writer(int lane) {
    return (lane & (32 / N - 1)) == 0;
}

// K1 (the batched band solve) lives in slr_band.cu.

// ------------------------------------------------------------------ K2
// Y = A X for a block of columns (CSR A; given G: Y = G - A X), as the coupling
// products E y and g - E^T t and the products with A and C use it.  A thread
// takes one row for kSpCols columns, so the row's entries are read once per
// group of columns; each column's sum runs over the row's entries in order
// (the same sums, bit for bit, whatever the number of columns).
constexpr int kSpCols = 8;

template <typename T>
__global__ void k_spmv_cols(int32_t rows, int32_t nrhs, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const T* __restrict__ v, const T* x, int64_t ldx,
                            const T* g, int64_t ldg, T* y, int64_t ldy) {
    const int32_t ngr = (nrhs + kSpCols - 1) / kSpCols;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * ngr) return;
    const int32_t i = (int32_t)(idx % rows), j0 = (int32_t)(idx / rows) * kSpCols;
    const int nc = min(kSpCols, nrhs - j0);
    T acc[kSpCols];
#pragma unroll
    for (int c = 0; c < kSpCols; ++c) acc[c] = T(0);
    const int32_t e1 = rp[i + 1];
    for (int32_t q = rp[i]; q < e1; ++q) {
        const T a = v[q];
        const int64_t col = ci[q];
#pragma unroll
        for (int c = 0; c < kSpCols; ++c)
            if (c < nc) acc[c] += a * x[col + (int64_t)(j0 + c) * ldx];
    }
#pragma unroll
    for (int c = 0; c < kSpCols; ++c)
        if (c < nc) {
            const int64_t o = (int64_t)(j0 + c);
            y[i + o * ldy] = g ? g[i + o * ldg] - acc[c] : acc[c];
        }
}

// ------------------------------------------------------------------ K3
// Supernode J owns factor positions [c0[J], c0[J+1]) (n_J of them).  Its
// diagonal block is stored inverted (packed lower, column-major: column j
// starts at cs(j) = j n_J - j (j-1) / 2) and its off-diagonal rows R_J carry
// the row-major panel M_J = L[R_J, J] L_JJ^{-1} (|R_J| x n_J): the off-diagonal
// block of the unit block factor Lhat = L D^{-1}, D = diag(L_JJ).  With
// L^{-1} = D^{-1} Lhat^{-1} and L^{-T} = Lhat^{-T} D^{-T}:
//   forward   t_J = g_J - sum of the panel products w that hold J's rows,
//             then x_J = L_JJ^{-1} t_J and w_J = M_J t_J, both from t_J
//   backward  x_J = L_JJ^{-T} y_J - M_J^T x_{R_J}
// so every level (leaves -> root forward, root -> leaves backward) is one
// dependent step.  A forward task is a block of <= 32 rows of L_JJ^{-1} or of
// M_J (every task of J gathers all of t_J itself); a backward task is a block
// of <= 32 columns of J.  Tasks are (J, first, count, 0).
//
// Levels whose supernodes are many and small run one group of threads per
// supernode (all its tasks in one group).  The per-level kernels wrap one
// level in one launch; the persistent kernels run every level in one
// cooperative launch with a grid barrier between levels.
__device__ __forceinline__ int64_t packed_col(int j, int n) { return (int64_t)j * n - (int64_t)j * (j - 1) / 2; }

// Plain view of a DevCFactor (device pointers and sizes) passed by value.
template <typename T>
struct CView {
    int32_t s, nlev, nsteps;
    int64_t nrow;
    int64_t wr;        // row stride of wbuf and tws: the call's right-hand sides are contiguous per row
    int64_t xr;        // row stride of the backward's solution x (factor order; right-hand sides contiguous)
    const int32_t *cperm, *c0, *rows, *seg_row, *lev_sn;
    const int64_t *r_off, *pan_off, *dinv_off, *seg_ptr;
    const T *panel, *dinv;
    T* wbuf;
    const T* gf;       // the forward's input g in factor order, position pos's right-hand sides at pos wr,
                       // or null: g is read through cperm
    T* tws;            // t_J of the level's supernodes gathered by k_cfwd_gather (s x nrhs), or null:
                       // each forward task gathers t_J itself
    const int4 *tasks, *ptasks;
    const int32_t *lev_task_ptr, *lev_ptask_ptr, *lev_sn_ptr;
    const uint8_t* lev_small;
    int64_t red_off;   // persistent kernels: reduction array offset in shared memory (elements)
    int32_t pers_rb, pers_tstride;   // persistent forward: right-hand sides per matrix load, t_J stride
    int32_t stage_cap; // persistent kernels: stage buffer of each fused-level group (elements)
    // top zone
    int32_t nT, tf_parts, tb_parts;
    const int32_t *tpos, *tseg_row, *tsk_lo, *tp_pos, *tb_cb_part;
    const int64_t *tseg_ptr, *tsk_off, *tb_off, *tp_off;
    const T *tsk, *tb;
    const int4 *tf_rb, *tf_tasks, *tb_cb, *tb_tasks;
    T *tT, *tf_part, *tb_part;
    int32_t *tf_cnt, *tb_cnt;
    unsigned* bar;
    int32_t* err;
    long long spin;    // polls of a grid-barrier wait before it gives up
};

// sum of w[seg_row[e] wr] for e = e0 .. e1-1, in that order: indices and values are
// loaded 8 at a time so that the two dependent loads are not paid per term
template <typename T>
__device__ __forceinline__ T gather_sum(const T* w, int64_t wr, const int32_t* __restrict__ seg_row, int64_t e0,
                                       int64_t e1) {
    T acc = T(0);
    for (int64_t e = e0; e < e1; e += 8) {
        int32_t idx[8];
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) idx[u] = e + u < e1 ? seg_row[e + u] : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = idx[u] >= 0 ? w[(int64_t)idx[u] * wr] : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (e + u < e1) acc += v[u];
    }
    return acc;
}

// the forward's input at factor position pos, right-hand side j
template <typename T>
__device__ __forceinline__ T g_at(const CView<T>& cf, int32_t pos, const T* g, int64_t ldg, int j) {
    return cf.gf ? cf.gf[(int64_t)pos * cf.wr + j] : g[cf.cperm[pos] + (int64_t)j * ldg];
}

// entry pos of t = g - gathered panel products, right-hand side j
template <typename T>
__device__ __forceinline__ T t_entry(const CView<T>& cf, int32_t pos, const T* g, int64_t ldg, int j) {
    return g_at(cf, pos, g, ldg, j) -
           gather_sum(cf.wbuf + j, cf.wr, cf.seg_row, cf.seg_ptr[pos], cf.seg_ptr[pos + 1]);
}

// t at position pos for right-hand sides j .. j + nb - 1 (nb <= 8) into out[0 .. 8)
// (zeros past nb): the index chain is loaded once for the eight, each sum still
// takes its contributions in order, as t_entry does
template <typename T>
__device__ __forceinline__ void t_entry8(const CView<T>& cf, int32_t pos, const T* g, int64_t ldg, int j, int nb,
                                         T (&out)[8]) {
    const int64_t e0 = cf.seg_ptr[pos], e1 = cf.seg_ptr[pos + 1];
    T acc[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[b] = T(0);
    for (int64_t e = e0; e < e1; e += 4) {
        int32_t idx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) idx[u] = e + u < e1 ? cf.seg_row[e + u] : -1;
        T v[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int b = 0; b < 8; ++b)
                v[u][b] = (idx[u] >= 0 && b < nb) ? cf.wbuf[(int64_t)idx[u] * cf.wr + j + b] : T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (idx[u] >= 0) {
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[b] += v[u][b];
            }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) out[b] = b < nb ? g_at(cf, pos, g, ldg, j + b) - acc[b] : T(0);
}

// t_J = g_J - gathered panel products into ts[0 .. n_J) by NTH threads (thread gt)
template <typename T>
__device__ __forceinline__ void gather_t(const CView<T>& cf, int J, int gt, int nth, T* ts, const T* g, int64_t ldg,
                                         int j) {
    const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
    for (int i = gt; i < nJ; i += nth) ts[i] = t_entry(cf, a0 + i, g, ldg, j);
}

// eight consecutive values from shared memory (p 16-byte aligned)
template <typename T>
__device__ __forceinline__ void ld8(const T* p, T (&v)[8]) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 a = reinterpret_cast<const double2*>(p)[q];
            v[2 * q] = a.x;
            v[2 * q + 1] = a.y;
        }
    }
}
// right-hand sides per pass of the tiled small-supernode paths
template <typename T>
__host__ __device__ constexpr int tile_rp() { return sizeof(T) == 4 ? 32 : 16; }

// Forward task (one CTA of NW warps) on RB right-hand sides j0 .. j0 + RB - 1: t_J of
// each into ts (column b at ts + b * tstride), then rows tk.y .. tk.y + tk.z - 1 of
// w_J = M_J t_J (panel task: a warp per row, lanes over the columns, 8 loads in
// flight) or of x_J = L_JJ^{-1} t_J (diagonal task: lane = row, the warps split the
// columns, partial sums added in a fixed order).  Each matrix entry is loaded once
// for the RB columns; every column sees the same sequence of multiply-adds for any
// RB, so a column gives the same bits alone and in a block.
template <typename T, int NW, int RB>
__device__ void cfwd_task_rb(const CView<T>& cf, const int4 tk, bool pan, T* ts, int tstride, T (*red)[33],
                             const T* g, int64_t ldg, T* xf, int j0, T* red2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t J = tk.x, a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        if (cf.tws) {                   // gathered once for the level (the same values)
            for (int i = threadIdx.x; i < nJ; i += NW * 32) ts[b * tstride + i] = cf.tws[(a0 + i) * cf.wr + j0 + b];
        } else {
            gather_t(cf, J, threadIdx.x, NW * 32, ts + b * tstride, g, ldg, j0 + b);
        }
    }
    __syncthreads();
    if (pan) {
        const T* P = cf.panel + cf.pan_off[J];
        for (int pr = warp; pr < tk.z; pr += NW) {
            const int64_t p = tk.y + pr;
            const T* Pp = P + p * nJ;
            T acc[RB];
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[b] = T(0);
            int c = lane;
            for (; c + 7 * 32 < nJ; c += 8 * 32) {
                T pv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) pv[u] = Pp[c + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int b = 0; b < RB; ++b) acc[b] += pv[u] * ts[b * tstride + c + 32 * u];
            }
            for (; c < nJ; c += 32) {
                const T pv = Pp[c];
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] += pv * ts[b * tstride + c];
            }
            const T v = reduce_scatter<T, RB>(acc, lane);
            if (rs_writer<RB>(lane)) cf.wbuf[(cf.r_off[J] + p) * cf.wr + j0 + rs_index<RB>(lane)] = v;
        }
    } else {
        const T* D = cf.dinv + cf.dinv_off[J];
        const int il = tk.y + lane;
        const int ncol = tk.y + tk.z;   // columns 0 .. ncol-1 reach these rows
        const int chunk = (ncol + NW - 1) / NW;
        const int jb = warp * chunk, je = min(ncol, jb + chunk);
        T acc[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[b] = T(0);
        if (lane < tk.z) {
            const int jend = min(je, il + 1);
            int jj = jb;
            for (; jj + 7 < jend; jj += 8) {
                T d[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) d[u] = D[packed_col(jj + u, nJ) + (il - jj - u)];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int b = 0; b < RB; ++b) acc[b] += d[u] * ts[b * tstride + jj + u];
            }
            for (; jj < jend; ++jj) {
                const T d = D[packed_col(jj, nJ) + (il - jj)];
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] += d * ts[b * tstride + jj];
            }
        }
        if (red2) {
            // the warps' partial sums of all RB columns at once (red2: NW x RB x 32),
            // then each column's added over the warps in order, as below
#pragma unroll
            for (int b = 0; b < RB; ++b) red2[(warp * RB + b) * 32 + lane] = acc[b];
            __syncthreads();
            for (int b = warp; b < RB; b += NW) {
                T v = T(0);
#pragma unroll 8
                for (int w = 0; w < NW; ++w) v += red2[(w * RB + b) * 32 + lane];
                if (lane < tk.z) xf[a0 + il + (int64_t)(j0 + b) * cf.s] = v;
            }
        } else {
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                red[warp][lane] = acc[b];
                __syncthreads();
                if (warp == 0) {
                    T v = T(0);
#pragma unroll 8
                    for (int w = 0; w < NW; ++w) v += red[w][lane];
                    if (lane < tk.z) xf[a0 + il + (int64_t)(j0 + b) * cf.s] = v;
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
}

// All nrhs columns: blocks of 8 or 4 while ts holds that many columns (rbmax), then one at a time.
// red2 (NW x rbmax x 32, or null): the diagonal tasks' partial sums of a block at once.
template <typename T, int NW, int RBMAX = 8>
__device__ void cfwd_task_cta(const CView<T>& cf, const int4 tk, bool pan, T* ts, int tstride, int rbmax,
                              T (*red)[33], const T* g, int64_t ldg, T* xf, int32_t nrhs, T* red2 = nullptr) {
    int j0 = 0;
    if constexpr (RBMAX >= 8) {
        if (rbmax >= 8)
            for (; j0 + 8 <= nrhs; j0 += 8)
                cfwd_task_rb<T, NW, 8>(cf, tk, pan, ts, tstride, red, g, ldg, xf, j0, red2);
    }
    if (rbmax >= 4)
        for (; j0 + 4 <= nrhs; j0 += 4) cfwd_task_rb<T, NW, 4>(cf, tk, pan, ts, tstride, red, g, ldg, xf, j0, red2);
    for (; j0 < nrhs; ++j0) cfwd_task_rb<T, NW, 1>(cf, tk, pan, ts, tstride, red, g, ldg, xf, j0, nullptr);
}

// four consecutive values from shared memory (p 16-byte aligned)
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

// Forward task on a block of RP right-hand sides j0 .. j0 + nb - 1 in one pass (RP 16
// or 32; columns past nb are zeros): t_J from the level's gather, stored right-hand
// sides contiguous with row stride RP + 4 (16-byte loads by the lanes of different
// columns then meet distinct banks).  Panel rows: a warp per row, lanes over the
// columns with RP sums each, then one reduce-scatter; diagonal rows: lane = row, the
// warps split the columns and their partial sums are added in order.  Every (row,
// right-hand side) gets the multiply-adds and additions of cfwd_task_rb, bit for bit.
// red2: NW x RP x 32.
template <typename T, int NW, int RP>
__device__ void cfwd_task_blk(const CView<T>& cf, const int4 tk, bool pan, T* ts, T* red2, T* xf, int j0, int nb) {
    constexpr int RS = RP + 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t J = tk.x, a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
    const int ncl = pan ? nJ : tk.y + tk.z;        // columns the task reads
    for (int idx = threadIdx.x; idx < ncl * RP; idx += NW * 32) {
        const int i = idx / RP, b = idx - i * RP;     // right-hand sides fastest: contiguous in the gather
        ts[i * RS + b] = b < nb ? cf.tws[(int64_t)(a0 + i) * cf.wr + j0 + b] : T(0);
    }
    __syncthreads();
    if (pan) {
        const T* P = cf.panel + cf.pan_off[J];
        for (int pr = warp; pr < tk.z; pr += NW) {
            const int64_t p = tk.y + pr;
            const T* Pp = P + p * nJ;
            T acc[RP];
#pragma unroll
            for (int b = 0; b < RP; ++b) acc[b] = T(0);
            auto madd = [&](T a, int c) {
#pragma unroll
                for (int q = 0; q < RP; q += 4) {
                    T t4[4];
                    ld4(ts + c * RS + q, t4);
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[q + e] += a * t4[e];
                }
            };
            int c = lane;
            for (; c + 7 * 32 < nJ; c += 8 * 32) {
                T pv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) pv[u] = Pp[c + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; ++u) madd(pv[u], c + 32 * u);
            }
            for (; c < nJ; c += 32) madd(Pp[c], c);
            const T v = reduce_scatter<T, RP>(acc, lane);
            const int k = rs_index<RP>(lane);
            if (rs_writer<RP>(lane) && k < nb) cf.wbuf[(cf.r_off[J] + p) * cf.wr + j0 + k] = v;
        }
    } else {
        const T* D = cf.dinv + cf.dinv_off[J];
        const int il = tk.y + lane;
        const int ncol = tk.y + tk.z;
        const int chunk = (ncol + NW - 1) / NW;
        const int jb = warp * chunk, je = min(ncol, jb + chunk);
        T acc[RP];
#pragma unroll
        for (int b = 0; b < RP; ++b) acc[b] = T(0);
        auto madd = [&](T a, int c) {
#pragma unroll
            for (int q = 0; q < RP; q += 4) {
                T t4[4];
                ld4(ts + c * RS + q, t4);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[q + e] += a * t4[e];
            }
        };
        if (lane < tk.z) {
            const int jend = min(je, il + 1);
            int jj = jb;
            for (; jj + 7 < jend; jj += 8) {
                T d[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) d[u] = D[packed_col(jj + u, nJ) + (il - jj - u)];
#pragma unroll
                for (int u = 0; u < 8; ++u) madd(d[u], jj + u);
            }
            for (; jj < jend; ++jj) madd(D[packed_col(jj, nJ) + (il - jj)], jj);
        }
#pragma unroll
        for (int b = 0; b < RP; ++b) red2[(warp * RP + b) * 32 + lane] = acc[b];
        __syncthreads();
        for (int b = warp; b < nb; b += NW) {
            T v = T(0);
#pragma unroll 8
            for (int w = 0; w < NW; ++w) v += red2[(w * RP + b) * 32 + lane];
            if (lane < tk.z) xf[a0 + il + (int64_t)(j0 + b) * cf.s] = v;
        }
    }
    __syncthreads();
}

// Backward task (one CTA of NW warps) on RB right-hand sides: columns
// c = tk.y .. tk.y + tk.z - 1 of x_J = L_JJ^{-T} y_J - M_J^T x_{R_J}.  The diagonal
// part runs a warp per column (lanes over column c of L_JJ^{-1}, contiguous in the
// packed layout); the panel part has lanes over the columns and the warps splitting
// the panel rows, DEPTH loads in flight per lane.  Each matrix entry is loaded once
// for the RB columns, with the same per-column sequence of multiply-adds for any RB.
// Optional scatter of the result to DD order.  us: RB x 32.
template <typename T, int NW, int DEPTH, int RB>
__device__ void cbwd_task_rb(const CView<T>& cf, const int4 tk, T* us, T (*red)[33], const T* yf, T* xf, T* y_dd,
                             int64_t ldy, int j0, T* red2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t J = tk.x, a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0, jl = tk.y + lane;
    const int64_t nr = cf.r_off[J + 1] - cf.r_off[J];
    const int32_t* R = cf.rows + cf.r_off[J];
    const T* Pn = cf.panel + cf.pan_off[J] + jl;
    const T* D = cf.dinv + cf.dinv_off[J];
    const int64_t chunk = (nr + NW - 1) / NW, pb = warp * chunk, pe = min(nr, pb + chunk);
    const T* y = yf + a0 + (int64_t)j0 * cf.s;
    const T* x = xf + j0;                    // x(pos, b) at x[pos xr + b]
    for (int cc = warp; cc < tk.z; cc += NW) {
        const int c = tk.y + cc;
        const T* Dc = D + packed_col(c, nJ) - c;   // Dc[i] = (L_JJ^{-1})[i, c], i >= c
        T acc[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[b] = T(0);
        int i = c + lane;
        for (; i + 7 * 32 < nJ; i += 8 * 32) {
            T d[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) d[u] = Dc[i + 32 * u];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] += d[u] * y[(int64_t)b * cf.s + i + 32 * u];
        }
        for (; i < nJ; i += 32) {
            const T d = Dc[i];
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[b] += d * y[(int64_t)b * cf.s + i];
        }
        const T v = reduce_scatter<T, RB>(acc, lane);
        if (rs_writer<RB>(lane)) us[rs_index<RB>(lane) * 32 + cc] = v;
    }
    T acc[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[b] = T(0);
    if (lane < tk.z) {
        int64_t p = pb;
        for (; p + DEPTH - 1 < pe; p += DEPTH) {
            T pv[DEPTH];
            int32_t rr[DEPTH];
#pragma unroll
            for (int u = 0; u < DEPTH; ++u) {
                pv[u] = Pn[(p + u) * nJ];
                rr[u] = R[p + u];
            }
#pragma unroll
            for (int u = 0; u < DEPTH; ++u)
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] += pv[u] * x[(int64_t)rr[u] * cf.xr + b];
        }
        for (; p < pe; ++p) {
            const T pv = Pn[p * nJ];
            const int32_t r = R[p];
#pragma unroll
            for (int b = 0; b < RB; ++b) acc[b] += pv * x[(int64_t)r * cf.xr + b];
        }
    }
    if (red2) {
        // all RB columns' partial sums at once (red2: NW x RB x 32), each column's then
        // added over the warps in order, as below
#pragma unroll
        for (int b = 0; b < RB; ++b) red2[(warp * RB + b) * 32 + lane] = acc[b];
        __syncthreads();
        for (int b = warp; b < RB; b += NW) {
            if (lane < tk.z) {
                T v = T(0);
#pragma unroll 8
                for (int w = 0; w < NW; ++w) v += red2[(w * RB + b) * 32 + lane];
                const T r = us[b * 32 + lane] - v;
                xf[(int64_t)(a0 + jl) * cf.xr + j0 + b] = r;
                if (y_dd) y_dd[cf.cperm[a0 + jl] + (int64_t)(j0 + b) * ldy] = r;
            }
        }
        __syncthreads();
        return;
    }
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        red[warp][lane] = acc[b];
        __syncthreads();
        if (warp == 0 && lane < tk.z) {
            T v = T(0);
#pragma unroll 8
            for (int w = 0; w < NW; ++w) v += red[w][lane];
            const T r = us[b * 32 + lane] - v;
            xf[(int64_t)(a0 + jl) * cf.xr + j0 + b] = r;
            if (y_dd) y_dd[cf.cperm[a0 + jl] + (int64_t)(j0 + b) * ldy] = r;
        }
        __syncthreads();
    }
}

// Backward task on a block of RP right-hand sides j0 .. j0 + nb - 1 in one pass: the
// diagonal part as in cbwd_task_rb (a warp per column, lanes over the rows) with RP
// sums per lane and one reduce-scatter; the panel part with lanes over the columns
// and the warps splitting the panel rows, each warp staging the gathered rows of
// x_{R_J} (32 rows x RP, one right-hand side per lane, row stride RP + 4) in its own
// part of xs and reading them back by 16-byte broadcasts; its
// partial sums then go to xs (the same buffer) and are added over the warps in
// order.  Every column gets cbwd_task_rb's multiply-adds and additions, bit for bit.
// us: RP x 32; xs: NW x 32 x (RP + 4).
template <typename T, int NW, int RP>
__device__ void cbwd_task_blk(const CView<T>& cf, const int4 tk, T* us, T* xs, const T* yf, T* xf, T* y_dd,
                              int64_t ldy, int j0, int nb) {
    constexpr int RS = RP + 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t J = tk.x, a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0, jl = tk.y + lane;
    const int64_t nr = cf.r_off[J + 1] - cf.r_off[J];
    const int32_t* R = cf.rows + cf.r_off[J];
    const T* Pn = cf.panel + cf.pan_off[J] + jl;
    const T* D = cf.dinv + cf.dinv_off[J];
    const int64_t chunk = (nr + NW - 1) / NW, pb = warp * chunk, pe = min(nr, pb + chunk);
    const T* y = yf + a0 + (int64_t)j0 * cf.s;
    const T* x = xf + j0;                    // x(pos, b) at x[pos xr + b]
    // right-hand side b of the block (zero past nb)
    auto yv = [&](int b, int64_t i) { return b < nb ? y[(int64_t)b * cf.s + i] : T(0); };
    for (int cc = warp; cc < tk.z; cc += NW) {
        const int c = tk.y + cc;
        const T* Dc = D + packed_col(c, nJ) - c;   // Dc[i] = (L_JJ^{-1})[i, c], i >= c
        T acc[RP];
#pragma unroll
        for (int b = 0; b < RP; ++b) acc[b] = T(0);
        int i = c + lane;
        for (; i + 7 * 32 < nJ; i += 8 * 32) {
            T d[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) d[u] = Dc[i + 32 * u];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int b = 0; b < RP; ++b) acc[b] += d[u] * yv(b, i + 32 * u);
        }
        for (; i < nJ; i += 32) {
            const T d = Dc[i];
#pragma unroll
            for (int b = 0; b < RP; ++b) acc[b] += d * yv(b, i);
        }
        const T v = reduce_scatter<T, RP>(acc, lane);
        if (rs_writer<RP>(lane)) us[rs_index<RP>(lane) * 32 + cc] = v;
    }
    T acc[RP];
#pragma unroll
    for (int b = 0; b < RP; ++b) acc[b] = T(0);
    T* xw = xs + (size_t)warp * 32 * RS;               // this warp's rows
    for (int64_t q0 = pb; q0 < pe; q0 += 32) {
        const int nq = (int)min((int64_t)32, pe - q0);
        // x_{R_J} rows q0 .. q0 + nq - 1: lane b loads right-hand side b of each
        if (lane < RP) {
            T v[8];
            for (int pp0 = 0; pp0 < nq; pp0 += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = (pp0 + u < nq && lane < nb) ? x[(int64_t)R[q0 + pp0 + u] * cf.xr + lane] : T(0);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (pp0 + u < nq) xw[(pp0 + u) * RS + lane] = v[u];
            }
        }
        __syncwarp();
        if (lane < tk.z) {
            for (int pp = 0; pp < nq; ++pp) {
                const T pv = Pn[(q0 + pp) * nJ];
#pragma unroll
                for (int q = 0; q < RP; q += 4) {
                    T t4[4];
                    ld4(xw + pp * RS + q, t4);
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[q + e] += pv * t4[e];
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();                                    // every warp is done with its rows: xs takes the sums
#pragma unroll
    for (int b = 0; b < RP; ++b) xs[(warp * RP + b) * 32 + lane] = acc[b];
    __syncthreads();
    for (int b = warp; b < nb; b += NW) {
        if (lane < tk.z) {
            T v = T(0);
#pragma unroll 8
            for (int w = 0; w < NW; ++w) v += xs[(w * RP + b) * 32 + lane];
            const T r = us[b * 32 + lane] - v;
            xf[(int64_t)(a0 + jl) * cf.xr + j0 + b] = r;
            if (y_dd) y_dd[cf.cperm[a0 + jl] + (int64_t)(j0 + b) * ldy] = r;
        }
    }
    __syncthreads();
}

// All nrhs columns: blocks of 8 or 4 while us holds that many columns (rbmax), then
// one at a time (DEPTH4: loads in flight per lane in a block).
// red2 (NW x rbmax x 32, or null): the panel part's partial sums of a block at once.
template <typename T, int NW, int DEPTH, int DEPTH4, int RBMAX = 8>
__device__ void cbwd_task_cta(const CView<T>& cf, const int4 tk, T* us, int rbmax, T (*red)[33], const T* yf, T* xf,
                              T* y_dd, int64_t ldy, int32_t nrhs, T* red2 = nullptr) {
    int j0 = 0;
    if constexpr (RBMAX >= 8) {
        if (rbmax >= 8)
            for (; j0 + 8 <= nrhs; j0 += 8)
                cbwd_task_rb<T, NW, DEPTH4, 8>(cf, tk, us, red, yf, xf, y_dd, ldy, j0, red2);
    }
    if (rbmax >= 4)
        for (; j0 + 4 <= nrhs; j0 += 4) cbwd_task_rb<T, NW, DEPTH4, 4>(cf, tk, us, red, yf, xf, y_dd, ldy, j0, red2);
    for (; j0 < nrhs; ++j0) cbwd_task_rb<T, NW, DEPTH, 1>(cf, tk, us, red, yf, xf, y_dd, ldy, j0, nullptr);
}

// Synchronises the NT threads of a group: the whole CTA (GROUPS = 1) or group
// g of GROUPS equal groups (named barrier 1 + g).
template <int NT, int GROUPS>
__device__ __forceinline__ void group_sync() {
    if constexpr (GROUPS == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / NT)), "r"(NT) : "memory");
    }
}

// Copies n elements from global src to shared dst with asynchronous copies, the NT
// threads of a group each issuing several before any lands (one commit group).
template <typename T, int NT>
__device__ __forceinline__ void stage_async(T* dst, const T* src, int64_t n, int gt) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    for (int64_t i = gt; i < n; i += NT) {
        const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + i));
        if constexpr (sizeof(T) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src + i) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src + i) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stages A_J = [L_JJ^{-1} (packed); M_J] of a small supernode in the group's shared
// buffer stg (cap elements) when it fits; D and P then point there, else to HBM.
// The arithmetic is the same either way.
template <typename T, int NT>
__device__ __forceinline__ bool stage_block(const CView<T>& cf, int J, T* stg, int cap, int gt, const T*& D,
                                            const T*& P) {
    const int64_t nJ = cf.c0[J + 1] - cf.c0[J], nr = cf.r_off[J + 1] - cf.r_off[J];
    const int64_t nd = nJ * (nJ + 1) / 2;
    D = cf.dinv + cf.dinv_off[J];
    P = cf.panel + cf.pan_off[J];
    if (nd + nr * nJ > cap) return false;
    stage_async<T, NT>(stg, D, nd, gt);
    stage_async<T, NT>(stg + nd, P, nr * nJ, gt);
    D = stg;
    P = stg + nd;
    return true;
}

// Odd row stride of a staged panel: a warp reading one column across 32 panel
// rows then meets every shared-memory bank equally often.
__device__ __forceinline__ int32_t small_ldp(int32_t nJ) { return nJ | 1; }

// Forward staging of A_J: L_JJ^{-1} packed as stored, then M_J with row stride
// small_ldp(n_J); false (D and P in HBM, row stride n_J) when it does not fit cap.
template <typename T, int NT>
__device__ __forceinline__ bool stage_block_fwd(const CView<T>& cf, int J, T* stg, int cap, int gt, const T*& D,
                                                const T*& P) {
    const int32_t nJ = cf.c0[J + 1] - cf.c0[J], nr = (int32_t)(cf.r_off[J + 1] - cf.r_off[J]);
    const int32_t nd = nJ * (nJ + 1) / 2, ldp = small_ldp(nJ);
    D = cf.dinv + cf.dinv_off[J];
    P = cf.panel + cf.pan_off[J];
    if ((int64_t)nd + (int64_t)nr * ldp > cap) return false;
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    for (int32_t i = gt; i < nd; i += NT) {
        const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(stg + i));
        if constexpr (sizeof(T) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(D + i) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(D + i) : "memory");
    }
    // panel row q (n_J values, contiguous in HBM) to stg + nd + q * ldp, a warp per row
    constexpr int nw = NT / 32;
    const int lane = gt & 31;
    for (int32_t q = gt >> 5; q < nr; q += nw)
        for (int32_t c = lane; c < nJ; c += 32) {
            const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(stg + nd + q * ldp + c));
            const T* src = P + (int64_t)q * nJ + c;
            if constexpr (sizeof(T) == 8)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
        }
    asm volatile("cp.async.commit_group;" ::: "memory");
    D = stg;
    P = stg + nd;
    return true;
}

// Fused levels: one group of NT threads (a CTA, or a part of one) per supernode J
// with n_J <= kSmallN and |R_J| <= kSmallR.  Both directions use the stacked
// matrix A_J = [L_JJ^{-1}; M_J] ((n_J + |R_J|) x n_J; row r < n_J of the
// diagonal block is read from the packed column-major layout).
// forward: t_J gathered into ts, then [x_J; w_J] = A_J t_J.  Staged in shared
// memory, a thread computes a row (columns in order: one multiply-add per column,
// no cross-lane sums, which on this part's narrow FP64 unit cost more than the
// products); from HBM, a warp per row keeps the loads coalesced (lanes over the
// columns, four rows in flight per warp).  RB right-hand sides share each pass
// over A_J (ts holds RB vectors, kSmallN apart), each with the multiply-adds it
// gets alone; a supernode is staged or not whatever the right-hand sides, so
// every column gets the same bits alone and in a block.
// Blocks of right-hand sides on a staged supernode (tiled): the n_J rows of
// L_JJ^{-1}, padded to whole groups of 32, then the |R_J| panel rows form the
// virtual rows; a warp takes 128 of them (lane + 32 u, u < 4) for 8 right-hand
// sides, so that each thread holds 4 x 8 sums and a column costs four matrix loads
// and two 16-byte loads of t_J (stored right-hand sides contiguous, RP per pass)
// for 32 multiply-adds.  Each (row, right-hand side) still takes its multiply-adds
// over the columns in order from zero; a diagonal row adds exact zeros past its
// last column, so the bits are those of the row-per-thread path.
template <typename T, int NT, int GROUPS>
__device__ void cfwd_small_tiled(const CView<T>& cf, int J, T* ts, const T* g, int64_t ldg, T* xf, int32_t nrhs,
                                 const T* D, const T* Pn) {
    constexpr int nw = NT / 32, RPM = tile_rp<T>();
    const int gt = threadIdx.x % NT, lane = gt & 31, warp = gt >> 5;
    const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
    const int32_t nr = (int32_t)(cf.r_off[J + 1] - cf.r_off[J]);
    const int32_t ND = (nJ + 31) & ~31, RV = ND + nr, ldp = small_ldp(nJ);
    T* wb = cf.wbuf + cf.r_off[J] * cf.wr;
    for (int j0 = 0; j0 < nrhs; j0 += RPM) {
        const int nb = min(RPM, nrhs - j0), RP = (nb + 7) & ~7, ngrp = RP / 8;
        for (int it = gt; it < nJ * ngrp; it += NT) {
            const int i = it / ngrp, h = it - i * ngrp;
            T tv[8];
            t_entry8(cf, a0 + i, g, ldg, j0 + 8 * h, nb - 8 * h, tv);
#pragma unroll
            for (int b = 0; b < 8; ++b) ts[i * RP + 8 * h + b] = tv[b];
        }
        if (j0 == 0) stage_wait();
        group_sync<NT, GROUPS>();
        const int items = ((RV + 127) >> 7) * ngrp;
        for (int it = warp; it < items; it += nw) {
            const int tile = it / ngrp, h = it - tile * ngrp, rbase = tile * 128;
            int kind[4], r[4], cend = 0;       // kind (warp-uniform): 0 none, 1 diagonal, 2 panel
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int v0 = rbase + 32 * u;
                kind[u] = v0 < ND ? 1 : (v0 < RV ? 2 : 0);
                r[u] = v0 + lane;
                if (kind[u] == 1) cend = max(cend, min(nJ, v0 + 32));
                if (kind[u] == 2) cend = nJ;
            }
            T acc[4][8];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[u][b] = T(0);
            int32_t pcm = 0;                   // packed_col(c) - c
            for (int c = 0; c < cend; ++c) {
                T tv[8];
                ld8(ts + c * RP + 8 * h, tv);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (kind[u] == 0) continue;
                    T a = T(0);
                    if (kind[u] == 1) {
                        if (r[u] >= c && r[u] < nJ) a = D[pcm + r[u]];
                    } else if (r[u] < RV) {
                        a = Pn[(r[u] - ND) * ldp + c];
                    }
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[u][b] = fma(a, tv[b], acc[u][b]);
                }
                pcm += nJ - c - 1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int j = 8 * h + b;
                    if (j >= nb) continue;
                    if (kind[u] == 1 && r[u] < nJ) xf[a0 + r[u] + (int64_t)(j0 + j) * cf.s] = acc[u][b];
                    else if (kind[u] == 2 && r[u] < RV) wb[(int64_t)(r[u] - ND) * cf.wr + j0 + j] = acc[u][b];
                }
        }
        group_sync<NT, GROUPS>();
    }
}

template <typename T, int NT, int GROUPS, int RB>
__device__ void cfwd_small_cta(const CView<T>& cf, int J, T* ts, const T* g, int64_t ldg, T* xf, int32_t nrhs, T* stg,
                               int cap, bool tiled = false) {
    constexpr int nw = NT / 32;
    const int gt = threadIdx.x % NT, lane = gt & 31, warp = gt >> 5;
    const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
    const int64_t nr = cf.r_off[J + 1] - cf.r_off[J], rtot = nJ + nr;
    const T *D, *Pn;
    const bool staged = stage_block_fwd<T, NT>(cf, J, stg, cap, gt, D, Pn);   // lands while t_J is gathered
    if (tiled && staged) {
        cfwd_small_tiled<T, NT, GROUPS>(cf, J, ts, g, ldg, xf, nrhs, D, Pn);
        return;
    }
    if (tiled) {
        // Blocks of 8 or more on a block left in HBM: t_J of up to tile_rp<T>() columns
        // gathered at once (column-major, kSmallN apart: ts holds kSmallN x tile_rp), then
        // the warp-per-four-rows products of the path below for each group of 8 columns,
        // whose 32 warp sums per quad of rows are formed by one reduce-scatter (warp_sum's
        // tree, bit for bit); the block is re-read from cache for each group.
        constexpr int RPM = tile_rp<T>();
        for (int j0 = 0; j0 < nrhs; j0 += RPM) {
            const int nbp = min(RPM, nrhs - j0);
            for (int it = gt; it < nJ * ((nbp + 7) / 8); it += NT) {
                const int i = it % nJ, h = it / nJ;
                T tv[8];
                t_entry8(cf, a0 + i, g, ldg, j0 + 8 * h, nbp - 8 * h, tv);
#pragma unroll
                for (int b = 0; b < 8; ++b) ts[(8 * h + b) * kSmallN + i] = tv[b];
            }
            group_sync<NT, GROUPS>();
            for (int h = 0; h < (nbp + 7) / 8; ++h) {
                const T* th = ts + (size_t)(8 * h) * kSmallN;
                const int nb = min(8, nbp - 8 * h);
                for (int64_t r0 = 4 * warp; r0 < rtot; r0 += 4 * nw) {
                    T acc[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) acc[q] = T(0);
                    for (int c = lane; c < nJ; c += 32) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int64_t r = r0 + u;
                            T a = T(0);
                            if (r < nJ) {
                                if (c <= r) a = D[packed_col(c, nJ) + (r - c)];
                            } else if (r < rtot) {
                                a = Pn[(r - nJ) * nJ + c];
                            }
#pragma unroll
                            for (int b = 0; b < 8; ++b) acc[8 * u + b] += a * th[b * kSmallN + c];
                        }
                    }
                    const T v = reduce_scatter<T, 32>(acc, lane);
                    const int64_t r = r0 + lane / 8;             // sum lane = 8 u + b
                    const int b = lane % 8;
                    if (r < rtot && b < nb) {
                        if (r < nJ) xf[a0 + r + (int64_t)(j0 + 8 * h + b) * cf.s] = v;
                        else cf.wbuf[(cf.r_off[J] + (r - nJ)) * cf.wr + j0 + 8 * h + b] = v;
                    }
                }
            }
            group_sync<NT, GROUPS>();
        }
        return;
    }
    for (int j0 = 0; j0 < nrhs; j0 += RB) {
        const int nb = min(RB, nrhs - j0);
        for (int b = 0; b < nb; ++b) gather_t(cf, J, gt, NT, ts + b * kSmallN, g, ldg, j0 + b);
        if (j0 == 0 && staged) stage_wait();
        group_sync<NT, GROUPS>();
        if (staged) {
            const int32_t ldp = small_ldp(nJ);
            for (int32_t r = gt; r < rtot; r += NT) {
                T acc[RB];
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] = T(0);
                if (r < nJ) {
                    // (L_JJ^{-1})[r, c] = D[packed_col(c) + r - c]; the next column's entry is n_J - c - 1 further
                    int32_t e = r;
#pragma unroll 4
                    for (int32_t c = 0; c <= r; ++c) {
                        const T a = D[e];
#pragma unroll
                        for (int b = 0; b < RB; ++b) acc[b] += a * ts[b * kSmallN + c];
                        e += nJ - c - 1;
                    }
                    for (int b = 0; b < nb; ++b) xf[a0 + r + (int64_t)(j0 + b) * cf.s] = acc[b];
                } else {
                    const T* Mr = Pn + (r - nJ) * ldp;
#pragma unroll 4
                    for (int32_t c = 0; c < nJ; ++c) {
                        const T a = Mr[c];
#pragma unroll
                        for (int b = 0; b < RB; ++b) acc[b] += a * ts[b * kSmallN + c];
                    }
                    for (int b = 0; b < nb; ++b) cf.wbuf[(cf.r_off[J] + (r - nJ)) * cf.wr + j0 + b] = acc[b];
                }
            }
        } else {
            for (int64_t r0 = 4 * warp; r0 < rtot; r0 += 4 * nw) {
                T acc[4][RB];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int b = 0; b < RB; ++b) acc[u][b] = T(0);
                for (int c = lane; c < nJ; c += 32) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t r = r0 + u;
                        T a = T(0);
                        if (r < nJ) {
                            if (c <= r) a = D[packed_col(c, nJ) + (r - c)];
                        } else if (r < rtot) {
                            a = Pn[(r - nJ) * nJ + c];
                        }
#pragma unroll
                        for (int b = 0; b < RB; ++b) acc[u][b] += a * ts[b * kSmallN + c];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int b = 0; b < RB; ++b) {
                        const T v = warp_sum(acc[u][b]);
                        const int64_t r = r0 + u;
                        if (lane == 0 && r < rtot && b < nb) {
                            if (r < nJ) xf[a0 + r + (int64_t)(j0 + b) * cf.s] = v;
                            else cf.wbuf[(cf.r_off[J] + (r - nJ)) * cf.wr + j0 + b] = v;
                        }
                    }
            }
        }
        group_sync<NT, GROUPS>();
    }
}

// backward: x_J = A_J^T [y_J; -x_{R_J}] (and scatter to DD order).  The vector is
// staged in vs; the columns, padded to a power of two P >= n_J, take P threads
// each of the NT / P parts, and part q sums its share of the rows of A_J; the
// parts' partial sums (in red) are added in a fixed order.  RB right-hand sides
// per pass (vs: RB vectors kSmallN + kSmallR apart, red: RB x NT), each with its
// single-column sequence of multiply-adds.
// shared-memory elements of the tiled backward's vector (and partial-sum) buffer
template <typename T>
__host__ __device__ constexpr int tile_vs() { return sizeof(T) == 4 ? 8192 : 4096; }

// Blocks of right-hand sides (tiled backward): the rows of A_J split into the same
// parts as the column-per-thread path below, and a thread takes 4 columns x 8
// right-hand sides of one part (a row costs four matrix loads and two 16-byte loads
// of the stacked vector, stored right-hand sides contiguous, for 32 multiply-adds).
// Each (column, part) sums its rows in order from zero (diagonal rows above the
// column add exact zeros) and the parts are added in order, as there: the same bits.
// The vector buffer (rows x RP) then holds the parts' sums (at most NT x RP).
template <typename T, int NT, int GROUPS>
__device__ void cbwd_small_tiled(const CView<T>& cf, int J, T* vs, const T* yf, T* xf, T* y_dd, int64_t ldy,
                                 int32_t nrhs, const T* D, const T* Pn, int rpm) {
    const int gt = threadIdx.x % NT;
    const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
    const int64_t nr = cf.r_off[J + 1] - cf.r_off[J], rtot = nJ + nr;
    const int32_t* R = cf.rows + cf.r_off[J];
    int P = 32;
    while (P < nJ) P *= 2;
    const int parts = NT / P, ncg = (nJ + 3) / 4;
    const int64_t len = (rtot + parts - 1) / parts;
    int32_t pcm[4];                                      // packed_col(c) - c of the thread's columns
    for (int j0 = 0; j0 < nrhs; j0 += rpm) {
        const int nb = min(rpm, nrhs - j0), RP = (nb + 7) & ~7, ngrp = RP / 8;
        // rows of [y_J; -x_{R_J}], eight right-hand sides per item (one index load)
        for (int64_t it = gt; it < rtot * ngrp; it += NT) {
            const int64_t r = it / ngrp;
            const int h = (int)(it - r * ngrp);
            const int64_t src = r < nJ ? a0 + r : R[r - nJ];
            T v[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int j = 8 * h + b;
                v[b] = T(0);
                if (j < nb) v[b] = r < nJ ? yf[src + (int64_t)(j0 + j) * cf.s] : -xf[src * cf.xr + j0 + j];
            }
#pragma unroll
            for (int b = 0; b < 8; ++b) vs[r * RP + 8 * h + b] = v[b];
        }
        if (j0 == 0) stage_wait();
        group_sync<NT, GROUPS>();
        const int items = parts * ngrp * ncg;          // at most NT: one per thread
        const bool act = gt < items;
        const int cg = act ? gt % ncg : 0, h = act ? (gt / ncg) % ngrp : 0, q = act ? gt / (ncg * ngrp) : 0;
        T acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[i][b] = T(0);
            const int c = 4 * cg + i;
            pcm[i] = (int32_t)(packed_col(c, nJ) - c);
        }
        if (act) {
            const int64_t rb = q * len, re = min(rtot, rb + len);
            for (int64_t r = rb; r < re; ++r) {
                T tv[8];
                ld8(vs + r * RP + 8 * h, tv);
                T a[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = 4 * cg + i;
                    a[i] = T(0);
                    if (c < nJ) {
                        if (r >= nJ) a[i] = Pn[(r - nJ) * nJ + c];
                        else if (r >= c) a[i] = D[pcm[i] + r];
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[i][b] = fma(a[i], tv[b], acc[i][b]);
            }
        }
        group_sync<NT, GROUPS>();                      // the vector is read: its buffer takes the sums
        if (act) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int c = 4 * cg + i, j = 8 * h + b;
                    if (c < nJ && j < nb) vs[((int64_t)q * nJ + c) * RP + j] = acc[i][b];
                }
        }
        group_sync<NT, GROUPS>();
        for (int idx = gt; idx < nJ * nb; idx += NT) {
            const int c = idx / nb, j = idx - c * nb;
            T v = T(0);
            for (int qq = 0; qq < parts; ++qq) v += vs[((int64_t)qq * nJ + c) * RP + j];
            xf[(int64_t)(a0 + c) * cf.xr + j0 + j] = v;
            if (y_dd) y_dd[cf.cperm[a0 + c] + (int64_t)(j0 + j) * ldy] = v;
        }
        group_sync<NT, GROUPS>();
    }
}

template <typename T, int NT, int GROUPS, int RB>
__device__ void cbwd_small_cta(const CView<T>& cf, int J, T* vs, T* red, const T* yf, T* xf, T* y_dd, int64_t ldy,
                               int32_t nrhs, T* stg, int cap, bool tiled = false) {
    static_assert(NT % kSmallN == 0 && NT <= 1024, "whole parts per column");
    constexpr int VS = kSmallN + kSmallR;
    const int gt = threadIdx.x % NT;
    const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
    const int64_t nr = cf.r_off[J + 1] - cf.r_off[J], rtot = nJ + nr;
    const int32_t* R = cf.rows + cf.r_off[J];
    const T *D, *Pn;
    const bool staged = stage_block<T, NT>(cf, J, stg, cap, gt, D, Pn);   // lands while the vector is staged
    if (tiled) {
        // right-hand sides per pass: the vector (rows x RP) and the sums (NT x RP) fit the buffer
        const int rpm = min(tile_rp<T>(), (int)(tile_vs<T>() / max(rtot, (int64_t)NT)) & ~7);
        if (rpm >= 8) {
            cbwd_small_tiled<T, NT, GROUPS>(cf, J, vs, yf, xf, y_dd, ldy, nrhs, D, Pn, rpm);
            return;
        }
    }
    int P = 32;
    while (P < nJ) P *= 2;
    const int parts = NT / P, part = gt / P, c = gt % P;
    const int64_t len = (rtot + parts - 1) / parts, rb = part * len, re = min(rtot, rb + len);
    for (int j0 = 0; j0 < nrhs; j0 += RB) {
        const int nb = min(RB, nrhs - j0);
        for (int b = 0; b < nb; ++b) {
            const T* x = xf + j0 + b;
            const T* y = yf + a0 + (int64_t)(j0 + b) * cf.s;
            for (int64_t r = gt; r < rtot; r += NT) vs[b * VS + r] = r < nJ ? y[r] : -x[(int64_t)R[r - nJ] * cf.xr];
        }
        if (j0 == 0 && staged) stage_wait();
        group_sync<NT, GROUPS>();
        T acc[RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[b] = T(0);
        if (c < nJ) {
            // rows of the diagonal block: (L_JJ^{-1})[r, c] for r >= c
            const T* Dc = D + packed_col(c, nJ) - c;
            const int64_t de = min(re, (int64_t)nJ);
            int64_t r = max(rb, (int64_t)c);
            for (; r + 7 < de; r += 8) {
                T a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = Dc[r + u];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int b = 0; b < RB; ++b) acc[b] += a[u] * vs[b * VS + r + u];
            }
            for (; r < de; ++r) {
                const T a = Dc[r];
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] += a * vs[b * VS + r];
            }
            // rows of the panel: M_J[r - n_J, c]
            r = max(rb, (int64_t)nJ);
            for (; r + 7 < re; r += 8) {
                T a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = Pn[(r + u - nJ) * nJ + c];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int b = 0; b < RB; ++b) acc[b] += a[u] * vs[b * VS + r + u];
            }
            for (; r < re; ++r) {
                const T a = Pn[(r - nJ) * nJ + c];
#pragma unroll
                for (int b = 0; b < RB; ++b) acc[b] += a * vs[b * VS + r];
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) red[b * NT + gt] = acc[b];
        group_sync<NT, GROUPS>();
        for (int cc = gt; cc < nJ; cc += NT)
            for (int b = 0; b < nb; ++b) {
                T v = T(0);
                for (int q = 0; q < parts; ++q) v += red[b * NT + q * P + cc];
                xf[(int64_t)(a0 + cc) * cf.xr + j0 + b] = v;
                if (y_dd) y_dd[cf.cperm[a0 + cc] + (int64_t)(j0 + b) * ldy] = v;
            }
        group_sync<NT, GROUPS>();
    }
}

constexpr int kSmallT = 256;                  // threads per supernode group of the fused levels

// ---- per-level kernels: one launch per level, NW warps per CTA (8 when the
// level has more tasks than there are SMs, so that several CTAs share an SM;
// 32 for the few wide tasks near the root)
// forward: CTA q runs panel task q (q < np) or diagonal task q - np of the level
// dynamic shared memory: t_J of rbmax right-hand sides, tstride elements apart
template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 4 : 1)
k_cfwd_level(const CView<T> cf, int32_t t0, int32_t p0, int32_t np, const T* g, int64_t ldg, T* xf, int32_t nrhs,
             int32_t tstride, int32_t rbmax) {
    extern __shared__ __align__(16) unsigned char csm[];
    __shared__ T red[NW][33];
    const int q = blockIdx.x;
    const bool pan = q < np;
    T* ts = reinterpret_cast<T*>(csm);
    T* red2 = rbmax > 1 ? ts + (size_t)rbmax * tstride : nullptr;     // NW x rbmax x 32 after t_J
    cfwd_task_cta<T, NW>(cf, pan ? cf.ptasks[p0 + q] : cf.tasks[t0 + q - np], pan, ts, tstride, rbmax, red, g, ldg, xf,
                         nrhs, red2);
}

// forward level, blocks of right-hand sides in passes of RP (cfwd_task_blk); dynamic
// shared memory: t_J (tstride x (RP + 4)), then NW x RP x 32 partial sums
template <typename T, int NW, int RP>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 2 : 1)
k_cfwd_level_blk(const CView<T> cf, int32_t t0, int32_t p0, int32_t np, T* xf, int32_t nrhs, int32_t tstride) {
    extern __shared__ __align__(16) unsigned char csm[];
    const int q = blockIdx.x;
    const bool pan = q < np;
    T* ts = reinterpret_cast<T*>(csm);
    T* red2 = ts + (size_t)tstride * (RP + 4);
    const int4 tk = pan ? cf.ptasks[p0 + q] : cf.tasks[t0 + q - np];
    for (int j0 = 0; j0 < nrhs; j0 += RP) cfwd_task_blk<T, NW, RP>(cf, tk, pan, ts, red2, xf, j0, min(RP, nrhs - j0));
}

// gf[ciperm[i] wr + j] = g[i + j ldg]: the forward's input in factor order, a row per position.
// A CTA takes 32 DD indices x 32 right-hand sides: it reads them along the indices (coalesced),
// transposes them in shared memory and writes each factor-order row's right-hand sides together.
template <typename T>
__global__ void __launch_bounds__(256)
k_cperm_g(int32_t s, int32_t nrhs, const int32_t* __restrict__ ciperm, const T* __restrict__ g, int64_t ldg, T* gf) {
    __shared__ T tile[32][33];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + ty + 8 * q, i = i0 + tx;
        tile[ty + 8 * q][tx] = (i < s && j < nrhs) ? g[i + (int64_t)j * ldg] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int il = ty + 8 * q, i = i0 + il, j = j0 + tx;
        if (i < s && j < nrhs) gf[(int64_t)ciperm[i] * nrhs + j] = tile[tx][il];
    }
}

// t_J = g_J - (gathered panel products) for every supernode of a level, once, into
// cf.tws: block (q, c) takes entries c * 256 .. c * 256 + 255 of the (position,
// right-hand side) pairs of the level's q-th supernode.  The per-level forward tasks
// then read t_J instead of each gathering it again.
template <typename T>
__global__ void __launch_bounds__(256)
k_cfwd_gather(const CView<T> cf, int32_t s0, const T* g, int64_t ldg, int32_t nrhs) {
    const int32_t J = cf.lev_sn[s0 + blockIdx.x];
    const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
    const int64_t e = (int64_t)blockIdx.y * 256 + threadIdx.x;
    if (e >= (int64_t)nJ * nrhs) return;
    const int32_t i = (int32_t)(e / nrhs), j = (int32_t)(e % nrhs);   // right-hand sides fastest
    const int32_t pos = a0 + i;
    cf.tws[(int64_t)pos * cf.wr + j] =
        g_at(cf, pos, g, ldg, j) -
        gather_sum(cf.wbuf + j, cf.wr, cf.seg_row, cf.seg_ptr[pos], cf.seg_ptr[pos + 1]);
}

// backward: one CTA per column task, 16 (FP32) or 8 (FP64) panel loads in flight per
// lane for one right-hand side, 4 for a block of four
template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 4 : 1)
k_cbwd_level(const CView<T> cf, int32_t t0, const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char csm[];
    __shared__ T red[NW][33];
    __shared__ T us[8 * 32];
    T* red2 = nrhs >= 4 ? reinterpret_cast<T*>(csm) : nullptr;        // NW x 8 x 32
    cbwd_task_cta<T, NW, sizeof(T) == 4 ? 16 : 8, 4>(cf, cf.tasks[t0 + blockIdx.x], us, 8, red, yf, xf, y_dd, ldy,
                                                      nrhs, red2);
}

// backward level, blocks of right-hand sides in passes of RP (cbwd_task_blk); dynamic
// shared memory: us (RP x 32), then xs (NW x 32 x (RP + 4))
template <typename T, int NW, int RP>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 2 : 1)
k_cbwd_level_blk(const CView<T> cf, int32_t t0, const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char csm[];
    T* us = reinterpret_cast<T*>(csm);
    T* xs = us + RP * 32;
    const int4 tk = cf.tasks[t0 + blockIdx.x];
    for (int j0 = 0; j0 < nrhs; j0 += RP)
        cbwd_task_blk<T, NW, RP>(cf, tk, us, xs, yf, xf, y_dd, ldy, j0, min(RP, nrhs - j0));
}

// right-hand sides per pass of the fused small levels' per-level kernels
constexpr int kSmallRBf = 8, kSmallRBb = 4;

// dynamic shared memory: t_J (tsz elements: kSmallRBf right-hand sides, or tile_rp
// contiguous ones for the tiled path of blocks of 8 or more), then the stage buffer
// of cap elements
template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2)
k_cfwd_small(const CView<T> cf, int32_t s0, const T* g, int64_t ldg, T* xf, int32_t nrhs, int32_t cap, int32_t tsz) {
    extern __shared__ __align__(16) unsigned char csm[];
    T* ts = reinterpret_cast<T*>(csm);
    cfwd_small_cta<T, kThreads, 1, kSmallRBf>(cf, cf.lev_sn[s0 + blockIdx.x], ts, g, ldg, xf, nrhs, ts + tsz, cap,
                                              tsz == kSmallN * tile_rp<T>());
}

// dynamic shared memory (vsz elements): kSmallRBb vectors of kSmallN + kSmallR and
// kSmallRBb x kThreads partial sums, or for blocks of 8 or more the tiled path's
// buffer, then the stage buffer of cap elements
template <typename T>
__host__ __device__ constexpr int small_bwd_vsz(bool tiled) {
    return tiled ? (tile_vs<T>() > kSmallRBb * (kSmallN + kSmallR + kThreads) ? tile_vs<T>()
                                                                              : kSmallRBb * (kSmallN + kSmallR + kThreads))
                 : kSmallRBb * (kSmallN + kSmallR + kThreads);
}
template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2)
k_cbwd_small(const CView<T> cf, int32_t s0, const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs, int32_t cap,
             bool tiled) {
    extern __shared__ __align__(16) unsigned char csm[];
    T* vs = reinterpret_cast<T*>(csm);
    T* red = vs + kSmallRBb * (kSmallN + kSmallR);
    cbwd_small_cta<T, kThreads, 1, kSmallRBb>(cf, cf.lev_sn[s0 + blockIdx.x], vs, red, yf, xf, y_dd, ldy, nrhs,
                                              vs + small_bwd_vsz<T>(tiled), cap, tiled);
}


// ---- top zone: x_T = L_TT^{-1} t_T and y_T = L_TT^{-T} x_T with the explicit inverse
// (local index la of the zone's positions; tpos maps it to the factor order)
constexpr int kTopT = 256;   // threads of the zone kernels (8 warps)

// t_T = g_T - (panel products of the supernodes below the zone), one thread per (la, j)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_ctop_gather(const CView<T> cf, const T* g, int64_t ldg, int32_t nrhs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)cf.nT * nrhs) return;
    const int32_t la = (int32_t)(i % cf.nT), j = (int32_t)(i / cf.nT);
    cf.tT[i] = g_at(cf, cf.tpos[la], g, ldg, j) -
               gather_sum(cf.wbuf + j, cf.wr, cf.tseg_row, cf.tseg_ptr[la], cf.tseg_ptr[la + 1]);
}

// Adds the chunks' partial sums of a block once all its tasks have stored theirs:
// every task fences its stores and counts itself in; the last one to arrive reads
// the partials (in chunk order, so the sum does not depend on the arrival order),
// calls out(r, j, sum) and clears the counter for the next solve.
template <typename T, typename Out>
__device__ __forceinline__ void last_task_sum(int32_t* cnt, int nch, const T* part, int64_t pstride, int count,
                                              int32_t nrhs, Out out) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(cnt, 1) == nch - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < count * nrhs; i += blockDim.x) {
        const int r = i % count, j = i / count;
        const T* pj = part + (int64_t)j * pstride + r;
        T v = T(0);
        for (int k = 0; k < nch; ++k) v += __ldcg(pj + (int64_t)k * 32);
        out(r, j, v);
    }
    if (threadIdx.x == 0) *cnt = 0;
}

// forward task (row block rb, columns [cb, ce), chunk k): partial sums of rows
// r0 .. r0 + count - 1 of L_TT^{-1} t_T over the chunk; a warp takes rows
// w, w + 8, w + 16, w + 24 (four in flight), lanes over the columns
template <typename T>
__global__ void __launch_bounds__(kTopT)
k_ctop_fwd(const CView<T> cf, T* xf, int32_t nrhs) {
    __shared__ T ts[kTopCW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 tk = cf.tf_tasks[blockIdx.x];
    const int4 rb = cf.tf_rb[tk.x];
    int64_t off[4];
    int la[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = warp + 8 * u;
        la[u] = r < rb.y ? rb.x + r : -1;
        off[u] = r < rb.y ? cf.tsk_off[la[u]] - cf.tsk_lo[la[u]] : 0;
    }
    for (int j = 0; j < nrhs; ++j) {
        const T* t = cf.tT + (int64_t)j * cf.nT;
        for (int c = tk.y + threadIdx.x; c < tk.z; c += kTopT) ts[c - tk.y] = t[c];
        __syncthreads();
        T acc[4] = {T(0), T(0), T(0), T(0)};
        int c = tk.y + lane;
        // sixteen loads in flight per lane (four rows x four columns); entries right
        // of a row's diagonal, and rows past the block, load nothing
        for (; c + 96 < tk.z; c += 128) {
            T a[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < 4; ++q) a[u][q] = c + 32 * q <= la[u] ? cf.tsk[off[u] + c + 32 * q] : T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T tv = ts[c + 32 * q - tk.y];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] += a[u][q] * tv;
            }
        }
        for (; c < tk.z; c += 32) {
            const T tv = ts[c - tk.y];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c <= la[u]) acc[u] += cf.tsk[off[u] + c] * tv;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T v = warp_sum(acc[u]);
            if (lane == 0 && la[u] >= 0)
                cf.tf_part[(int64_t)j * cf.tf_parts + rb.w + tk.w * 32 + warp + 8 * u] = v;
        }
        __syncthreads();
    }
    last_task_sum(cf.tf_cnt + tk.x, rb.z, cf.tf_part + rb.w, cf.tf_parts, rb.y, nrhs,
                  [&](int r, int j, T v) { xf[cf.tpos[rb.x + r] + (int64_t)j * cf.s] = v; });
}

// backward task (column block cb of J, path rows [r0, r1), chunk k): partial sums of
// columns c0 .. c0 + count - 1 of X_J^T x over the chunk (lanes over the columns,
// the warps split the rows, 16 (FP32) or 8 (FP64) loads in flight); the chunk's x
// values are staged in shared memory
template <typename T>
__global__ void __launch_bounds__(kTopT)
k_ctop_bwd(const CView<T> cf, const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs) {
    constexpr int NW = kTopT / 32, DEPTH = sizeof(T) == 4 ? 16 : 8;
    __shared__ T xs[kTopRCH];
    __shared__ T red[NW][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 tk = cf.tb_tasks[blockIdx.x];
    const int4 cb = cf.tb_cb[tk.x];
    const int32_t J = cb.x, nJ = cf.c0[J + 1] - cf.c0[J], pofs = cf.tb_cb_part[tk.x];
    const T* X = cf.tb + cf.tb_off[J] + cb.y + lane;
    const int32_t* pp = cf.tp_pos + cf.tp_off[J];
    const int nrw = tk.z - tk.y, per = (nrw + NW - 1) / NW;
    const int rb = tk.y + warp * per, re = min(tk.z, rb + per);
    for (int j = 0; j < nrhs; ++j) {
        for (int r = tk.y + threadIdx.x; r < tk.z; r += kTopT) xs[r - tk.y] = yf[pp[r] + (int64_t)j * cf.s];
        __syncthreads();
        T acc = T(0);
        if (lane < cb.z) {
            int r = rb;
            for (; r + DEPTH - 1 < re; r += DEPTH) {
                T a[DEPTH];
#pragma unroll
                for (int u = 0; u < DEPTH; ++u) a[u] = X[(int64_t)(r + u) * nJ];
#pragma unroll
                for (int u = 0; u < DEPTH; ++u) acc += a[u] * xs[r + u - tk.y];
            }
            for (; r < re; ++r) acc += X[(int64_t)r * nJ] * xs[r - tk.y];
        }
        red[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && lane < cb.z) {
            T v = T(0);
#pragma unroll
            for (int w = 0; w < NW; ++w) v += red[w][lane];
            cf.tb_part[(int64_t)j * cf.tb_parts + pofs + tk.w * 32 + lane] = v;
        }
        __syncthreads();
    }
    const int32_t a0 = cf.c0[J] + cb.y;
    last_task_sum(cf.tb_cnt + tk.x, cb.w, cf.tb_part + pofs, cf.tb_parts, cb.z, nrhs, [&](int c, int j, T v) {
        xf[(int64_t)(a0 + c) * cf.xr + j] = v;
        if (y_dd) y_dd[cf.cperm[a0 + c] + (int64_t)j * ldy] = v;
    });
}

// ---- persistent kernels: every level in one cooperative launch
constexpr int kPersT = 1024;                  // 32 warps, one CTA per SM
constexpr int kPersW = kPersT / 32;
constexpr int kSmallG = kPersT / kSmallT;     // fused levels: 4 groups of 256 threads, a supernode each
// All CTAs arrive; the counter (zeroed before the launch) reaches target =
// round x gridDim.x.  A wait polls at most `spin` times (64 ns sleep between
// polls); one that runs out sets the status word and goes on (the CTAs then
// compute on inputs that may not be final: every index they use comes from the
// factor's structure, so nothing reads or writes out of bounds); once the
// status word is set, later waits give up early too.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned target, int32_t* err, long long spin) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        long long it = 0;
        while (*reinterpret_cast<volatile unsigned*>(bar) < target) {
            if (++it > spin) {
                atomicExch(err, 2);
                break;
            }
            if ((it & 1023) == 0 && *reinterpret_cast<volatile int32_t*>(err)) break;   // already failed
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

// Shared memory of the persistent kernels (elements): t_J plus the reduction
// array of a forward task, or the fused levels' buffers, whichever is larger.
// The reduction array starts at a multiple of 32 elements.
// t_J of rb right-hand sides (rb x max_n) before it; at least the backward's
// 4 x 32 block of diagonal results, which shares the start of the buffer.
inline int64_t pers_red_off(int32_t max_n, int32_t rb = 1) {
    return std::max<int64_t>(((int64_t)rb * max_n + 31) / 32 * 32, 4 * 32);
}
// Each fused-level group also gets a stage buffer of stage_cap elements.
inline size_t pers_smem_bytes(int32_t max_n, size_t elem, int32_t stage_cap, int32_t rb = 1) {
    const int64_t task = pers_red_off(max_n, rb) + kPersW * 33 + 32;
    const int64_t small_fwd = kSmallG * ((int64_t)kSmallN + stage_cap),
                  small_bwd = kSmallG * ((int64_t)kSmallN + kSmallR + kSmallT + stage_cap);
    return (size_t)std::max({task, small_fwd, small_bwd}) * elem;
}

template <typename T>
__global__ void __launch_bounds__(kPersT, 1)
k_cfwd_persistent(const CView<T> cf, const T* g, int64_t ldg, T* xf, int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char psm[];
    T* sm = reinterpret_cast<T*>(psm);
    T(*red)[33] = reinterpret_cast<T(*)[33]>(sm + cf.red_off);
    unsigned round = 0;
    int steps_left = cf.nsteps;
    for (int l = 0; l < cf.nlev; ++l) {
        bool any;
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            any = ns > 0;
            const int grp = threadIdx.x / kSmallT;
            T* gs = sm + grp * ((int64_t)kSmallN + cf.stage_cap);
            for (int q = blockIdx.x * kSmallG + grp; q < ns; q += gridDim.x * kSmallG)
                cfwd_small_cta<T, kSmallT, kSmallG, 1>(cf, cf.lev_sn[s0 + q], gs, g, ldg, xf, nrhs, gs + kSmallN,
                                                    cf.stage_cap);
        } else {
            const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
            const int p0 = cf.lev_ptask_ptr[l], np = cf.lev_ptask_ptr[l + 1] - p0;
            any = nt + np > 0;
            for (int q = blockIdx.x; q < np + nt; q += gridDim.x) {
                const bool pan = q < np;
                cfwd_task_cta<T, kPersW, 4>(cf, pan ? cf.ptasks[p0 + q] : cf.tasks[t0 + q - np], pan, sm,
                                            cf.pers_tstride, cf.pers_rb, red, g, ldg, xf, nrhs);
            }
        }
        if (any && --steps_left > 0) grid_barrier(cf.bar, ++round * gridDim.x, cf.err, cf.spin);
    }
}

template <typename T>
__global__ void __launch_bounds__(kPersT, 1)
k_cbwd_persistent(const CView<T> cf, const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char psm[];
    T* sm = reinterpret_cast<T*>(psm);
    T(*red)[33] = reinterpret_cast<T(*)[33]>(sm + cf.red_off);
    unsigned round = 0;
    int steps_left = cf.nsteps;
    for (int l = cf.nlev - 1; l >= 0; --l) {
        bool any;
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            any = ns > 0;
            const int grp = threadIdx.x / kSmallT;
            T* gs = sm + grp * ((int64_t)kSmallN + kSmallR + kSmallT + cf.stage_cap);
            for (int q = blockIdx.x * kSmallG + grp; q < ns; q += gridDim.x * kSmallG)
                cbwd_small_cta<T, kSmallT, kSmallG, 1>(cf, cf.lev_sn[s0 + q], gs, gs + kSmallN + kSmallR, yf, xf, y_dd,
                                                    ldy, nrhs, gs + kSmallN + kSmallR + kSmallT, cf.stage_cap);
        } else {
            const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
            any = nt > 0;
            for (int q = blockIdx.x; q < nt; q += gridDim.x)
                cbwd_task_cta<T, kPersW, 8, 4, 4>(cf, cf.tasks[t0 + q], sm, 4, red, yf, xf, y_dd, ldy, nrhs);
        }
        if (any && --steps_left > 0) grid_barrier(cf.bar, ++round * gridDim.x, cf.err, cf.spin);
    }
}

// ------------------------------------------------------------------ K4
// w' = cinv w + U (d o (U^T w)) (Eq. 4.7 in U-form), U s x k column-major, w s x nrhs
// column-major (leading dimension ldw).  Each pass reads U once:
//   k_lr_vt     part[b][kk][j] = sum over block b's rows of U[i, kk] w[i, j]
//   k_lr_vt_fin vk[kk + j k] = d[kk] * sum over b of part[b][kk][j]
//   k_lr_update w[i, j] = cinv w[i, j] + sum over kk of U[i, kk] vk[kk + j k]
// Every sum runs in a fixed order that depends on s and k only (block b owns rows
// [b R, b R + R), lanes stride them, the warp's sums follow warp_sum's tree; the
// blocks are added in fixed segments), so a column gives the same bits alone and
// inside a block.
constexpr int kLrMaxBlocks = 1024;

// row blocks of the first pass: enough to fill the SMs, a fixed function of s
__host__ __device__ inline int lr_blocks(int32_t s) {
    const int b = (s + 127) / 128;
    return b < 1 ? 1 : (b > kLrMaxBlocks ? kLrMaxBlocks : b);
}

// Pass 1: CTA b owns rows [b R, b R + R) of s; warp w takes the columns kk = w, w + 8,
// ... of U; its lanes stride the rows (U and w read coalesced, U once), each lane
// keeping eight right-hand sides' sums, which one reduce-scatter (warp_sum's tree)
// turns into the CTA's partial sums.  The order of every sum depends on s only.
template <typename T>
__global__ void __launch_bounds__(256)
k_lr_vt(int32_t s, int32_t k, int32_t nrhs, const T* __restrict__ U, const T* __restrict__ w, int64_t ldw, T* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = (s + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * R, r1 = min(s, r0 + R);
    if (nrhs == 1 && k <= 128) {
        // one right-hand side: the warp's columns kk = warp + 8 q (q < 16) all at once, w read
        // once per row and their loads of U in flight together; each sum has the operands and
        // the tree of the block path below, so the bits are the same
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = T(0);
        for (int i = r0 + lane; i < r1; i += 32) {
            const T wv = w[i];
            T u[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) u[q] = warp + 8 * q < k ? U[i + (int64_t)(warp + 8 * q) * s] : T(0);
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (warp + 8 * q < k) acc[q] = fma(u[q], wv, acc[q]);
        }
        const T v = reduce_scatter<T, 16>(acc, lane);
        const int kk = warp + 8 * rs_index<16>(lane);
        if (rs_writer<16>(lane) && kk < k) part[(int64_t)blockIdx.x * k + kk] = v;
        return;
    }
    for (int kk = warp; kk < k; kk += 8) {
        const T* Uc = U + (int64_t)kk * s;
        for (int j0 = 0; j0 < nrhs; j0 += 8) {
            const int jn = min(8, nrhs - j0);
            T acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = T(0);
            for (int i = r0 + lane; i < r1; i += 32) {
                const T u = Uc[i];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < jn) acc[q] = fma(u, w[i + (int64_t)(j0 + q) * ldw], acc[q]);
            }
            const T v = reduce_scatter<T, 8>(acc, lane);
            const int q = rs_index<8>(lane);
            if (rs_writer<8>(lane) && q < jn) part[((int64_t)blockIdx.x * k + kk) * nrhs + j0 + q] = v;
        }
    }
}

// vk = d o (sum over the G pass-1 blocks), in a fixed order: block (kk, group of 16
// right-hand sides) sums kFinSeg segments of the blocks in order, reading the
// right-hand sides coalesced, then adds the segments in order
constexpr int kLrSeg = 16, kLrFinJ = 16;
template <typename T>
__global__ void __launch_bounds__(kLrSeg * kLrFinJ)
k_lr_vt_fin(int32_t k, int32_t nrhs, int32_t G, const T* __restrict__ part, const T* __restrict__ dvec, T* vk) {
    __shared__ T seg[kLrSeg][kLrFinJ];
    const int kk = blockIdx.x, jl = threadIdx.x % kLrFinJ, q = threadIdx.x / kLrFinJ;
    const int j = blockIdx.y * kLrFinJ + jl;
    const int len = (G + kLrSeg - 1) / kLrSeg, b0 = q * len, b1 = min(G, b0 + len);
    T acc = T(0);
    if (j < nrhs) {
        int b = b0;
        for (; b + 4 <= b1; b += 4) {
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = part[((int64_t)(b + u) * k + kk) * nrhs + j];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += v[u];
        }
        for (; b < b1; ++b) acc += part[((int64_t)b * k + kk) * nrhs + j];
    }
    seg[q][jl] = acc;
    __syncthreads();
    if (q == 0 && j < nrhs) {
        T v = T(0);
        for (int qq = 0; qq < kLrSeg; ++qq) v += seg[qq][jl];
        vk[kk + (int64_t)j * k] = dvec[kk] * v;
    }
}

// thread = row i, JG right-hand sides (a block's columns j0 .. j0 + JG - 1 of nrhs)
template <typename T, int JG>
__global__ void __launch_bounds__(256)
k_lr_update(int32_t s, int32_t k, int32_t nrhs, const T* __restrict__ U, const T* __restrict__ vk, T cinv, T* w,
            int64_t ldw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s) return;
    const int j0 = blockIdx.y * JG;
    const int jn = min(JG, nrhs - j0);
    T acc[JG];
#pragma unroll
    for (int q = 0; q < JG; ++q) acc[q] = q < jn ? cinv * w[i + (int64_t)(j0 + q) * ldw] : T(0);
    int kk = 0;
    if constexpr (JG == 1)                              // one column: eight loads of U in flight, then their products
    for (; kk + 8 <= k; kk += 8) {
        T u[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) u[e] = U[i + (int64_t)(kk + e) * s];
#pragma unroll
        for (int e = 0; e < 8; ++e)
#pragma unroll
            for (int q = 0; q < JG; ++q)
                if (q < jn) acc[q] = fma(u[e], __ldg(&vk[kk + e + (int64_t)(j0 + q) * k]), acc[q]);
    }
    for (; kk < k; ++kk) {
        const T u = U[i + (int64_t)kk * s];
#pragma unroll
        for (int q = 0; q < JG; ++q)
            if (q < jn) acc[q] = fma(u, __ldg(&vk[kk + (int64_t)(j0 + q) * k]), acc[q]);
    }
#pragma unroll
    for (int q = 0; q < JG; ++q)
        if (q < jn) w[i + (int64_t)(j0 + q) * ldw] = acc[q];
}

// ------------------------------------------------------------------ helpers
template <typename TS, typename TD>
__global__ void k_convert(int64_t rows, int32_t cols, const TS* src, int64_t lds, TD* dst, int64_t ldd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    dst[i + j * ldd] = (TD)src[i + j * lds];
}

__global__ void k_permute(int32_t n, int32_t nrhs, const int32_t* __restrict__ idx, const double* src, int64_t lds,
                          double* dst, int64_t ldd, int gather) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    const int32_t a = (int32_t)(t % n), j = (int32_t)(t / n);
    if (gather) dst[a + j * ldd] = src[idx[a] + j * lds];
    else dst[idx[a] + j * ldd] = src[a + j * lds];
}

__global__ void __launch_bounds__(kThreads)
k_dot_partial(int64_t n, const double* a, int64_t lda, const double* b, int64_t ldb, double* part) {
    __shared__ double red[kThreads / 32];
    const int j = blockIdx.y;
    const double* x = a + j * lda;
    const double* y = b + j * ldb;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * y[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[(int64_t)j * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_dot_final(int32_t cols, int32_t G, const double* part, double* out, int32_t stride) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= cols) return;
    double acc = 0.0;
    for (int b = lane; b < G; b += 32) acc += part[(int64_t)j * G + b];
    acc = warp_sum(acc);
    if (lane == 0) out[(int64_t)j * stride] = acc;
}

__global__ void k_gemv_n_sub(int32_t s, int32_t jn, const double* __restrict__ V, const double* __restrict__ h,
                             double* w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s) return;
    double acc = 0.0;
    for (int q = 0; q < jn; ++q) acc += V[i + (int64_t)q * s] * h[q];
    w[i] -= acc;
}

__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (b == 0.0) ? a * x[i] : a * x[i] + b * y[i];   // b = 0: y is not read
}

__global__ void k_gemm_nn(int32_t s, int32_t m, int32_t k, const double* __restrict__ V,
                          const double* __restrict__ Y, double* U) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)s * k) return;
    const int32_t i = (int32_t)(idx % s), kk = (int32_t)(idx / s);
    double acc = 0.0;
    for (int q = 0; q < m; ++q) acc += V[i + (int64_t)q * s] * Y[q + (int64_t)kk * m];
    U[i + (int64_t)kk * s] = acc;
}

// ------------------------------------------------------------------ K5 scalars
// scal[8 j + ...]: 0 rho, 1 p.q, 2 alpha, 3 r.r, 4 b.b, 5 beta, 6 rho_new, 7 r.z_old
// flags[4 j + ...]: 0 active, 1 iterations, 2 status (0 running, 1 converged,
// 2 breakdown); flags[4 nrhs] = number of active columns
__global__ void k_pcg_alpha(int32_t nrhs, double* scal, int32_t* flags) {
    const int j = threadIdx.x;
    if (j >= nrhs || !flags[4 * j]) return;
    double* sc = scal + 8 * j;
    if (!(sc[1] > 0.0)) {
        flags[4 * j] = 0;
        flags[4 * j + 2] = 2;
        sc[2] = 0.0;
        return;
    }
    sc[2] = sc[0] / sc[1];
}

__global__ void k_pcg_update_xr(int32_t n, int32_t nrhs, double* x, double* r, const double* p, const double* q,
                                const double* scal, const int32_t* flags) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    const int32_t j = (int32_t)(t / n);
    if (!flags[4 * j]) return;
    const double a = scal[8 * j + 2];
    x[t] += a * p[t];
    r[t] -= a * q[t];
}

__global__ void k_pcg_check(int32_t nrhs, double* scal, int32_t* flags, int32_t it, double tol) {
    if (threadIdx.x != 0) return;
    int32_t active = 0;
    for (int j = 0; j < nrhs; ++j) {
        if (!flags[4 * j]) continue;
        const double* sc = scal + 8 * j;
        flags[4 * j + 1] = it;
        if (sc[3] <= tol * tol * sc[4]) {
            flags[4 * j] = 0;
            flags[4 * j + 2] = 1;
        } else {
            ++active;
        }
    }
    flags[4 * nrhs] = active;
}

// PCG start: a column is active unless its right-hand side is zero; iteration counter 0
__global__ void k_pcg_init(int32_t nrhs, const double* scal, int32_t* flags) {
    if (threadIdx.x != 0) return;
    int32_t act = 0;
    for (int j = 0; j < nrhs; ++j) {
        const bool zero = !(scal[8 * j + 4] > 0.0);
        flags[4 * j] = zero ? 0 : 1;
        flags[4 * j + 1] = 0;
        flags[4 * j + 2] = zero ? 1 : 0;
        flags[4 * j + 3] = 0;
        act += !zero;
    }
    flags[4 * nrhs] = act;
    flags[4 * nrhs + 1] = 0;
}

// Convergence test inside the PCG graph: ctl = [tol^2, maxit].  Sets the WHILE
// condition (another iteration is needed) and the IF condition that runs the
// preconditioner update at the top of every iteration after the first.
__global__ void k_pcg_check_graph(int32_t nrhs, const double* scal, int32_t* flags, const double* ctl,
                                  cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_if) {
    if (threadIdx.x != 0) return;
    const int32_t it = ++flags[4 * nrhs + 1];
    int32_t active = 0;
    for (int j = 0; j < nrhs; ++j) {
        if (!flags[4 * j]) continue;
        const double* sc = scal + 8 * j;
        flags[4 * j + 1] = it;
        if (sc[3] <= ctl[0] * sc[4]) {
            flags[4 * j] = 0;
            flags[4 * j + 2] = 1;
        } else {
            ++active;
        }
    }
    flags[4 * nrhs] = active;
    cudaGraphSetConditional(h_while, (active > 0 && it < (int32_t)ctl[1]) ? 1u : 0u);
    cudaGraphSetConditional(h_if, 1u);
}

__global__ void k_pcg_beta(int32_t nrhs, double* scal, const int32_t* flags, int32_t flexible) {
    const int j = threadIdx.x;
    if (j >= nrhs || !flags[4 * j]) return;
    double* sc = scal + 8 * j;
    const double num = flexible ? sc[6] - sc[7] : sc[6];
    sc[5] = num / sc[0];
    sc[0] = sc[6];
}

__global__ void k_pcg_update_p(int32_t n, int32_t nrhs, double* p, const double* z, const double* scal,
                               const int32_t* flags) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    const int32_t j = (int32_t)(t / n);
    if (!flags[4 * j]) return;
    p[t] = z[t] + scal[8 * j + 5] * p[t];
}

// Slot CG (continuous batching): slot j starts with p = 0, z = 0 and a unit
// placeholder for rho, so the preconditioner update of its first iteration gives
// p = z exactly and every slot runs the same kernels at every iteration.
// ctl[2 j] = tol^2, ctl[2 j + 1] = maxit of slot j.
__global__ void k_cg_slot_init(int32_t j, double tol, int32_t maxit, double* scal, int32_t* flags, double* ctl) {
    if (threadIdx.x != 0) return;
    double* sc = scal + 8 * j;
    const bool zero = !(sc[4] > 0.0);
    sc[0] = 1.0;
    sc[3] = sc[4];
    flags[4 * j] = zero ? 0 : 1;
    flags[4 * j + 1] = 0;
    flags[4 * j + 2] = zero ? 1 : 0;
    flags[4 * j + 3] = 0;
    ctl[2 * j] = tol * tol;
    ctl[2 * j + 1] = (double)maxit;
}

// after an iteration's test part: each active slot counts the iteration and stops
// when its residual meets its tolerance (status 1) or at its own maxit (status 0)
__global__ void k_cg_slot_check(int32_t width, int32_t count_at, const double* scal, int32_t* flags,
                                const double* ctl) {
    if (threadIdx.x != 0) return;
    int32_t active = 0;
    for (int j = 0; j < width; ++j) {
        if (!flags[4 * j]) continue;
        const double* sc = scal + 8 * j;
        const int32_t it = ++flags[4 * j + 1];
        if (sc[3] <= ctl[2 * j] * sc[4]) {
            flags[4 * j] = 0;
            flags[4 * j + 2] = 1;
        } else if (it >= (int32_t)ctl[2 * j + 1]) {
            flags[4 * j] = 0;
        } else {
            ++active;
        }
    }
    flags[count_at] = active;                  // past every slot's words
}

inline unsigned blocks_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// every kernel launch of the library goes through this counter
inline void counted(int n = 1) { count_launches(n); }

template <typename T>
cudaError_t spmv_cols(int32_t rows, int32_t nrhs, const int32_t* rp, const int32_t* ci, const T* v, const T* x,
                      int64_t ldx, const T* g, int64_t ldg, T* y, int64_t ldy, cudaStream_t st) {
    if (rows == 0 || nrhs == 0) return cudaSuccess;
    const int64_t threads = (int64_t)rows * ((nrhs + kSpCols - 1) / kSpCols);
    k_spmv_cols<T><<<blocks_for(threads), kThreads, 0, st>>>(rows, nrhs, rp, ci, v, x, ldx, g, ldg, y, ldy);
    counted();
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------------ launchers

template <typename T>
cudaError_t launch_gather_et(const DevOperator<T>& op, int32_t s, const T* g, int64_t ldg, const T* t,
                             int64_t ldt, T* gp, int64_t ldgp, int32_t nrhs, cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    return spmv_cols<T>(s, nrhs, op.et_rp, op.et_ci, op.et_v, t, ldt, g, ldg, gp, ldgp, st);
}

template <typename T>
cudaError_t launch_spmv_e(const DevOperator<T>& op, int32_t nI, const T* y, int64_t ldy, T* out, int64_t ldo,
                          int32_t nrhs, cudaStream_t st) {
    if (nI == 0) return cudaSuccess;
    return spmv_cols<T>(nI, nrhs, op.e_rp, op.e_ci, op.e_v, y, ldy, nullptr, 0, out, ldo, st);
}

// Grid of a persistent solve on the current device: one CTA per SM (fewer if
// no step has that many CTA tasks), 0 if the kernel cannot be co-resident.
// Raises a kernel's dynamic shared-memory limit to the opt-in maximum less its
// static shared memory, once per kernel (the limit is process-wide per kernel, so
// it is never set per launch).  False if the device refuses.
bool raise_smem_once(const void* kern) {
    static std::mutex mu;
    static std::vector<const void*> raised;
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(raised.begin(), raised.end(), kern) != raised.end()) return true;
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    raised.push_back(kern);
    return true;
}
constexpr size_t kLevSmem = 200 * 1024;   // dynamic shared memory a per-level forward kernel may take

template <typename K>
int pers_grid(K kern, size_t smem, int32_t max_cta_tasks) {
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (smem > 48 * 1024 && !raise_smem_once((const void*)kern)) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPersT, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return 0;
    }
    return std::max(1, std::min(nsm, max_cta_tasks));
}

template <typename T>
CView<T> make_view(const DevCFactor<T>& cf, int32_t nsteps) {
    CView<T> v;
    v.s = cf.s;
    v.nlev = cf.top_lev;   // the level-scheduled part: levels below the top zone
    v.nsteps = nsteps;
    v.nrow = cf.nrow;
    v.wr = 1;
    v.xr = 1;
    v.gf = nullptr;
    v.cperm = cf.cperm;
    v.c0 = cf.c0;
    v.rows = cf.rows;
    v.seg_row = cf.seg_row;
    v.lev_sn = cf.lev_sn;
    v.r_off = cf.r_off;
    v.pan_off = cf.pan_off;
    v.dinv_off = cf.dinv_off;
    v.seg_ptr = cf.seg_ptr;
    v.panel = cf.panel;
    v.dinv = cf.dinv;
    v.wbuf = cf.wbuf;
    v.tws = nullptr;
    v.tasks = cf.tasks;
    v.ptasks = cf.ptasks;
    v.lev_task_ptr = cf.d_lev_task_ptr;
    v.lev_ptask_ptr = cf.d_lev_ptask_ptr;
    v.lev_sn_ptr = cf.d_lev_sn_ptr;
    v.lev_small = cf.d_lev_small;
    v.red_off = pers_red_off(cf.max_n);
    v.pers_rb = 1;
    v.pers_tstride = 0;
    v.stage_cap = cf.stage_cap;
    v.nT = cf.nT;
    v.tf_parts = cf.tf_parts;
    v.tb_parts = cf.tb_parts;
    v.tpos = cf.tpos;
    v.tseg_row = cf.tseg_row;
    v.tsk_lo = cf.tsk_lo;
    v.tp_pos = cf.tp_pos;
    v.tb_cb_part = cf.tb_cb_part;
    v.tseg_ptr = cf.tseg_ptr;
    v.tsk_off = cf.tsk_off;
    v.tb_off = cf.tb_off;
    v.tp_off = cf.tp_off;
    v.tsk = cf.tsk;
    v.tb = cf.tb;
    v.tf_rb = cf.tf_rb;
    v.tf_tasks = cf.tf_tasks;
    v.tb_cb = cf.tb_cb;
    v.tb_tasks = cf.tb_tasks;
    v.tT = cf.tT;
    v.tf_part = cf.tf_part;
    v.tb_part = cf.tb_part;
    v.tf_cnt = cf.tf_cnt;
    v.tb_cnt = cf.tb_cnt;
    v.bar = cf.bar;
    v.err = cf.err;
    v.spin = cf.grid_spin;
    return v;
}

// one cooperative launch; the barrier counter is zeroed first on the same stream
template <typename K, typename... A>
cudaError_t launch_persistent(K kern, int grid, size_t smem, unsigned* bar, cudaStream_t st, A... args) {
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPersT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, args...);
    counted();
    return e;
}

template <typename T>
cudaError_t launch_c_forward(const DevCFactor<T>& cf, const T* g_dd, int64_t ldg, T* xf, int32_t nrhs,
                             cudaStream_t st) {
    if (nrhs > cf.ws_cols) return cudaErrorInvalidValue;
    CView<T> v = make_view(cf, cf.nsteps_fwd);
    v.wr = nrhs;     // wbuf and tws: a call's right-hand sides contiguous per row (one line per gathered row)
    if (nrhs >= 8 && cf.gfs && cf.s > 0) {
        // blocks: g in factor order, a row per position, so every gather of g reads whole lines
        k_cperm_g<T><<<dim3((cf.s + 31) / 32, (nrhs + 31) / 32), 256, 0, st>>>(cf.s, nrhs, cf.ciperm, g_dd, ldg,
                                                                               cf.gfs);
        counted();
        v.gf = cf.gfs;
    }
    bool levels_done = cf.nsteps_fwd == 0;
    if (!levels_done && !cf.per_level) {
        // blocks of four right-hand sides share each matrix load when t_J of four fits
        const int32_t rb = (nrhs >= 4 && pers_smem_bytes(cf.max_n, sizeof(T), cf.stage_cap, 4) <= kLevSmem) ? 4 : 1;
        v.pers_rb = rb;
        v.pers_tstride = cf.max_n;
        v.red_off = pers_red_off(cf.max_n, rb);
        const size_t smem = pers_smem_bytes(cf.max_n, sizeof(T), cf.stage_cap, rb);
        const int grid = pers_grid(k_cfwd_persistent<T>, smem, cf.max_cta_tasks);
        if (grid > 0) {
            const cudaError_t e = launch_persistent(k_cfwd_persistent<T>, grid, smem, cf.bar, st, v, g_dd, ldg, xf, nrhs);
            if (e != cudaSuccess) return e;
            levels_done = true;
        }
    }
    for (int l = 0; !levels_done && l < cf.top_lev; ++l) {
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            if (ns == 0) continue;
            const int32_t cap = cf.lev_stage[l];
            const int32_t tsz = nrhs >= 8 ? kSmallN * tile_rp<T>() : kSmallRBf * kSmallN;
            const size_t sm = ((size_t)tsz + cap) * sizeof(T);
            if (sm > 48 * 1024 && !raise_smem_once((const void*)k_cfwd_small<T>)) return cudaErrorInvalidValue;
            k_cfwd_small<T><<<ns, kThreads, sm, st>>>(v, s0, g_dd, ldg, xf, nrhs, cap, tsz);
            counted();
            continue;
        }
        const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
        const int p0 = cf.lev_ptask_ptr[l], np = cf.lev_ptask_ptr[l + 1] - p0;
        if (nt + np == 0) continue;
        // t_J of the level's supernodes, once (every task of a supernode reads it)
        CView<T> vl = v;
        if (cf.tws && cf.lev_maxn[l] > 0) {
            vl.tws = cf.tws;                  // the gather writes it, the level's tasks read it
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            const unsigned chunks = (unsigned)(((int64_t)cf.lev_maxn[l] * nrhs + 255) / 256);
            k_cfwd_gather<T><<<dim3(ns, chunks), 256, 0, st>>>(vl, s0, g_dd, ldg, nrhs);
            counted();
        }
        const bool wide = nt + np <= cf.nsm;
        // blocks of 8 or more with the level's gather: one pass per 32 (16 in the wide
        // variant, 8 when the level's widest supernode leaves no room for 16) right-hand
        // sides when t_J of that many fits; every variant forms the same sums in the same order
        if (nrhs >= 8 && vl.tws) {
            const int32_t ts_n = cf.lev_maxn[l] > 0 ? cf.lev_maxn[l] : cf.max_n;
            auto smem_for = [&](int rp, int nw) { return ((size_t)ts_n * (rp + 4) + (size_t)nw * rp * 32) * sizeof(T); };
            auto fits = [&](size_t sm, const void* kb) {
                return sm <= kLevSmem && (sm <= 48 * 1024 || raise_smem_once(kb));
            };
            if (!wide) {
                const size_t sm = smem_for(32, 8);
                if (fits(sm, (const void*)k_cfwd_level_blk<T, 8, 32>)) {
                    k_cfwd_level_blk<T, 8, 32><<<nt + np, 256, sm, st>>>(vl, t0, p0, np, xf, nrhs, ts_n);
                    counted();
                    continue;
                }
            } else {
                size_t sm = smem_for(16, 32);
                if (fits(sm, (const void*)k_cfwd_level_blk<T, 32, 16>)) {
                    k_cfwd_level_blk<T, 32, 16><<<nt + np, 1024, sm, st>>>(vl, t0, p0, np, xf, nrhs, ts_n);
                    counted();
                    continue;
                }
                sm = smem_for(8, 32);
                if (fits(sm, (const void*)k_cfwd_level_blk<T, 32, 8>)) {
                    k_cfwd_level_blk<T, 32, 8><<<nt + np, 1024, sm, st>>>(vl, t0, p0, np, xf, nrhs, ts_n);
                    counted();
                    continue;
                }
            }
        }
        // blocks of eight or four right-hand sides share each matrix load when t_J of that many fits
        const void* kern = wide ? (const void*)k_cfwd_level<T, 32> : (const void*)k_cfwd_level<T, 8>;
        // t_J of rbmax columns, then (blocks) the diagonal tasks' partial sums, NW x rbmax x 32
        auto need = [&](int32_t rb) {
            return ((size_t)rb * cf.max_n + (rb > 1 ? (size_t)(wide ? 32 : 8) * rb * 32 : 0)) * sizeof(T);
        };
        int32_t rbmax = 1;
        if (nrhs >= 8 && need(8) <= kLevSmem) rbmax = 8;
        else if (nrhs >= 4 && need(4) <= kLevSmem) rbmax = 4;
        if (rbmax > 1 && need(rbmax) > 40 * 1024 && !raise_smem_once(kern)) rbmax = 1;
        const size_t smem = need(rbmax);
        if (smem > 48 * 1024 && !raise_smem_once(kern)) return cudaErrorInvalidValue;
        if (!wide)
            k_cfwd_level<T, 8><<<nt + np, 256, smem, st>>>(vl, t0, p0, np, g_dd, ldg, xf, nrhs, cf.max_n, rbmax);
        else
            k_cfwd_level<T, 32><<<nt + np, 1024, smem, st>>>(vl, t0, p0, np, g_dd, ldg, xf, nrhs, cf.max_n, rbmax);
        counted();
    }
    if (cf.nT > 0) {
        k_ctop_gather<T><<<blocks_for((int64_t)cf.nT * nrhs), kThreads, 0, st>>>(v, g_dd, ldg, nrhs);
        k_ctop_fwd<T><<<cf.n_tf_tasks, kTopT, 0, st>>>(v, xf, nrhs);
        counted(2);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_c_backward(const DevCFactor<T>& cf, const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs,
                              cudaStream_t st) {
    if (cf.nT > 0 && nrhs > cf.ws_cols) return cudaErrorInvalidValue;
    CView<T> v = make_view(cf, cf.nsteps_bwd);
    v.xr = nrhs;     // the solution x (scratch): a call's right-hand sides contiguous per row
    if (cf.nT > 0) {
        k_ctop_bwd<T><<<cf.n_tb_tasks, kTopT, 0, st>>>(v, yf, xf, y_dd, ldy, nrhs);
        counted();
    }
    if (cf.nsteps_bwd == 0) return cudaGetLastError();
    if (!cf.per_level) {
        const size_t smem = pers_smem_bytes(cf.max_n, sizeof(T), cf.stage_cap);
        const int grid = pers_grid(k_cbwd_persistent<T>, smem, cf.max_cta_tasks);
        if (grid > 0)
            return launch_persistent(k_cbwd_persistent<T>, grid, smem, cf.bar, st, v, yf, xf, y_dd, ldy, nrhs);
    }
    for (int l = cf.top_lev - 1; l >= 0; --l) {
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            if (ns == 0) continue;
            const int32_t cap = cf.lev_stage[l];
            const bool tiled = nrhs >= 8;
            const size_t sm = ((size_t)small_bwd_vsz<T>(tiled) + cap) * sizeof(T);
            if (sm > 48 * 1024 && !raise_smem_once((const void*)k_cbwd_small<T>)) return cudaErrorInvalidValue;
            k_cbwd_small<T><<<ns, kThreads, sm, st>>>(v, s0, yf, xf, y_dd, ldy, nrhs, cap, tiled);
            counted();
            continue;
        }
        const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
        if (nt == 0) continue;
        if (nrhs >= 8) {                               // blocks of 8 or more: one pass per 32 (16 wide)
            const bool wide = nt <= cf.nsm;
            if (!wide) {
                const size_t sm = ((size_t)32 * 32 + (size_t)8 * 32 * 36) * sizeof(T);
                if (sm <= 48 * 1024 || raise_smem_once((const void*)k_cbwd_level_blk<T, 8, 32>)) {
                    k_cbwd_level_blk<T, 8, 32><<<nt, 256, sm, st>>>(v, t0, yf, xf, y_dd, ldy, nrhs);
                    counted();
                    continue;
                }
            } else {
                const size_t sm = ((size_t)16 * 32 + (size_t)32 * 32 * 20) * sizeof(T);
                if (sm <= 48 * 1024 || raise_smem_once((const void*)k_cbwd_level_blk<T, 32, 16>)) {
                    k_cbwd_level_blk<T, 32, 16><<<nt, 1024, sm, st>>>(v, t0, yf, xf, y_dd, ldy, nrhs);
                    counted();
                    continue;
                }
            }
        }
        // blocks of four or more: the panel part's partial sums, NW x 8 x 32
        if (nt > cf.nsm) {
            const size_t sm = nrhs >= 4 ? (size_t)8 * 8 * 32 * sizeof(T) : 0;
            k_cbwd_level<T, 8><<<nt, 256, sm, st>>>(v, t0, yf, xf, y_dd, ldy, nrhs);
        } else {
            const size_t sm = nrhs >= 4 ? (size_t)32 * 8 * 32 * sizeof(T) : 0;
            if (sm > 48 * 1024 && !raise_smem_once((const void*)k_cbwd_level<T, 32>)) return cudaErrorInvalidValue;
            k_cbwd_level<T, 32><<<nt, 1024, sm, st>>>(v, t0, yf, xf, y_dd, ldy, nrhs);
        }
        counted();
    }
    return cudaGetLastError();
}

// the two passes of K4 on any s x k column-major basis Ub (U_k in the U-form, Z_k in
// the Z-form of Proposition 4.3) and a block w of leading dimension ldw:
//   lowrank_v:      op.vk = d o (Ub^T w)
//   lowrank_update: w = cinv w + Ub op.vk
template <typename T>
cudaError_t launch_lowrank_v(const DevOperator<T>& op, int32_t s, int32_t k, const T* Ub, const T* w, int64_t ldw,
                             int32_t nrhs, cudaStream_t st) {
    if (s == 0 || k == 0) return cudaSuccess;
    const int G = lr_blocks(s);
    k_lr_vt<T><<<G, 256, 0, st>>>(s, k, nrhs, Ub, w, ldw, op.part);
    k_lr_vt_fin<T><<<dim3(k, (nrhs + kLrFinJ - 1) / kLrFinJ), kLrSeg * kLrFinJ, 0, st>>>(k, nrhs, G, op.part, op.dvec,
                                                                                        op.vk);
    counted(2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lowrank_update(const DevOperator<T>& op, int32_t s, int32_t k, const T* Ub, T* w, int64_t ldw,
                                  int32_t nrhs, cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    const dim3 grid((unsigned)((s + 255) / 256));
    // every column sees the same multiply-adds in the same order whatever JG is
    if (nrhs == 1) {
        k_lr_update<T, 1><<<grid, 256, 0, st>>>(s, k, nrhs, Ub, op.vk, op.cinv, w, ldw);
    } else if (nrhs <= 8) {
        k_lr_update<T, 8><<<grid, 256, 0, st>>>(s, k, nrhs, Ub, op.vk, op.cinv, w, ldw);
    } else {
        k_lr_update<T, 32><<<dim3(grid.x, (nrhs + 31) / 32), 256, 0, st>>>(s, k, nrhs, Ub, op.vk, op.cinv, w, ldw);
    }
    counted();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lowrank(const DevOperator<T>& op, int32_t s, int32_t k, T* w, int32_t nrhs, cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        if (lowrank_tc_usable(op, k, nrhs)) return launch_lowrank_tc(op, s, k, w, nrhs, st);
    }
    cudaError_t e = launch_lowrank_v<T>(op, s, k, op.U, w, s, nrhs, st);
    if (e != cudaSuccess) return e;
    return launch_lowrank_update<T>(op, s, k, op.U, w, s, nrhs, st);
}

// elements of the first pass's partial sums for rank k and nrhs columns
int64_t lowrank_part_elems(int32_t s, int32_t k, int32_t nrhs) { return (int64_t)lr_blocks(s) * k * nrhs; }

template <typename TS, typename TD>
cudaError_t launch_convert(int64_t rows, int32_t cols, const TS* src, int64_t lds, TD* dst, int64_t ldd,
                           cudaStream_t st) {
    if (rows * cols == 0) return cudaSuccess;
    k_convert<TS, TD><<<blocks_for(rows * cols), kThreads, 0, st>>>(rows, cols, src, lds, dst, ldd);
    counted();
    return cudaGetLastError();
}

cudaError_t launch_permute(int32_t n, int32_t nrhs, const int32_t* idx, const double* src, int64_t lds,
                           double* dst, int64_t ldd, bool gather, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_permute<<<blocks_for((int64_t)n * nrhs), kThreads, 0, st>>>(n, nrhs, idx, src, lds, dst, ldd, gather);
    counted();
    return cudaGetLastError();
}

cudaError_t launch_csr_spmv(int32_t n, const int32_t* rp, const int32_t* ci, const double* v, const double* x,
                            int64_t ldx, double* y, int64_t ldy, int32_t nrhs, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    return spmv_cols<double>(n, nrhs, rp, ci, v, x, ldx, nullptr, 0, y, ldy, st);
}

cudaError_t launch_dots(int64_t n, int32_t cols, const double* a, int64_t lda, const double* b, int64_t ldb,
                        double* part, double* out, int32_t out_stride, cudaStream_t st) {
    if (cols == 0) return cudaSuccess;
    k_dot_partial<<<dim3(kRedBlocks, cols), kThreads, 0, st>>>(n, a, lda, b, ldb, part);
    counted();
    k_dot_final<<<blocks_for((int64_t)cols * 32), kThreads, 0, st>>>(cols, kRedBlocks, part, out, out_stride);
    counted();
    return cudaGetLastError();
}

cudaError_t launch_gemv_t(int32_t s, int32_t j, const double* V, const double* w, double* part, double* h,
                          cudaStream_t st) {
    return launch_dots(s, j, V, s, w, 0, part, h, 1, st);
}

cudaError_t launch_gemv_n_sub(int32_t s, int32_t j, const double* V, const double* h, double* w, cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    k_gemv_n_sub<<<blocks_for(s), kThreads, 0, st>>>(s, j, V, h, w);
    counted();
    return cudaGetLastError();
}

cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_axpby<<<blocks_for(n), kThreads, 0, st>>>(n, a, x, b, y);
    counted();
    return cudaGetLastError();
}

cudaError_t launch_gemm_nn(int32_t s, int32_t m, int32_t k, const double* V, const double* Y, double* U,
                           cudaStream_t st) {
    if ((int64_t)s * k == 0) return cudaSuccess;
    k_gemm_nn<<<blocks_for((int64_t)s * k), kThreads, 0, st>>>(s, m, k, V, Y, U);
    counted();
    return cudaGetLastError();
}

cudaError_t launch_pcg_alpha(int32_t nrhs, double* scal, int32_t* flags, cudaStream_t st) {
    k_pcg_alpha<<<1, 64, 0, st>>>(nrhs, scal, flags);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_pcg_update_xr(int32_t n, int32_t nrhs, double* x, double* r, const double* p, const double* q,
                                 const double* scal, const int32_t* flags, cudaStream_t st) {
    k_pcg_update_xr<<<blocks_for((int64_t)n * nrhs), kThreads, 0, st>>>(n, nrhs, x, r, p, q, scal, flags);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_pcg_check(int32_t nrhs, double* scal, int32_t* flags, int32_t it, double tol, cudaStream_t st) {
    k_pcg_check<<<1, 32, 0, st>>>(nrhs, scal, flags, it, tol);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_cg_slot_init(int32_t j, double tol, int32_t maxit, double* scal, int32_t* flags, double* ctl,
                               cudaStream_t st) {
    k_cg_slot_init<<<1, 32, 0, st>>>(j, tol, maxit, scal, flags, ctl);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_cg_slot_check(int32_t width, int32_t count_at, const double* scal, int32_t* flags,
                                 const double* ctl, cudaStream_t st) {
    k_cg_slot_check<<<1, 32, 0, st>>>(width, count_at, scal, flags, ctl);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_pcg_init(int32_t nrhs, const double* scal, int32_t* flags, cudaStream_t st) {
    k_pcg_init<<<1, 32, 0, st>>>(nrhs, scal, flags);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_pcg_check_graph(int32_t nrhs, const double* scal, int32_t* flags, const double* ctl,
                                   cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hi, cudaStream_t st) {
    k_pcg_check_graph<<<1, 32, 0, st>>>(nrhs, scal, flags, ctl, hw, hi);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_pcg_beta(int32_t nrhs, double* scal, int32_t* flags, int32_t flexible, cudaStream_t st) {
    k_pcg_beta<<<1, 64, 0, st>>>(nrhs, scal, flags, flexible);
    counted();
    return cudaGetLastError();
}
cudaError_t launch_pcg_update_p(int32_t n, int32_t nrhs, double* p, const double* z, const double* scal,
                                const int32_t* flags, cudaStream_t st) {
    k_pcg_update_p<<<blocks_for((int64_t)n * nrhs), kThreads, 0, st>>>(n, nrhs, p, z, scal, flags);
    counted();
    return cudaGetLastError();
}

// explicit instantiations for the two precisions of the apply
#define SLR_INST(T)                                                                                             \
    template cudaError_t launch_gather_et<T>(const DevOperator<T>&, int32_t, const T*, int64_t, const T*,       \
                                             int64_t, T*, int64_t, int32_t, cudaStream_t);                      \
    template cudaError_t launch_spmv_e<T>(const DevOperator<T>&, int32_t, const T*, int64_t, T*, int64_t,       \
                                          int32_t, cudaStream_t);                                               \
    template cudaError_t launch_c_forward<T>(const DevCFactor<T>&, const T*, int64_t, T*, int32_t, cudaStream_t); \
    template cudaError_t launch_c_backward<T>(const DevCFactor<T>&, const T*, T*, T*, int64_t, int32_t,           \
                                              cudaStream_t);                                                    \
    template cudaError_t launch_lowrank<T>(const DevOperator<T>&, int32_t, int32_t, T*, int32_t, cudaStream_t);
SLR_INST(double)
SLR_INST(float)
#undef SLR_INST
template cudaError_t launch_lowrank_v<double>(const DevOperator<double>&, int32_t, int32_t, const double*,
                                              const double*, int64_t, int32_t, cudaStream_t);
template cudaError_t launch_lowrank_v<float>(const DevOperator<float>&, int32_t, int32_t, const float*, const float*,
                                             int64_t, int32_t, cudaStream_t);
template cudaError_t launch_lowrank_update<double>(const DevOperator<double>&, int32_t, int32_t, const double*,
                                                   double*, int64_t, int32_t, cudaStream_t);
template cudaError_t launch_lowrank_update<float>(const DevOperator<float>&, int32_t, int32_t, const float*, float*,
                                                  int64_t, int32_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(int64_t, int32_t, const double*, int64_t, float*, int64_t,
                                                   cudaStream_t);
template cudaError_t launch_convert<float, double>(int64_t, int32_t, const float*, int64_t, double*, int64_t,
                                                   cudaStream_t);
template cudaError_t launch_convert<double, double>(int64_t, int32_t, const double*, int64_t, double*, int64_t,
                                                    cudaStream_t);

}  // namespace slr

extern "C" int64_t slr_kernel_launches(void) { return slr::g_kernel_launches.load(); }
