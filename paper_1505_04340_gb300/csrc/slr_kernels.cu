// Hot-path kernels of the SLR apply (Eq. 4.1 with S~^{-1} of Eq. 4.7) and of
// the setup Lanczos on H (Eq. 3.2, Section 5.1), written for sm_103a.
//
//  K1  band solve      t = B^{-1} f, p independent banded Cholesky solves
//  K2  coupling SpMVs  g' = g - E^T t,  b = E y
//  K3  C solves        L^{-1} and L^{-T} with a supernodal, level-scheduled factor
//  K4  low rank        w' = w/(1-theta) + U_k (d o U_k^T w)
//  K5  PCG             A p, dots, axpys, scalar updates (FP64)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

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

// K1 (the batched band solve) lives in slr_band.cu.

// ------------------------------------------------------------------ K2
template <typename T>
__global__ void k_gather_et(int32_t s, int32_t nrhs, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const T* __restrict__ v, const T* g, int64_t ldg,
                            const T* t, int64_t ldt, T* gp, int64_t ldgp) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)s * nrhs) return;
    const int32_t i = (int32_t)(idx % s), j = (int32_t)(idx / s);
    T acc = T(0);
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) acc += v[q] * t[ci[q] + j * ldt];
    gp[i + j * ldgp] = g ? g[i + j * ldg] - acc : acc;
}

template <typename T>
__global__ void k_spmv(int32_t rows, int32_t nrhs, const int32_t* __restrict__ rp,
                       const int32_t* __restrict__ ci, const T* __restrict__ v, const T* x, int64_t ldx,
                       T* y, int64_t ldy) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * nrhs) return;
    const int32_t i = (int32_t)(idx % rows), j = (int32_t)(idx / rows);
    T acc = T(0);
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) acc += v[q] * x[ci[q] + j * ldx];
    y[i + j * ldy] = acc;
}

// ------------------------------------------------------------------ K3
// Supernode J owns factor positions [c0[J], c0[J+1]) (n_J of them); its
// off-diagonal rows R_J carry the row-major panel L[R_J, J] (|R_J| x n_J) and
// its diagonal block is stored inverted (packed lower, column-major: column j
// starts at cs(j) = j n_J - j (j-1) / 2).  Levels go leaves -> root.
// A column task is (J, first, count <= 32); a panel task is (J, first row, count <= 32).
//
// Each step is a device function run by one warp or one CTA of NW warps; the
// per-level kernels below wrap them one launch per step, and the persistent
// kernels run every level in one cooperative launch with a grid barrier
// between dependent steps.
__device__ __forceinline__ int64_t packed_col(int j, int n) { return (int64_t)j * n - (int64_t)j * (j - 1) / 2; }

// sum of w[seg_row[e]] for e = e0 .. e1-1, in that order: indices and values are
// loaded 8 at a time so that the two dependent loads are not paid per term
template <typename T>
__device__ __forceinline__ T gather_sum(const T* w, const int32_t* __restrict__ seg_row, int64_t e0, int64_t e1) {
    T acc = T(0);
    for (int64_t e = e0; e < e1; e += 8) {
        int32_t idx[8];
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) idx[u] = e + u < e1 ? seg_row[e + u] : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = idx[u] >= 0 ? w[idx[u]] : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (e + u < e1) acc += v[u];
    }
    return acc;
}

// forward, gather (one warp): t_i = g[cperm[i]] - sum of the panel products w that hold row i
template <typename T>
__device__ __forceinline__ void cfwd_gather_warp(const int4 tk, int lane, const int32_t* __restrict__ c0,
                                                 const int32_t* __restrict__ cperm,
                                                 const int64_t* __restrict__ seg_ptr,
                                                 const int32_t* __restrict__ seg_row, const T* wbuf, int64_t nrow,
                                                 const T* g, int64_t ldg, T* tf, int32_t s, int32_t nrhs) {
    if (lane >= tk.z) return;
    const int32_t i = c0[tk.x] + tk.y + lane;
    const int64_t e0 = seg_ptr[i], e1 = seg_ptr[i + 1];
    for (int j = 0; j < nrhs; ++j) {
        const T* w = wbuf + (int64_t)j * nrow;
        tf[i + (int64_t)j * s] = g[cperm[i] + j * ldg] - gather_sum(w, seg_row, e0, e1);
    }
}

// forward, diagonal (one CTA of NW warps): x_J = L_JJ^{-1} t_J for a block of
// <= 32 rows; the warps split the reduction over columns (lane = row), 8 loads
// in flight per lane
template <typename T, int NW>
__device__ void cfwd_diag_cta(const int4 tk, T (*red)[33], const int32_t* __restrict__ c0,
                              const int64_t* __restrict__ dinv_off, const T* __restrict__ dinv, const T* tf, T* xf,
                              int32_t s, int32_t nrhs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0;
    const int il = tk.y + lane;
    const int ncol = tk.y + tk.z;                  // columns 0 .. ncol-1 reach these rows
    const int chunk = (ncol + NW - 1) / NW;
    const int jb = warp * chunk, je = min(ncol, jb + chunk);
    const T* D = dinv + dinv_off[tk.x];
    for (int j = 0; j < nrhs; ++j) {
        const T* t = tf + a0 + (int64_t)j * s;
        T acc = T(0);
        if (lane < tk.z) {
            const int jend = min(je, il + 1);
            int jj = jb;
            for (; jj + 7 < jend; jj += 8) {
                T d[8], tv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    d[u] = D[packed_col(jj + u, nJ) + (il - jj - u)];
                    tv[u] = t[jj + u];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += d[u] * tv[u];
            }
            for (; jj < jend; ++jj) acc += D[packed_col(jj, nJ) + (il - jj)] * t[jj];
        }
        red[warp][lane] = acc;
        __syncthreads();
        if (warp == 0) {
            T v = T(0);
#pragma unroll 8
            for (int w = 0; w < NW; ++w) v += red[w][lane];
            if (lane < tk.z) xf[a0 + il + (int64_t)j * s] = v;
        }
        __syncthreads();
    }
}

// forward, panel (one CTA): w[r_off[J] + p] = L[R_J[p], J] . x_J (warp per panel
// row, lanes over columns); x_J staged in shared memory xs[n_J]
template <typename T, int NW>
__device__ void cfwd_panel_cta(const int4 tk, T* xs, const int32_t* __restrict__ c0,
                               const int64_t* __restrict__ r_off, const int64_t* __restrict__ pan_off,
                               const T* __restrict__ panel, const T* xf, T* wbuf, int64_t nrow, int32_t s,
                               int32_t nrhs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0;
    for (int j = 0; j < nrhs; ++j) {
        for (int c = threadIdx.x; c < nJ; c += NW * 32) xs[c] = xf[a0 + c + (int64_t)j * s];
        __syncthreads();
        for (int pr = warp; pr < tk.z; pr += NW) {
            const int64_t p = tk.y + pr;
            const T* P = panel + pan_off[tk.x] + p * nJ;
            T acc = T(0);
            int c = lane;
            for (; c + 7 * 32 < nJ; c += 8 * 32) {
                T pv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) pv[u] = P[c + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += pv[u] * xs[c + 32 * u];
            }
            for (; c < nJ; c += 32) acc += P[c] * xs[c];
            acc = warp_sum(acc);
            if (lane == 0) wbuf[r_off[tk.x] + p + (int64_t)j * nrow] = acc;
        }
        __syncthreads();
    }
}

// backward, panel (one CTA): t_j = y_j - sum_p L[R_J[p], j] x[R_J[p]] for <= 32
// columns (lane = column); the warps split the panel rows, 8 loads in flight
template <typename T, int NW, int DEPTH = 8>
__device__ void cbwd_panel_cta(const int4 tk, T (*red)[33], const int32_t* __restrict__ c0,
                               const int64_t* __restrict__ r_off, const int32_t* __restrict__ rows,
                               const int64_t* __restrict__ pan_off, const T* __restrict__ panel, T* yf,
                               const T* xf, int32_t s, int32_t nrhs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0, jl = tk.y + lane;
    const int64_t nr = r_off[tk.x + 1] - r_off[tk.x];
    const int32_t* R = rows + r_off[tk.x];
    const T* Pn = panel + pan_off[tk.x] + jl;
    const int64_t chunk = (nr + NW - 1) / NW, pb = warp * chunk, pe = min(nr, pb + chunk);
    for (int j = 0; j < nrhs; ++j) {
        const T* x = xf + (int64_t)j * s;
        T acc = T(0);
        if (lane < tk.z) {
            int64_t p = pb;
            for (; p + DEPTH - 1 < pe; p += DEPTH) {
                T pv[DEPTH], xv[DEPTH];
#pragma unroll
                for (int u = 0; u < DEPTH; ++u) {
                    pv[u] = Pn[(p + u) * nJ];
                    xv[u] = x[R[p + u]];
                }
#pragma unroll
                for (int u = 0; u < DEPTH; ++u) acc += pv[u] * xv[u];
            }
            for (; p < pe; ++p) acc += Pn[p * nJ] * x[R[p]];
        }
        red[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && lane < tk.z) {
            T v = T(0);
#pragma unroll 8
            for (int w = 0; w < NW; ++w) v += red[w][lane];
            yf[a0 + jl + (int64_t)j * s] -= v;
        }
        __syncthreads();
    }
}

// backward, diagonal (one CTA): x_J = L_JJ^{-T} t_J (warp per column, lanes over
// the column, 8 loads in flight per lane), optional scatter to DD order
template <typename T, int NW>
__device__ void cbwd_diag_cta(const int4 tk, const int32_t* __restrict__ c0, const int64_t* __restrict__ dinv_off,
                              const T* __restrict__ dinv, const int32_t* __restrict__ cperm, const T* tf, T* xf,
                              T* y_dd, int64_t ldy, int32_t s, int32_t nrhs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0;
    const T* D = dinv + dinv_off[tk.x];
    for (int cc = warp; cc < tk.z; cc += NW) {
        const int jl = tk.y + cc;
        const T* Dc = D + packed_col(jl, nJ) - jl;
        for (int j = 0; j < nrhs; ++j) {
            const T* t = tf + a0 + (int64_t)j * s;
            T acc = T(0);
            int i = jl + lane;
            for (; i + 7 * 32 < nJ; i += 8 * 32) {
                T d[8], tv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    d[u] = Dc[i + 32 * u];
                    tv[u] = t[i + 32 * u];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += d[u] * tv[u];
            }
            for (; i < nJ; i += 32) acc += Dc[i] * t[i];
            acc = warp_sum(acc);
            if (lane == 0) {
                xf[a0 + jl + (int64_t)j * s] = acc;
                if (y_dd) y_dd[cperm[a0 + jl] + j * ldy] = acc;
            }
        }
    }
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

// Fused levels: one group of NT threads (a CTA, or a part of one) per supernode J
// with n_J <= kSmallN and |R_J| <= kSmallR.
// forward: t_J = g_J - (gathered panel products); x_J = L_JJ^{-1} t_J; w_J = L[R_J, J] x_J
template <typename T, int NT, int GROUPS>
__device__ void cfwd_small_cta(int J, T* ts, T* xs, const int32_t* __restrict__ c0,
                               const int32_t* __restrict__ cperm, const int64_t* __restrict__ seg_ptr,
                               const int32_t* __restrict__ seg_row, const int64_t* __restrict__ r_off,
                               const int64_t* __restrict__ pan_off, const T* __restrict__ panel,
                               const int64_t* __restrict__ dinv_off, const T* __restrict__ dinv, T* wbuf,
                               int64_t nrow, const T* g, int64_t ldg, T* xf, int32_t s, int32_t nrhs) {
    constexpr int nw = NT / 32;
    const int gt = threadIdx.x % NT, lane = gt & 31, warp = gt >> 5;
    const int32_t a0 = c0[J], nJ = c0[J + 1] - a0;
    const int64_t nr = r_off[J + 1] - r_off[J];
    const T* D = dinv + dinv_off[J];
    const T* Pn = panel + pan_off[J];
    for (int j = 0; j < nrhs; ++j) {
        const T* w = wbuf + (int64_t)j * nrow;
        for (int i = gt; i < nJ; i += NT) {
            const int32_t pos = a0 + i;
            ts[i] = g[cperm[pos] + j * ldg] - gather_sum(w, seg_row, seg_ptr[pos], seg_ptr[pos + 1]);
        }
        group_sync<NT, GROUPS>();
        for (int i = gt; i < nJ; i += NT) {
            T acc = T(0);
            int jj = 0;
            for (; jj + 7 <= i; jj += 8) {
                T d[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) d[u] = D[packed_col(jj + u, nJ) + (i - jj - u)];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += d[u] * ts[jj + u];
            }
            for (; jj <= i; ++jj) acc += D[packed_col(jj, nJ) + (i - jj)] * ts[jj];
            xs[i] = acc;
            xf[a0 + i + (int64_t)j * s] = acc;
        }
        group_sync<NT, GROUPS>();
        // four panel rows per warp at a time: their loads are in flight together
        for (int64_t p0 = 4 * warp; p0 < nr; p0 += 4 * nw) {
            T acc[4] = {T(0), T(0), T(0), T(0)};
            for (int c = lane; c < nJ; c += 32) {
                const T xv = xs[c];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (p0 + u < nr) acc[u] += Pn[(p0 + u) * nJ + c] * xv;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T v = warp_sum(acc[u]);
                if (lane == 0 && p0 + u < nr) wbuf[r_off[J] + p0 + u + (int64_t)j * nrow] = v;
            }
        }
        group_sync<NT, GROUPS>();
    }
}

// backward: t_J = y_J - L[R_J, J]^T x_{R_J};  x_J = L_JJ^{-T} t_J (and scatter to DD order).
// NT / kSmallN threads share each column, each over a part of the panel rows.
template <typename T, int NT, int GROUPS>
__device__ void cbwd_small_cta(int J, T* xr, T* ts, T* red, const int32_t* __restrict__ c0,
                               const int64_t* __restrict__ r_off, const int32_t* __restrict__ rows,
                               const int64_t* __restrict__ pan_off, const T* __restrict__ panel,
                               const int64_t* __restrict__ dinv_off, const T* __restrict__ dinv,
                               const int32_t* __restrict__ cperm, const T* yf, T* xf, T* y_dd, int64_t ldy,
                               int32_t s, int32_t nrhs) {
    static_assert(NT % kSmallN == 0, "whole threads per column");
    constexpr int nw = NT / 32, parts = NT / kSmallN;
    const int gt = threadIdx.x % NT, lane = gt & 31, warp = gt >> 5;
    const int32_t a0 = c0[J], nJ = c0[J + 1] - a0;
    const int64_t nr = r_off[J + 1] - r_off[J];
    const int32_t* R = rows + r_off[J];
    const T* D = dinv + dinv_off[J];
    const T* Pn = panel + pan_off[J];
    for (int j = 0; j < nrhs; ++j) {
        const T* x = xf + (int64_t)j * s;
        for (int64_t p = gt; p < nr; p += NT) xr[p] = x[R[p]];
        group_sync<NT, GROUPS>();
        {
            const int part = gt / kSmallN, c = gt % kSmallN;
            T acc = T(0);
            if (c < nJ) {
                const int64_t len = (nr + parts - 1) / parts, pb = part * len, pe = min(nr, pb + len);
                int64_t p = pb;
                for (; p + 7 < pe; p += 8) {
                    T pv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) pv[u] = Pn[(p + u) * nJ + c];
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc += pv[u] * xr[p + u];
                }
                for (; p < pe; ++p) acc += Pn[p * nJ + c] * xr[p];
            }
            red[part * kSmallN + c] = acc;
        }
        group_sync<NT, GROUPS>();
        for (int c = gt; c < nJ; c += NT) {
            T v = T(0);
#pragma unroll
            for (int q = 0; q < parts; ++q) v += red[q * kSmallN + c];
            ts[c] = yf[a0 + c + (int64_t)j * s] - v;
        }
        group_sync<NT, GROUPS>();
        for (int c = warp; c < nJ; c += nw) {
            const T* Dc = D + packed_col(c, nJ) - c;
            T acc = T(0);
            for (int i = c + lane; i < nJ; i += 32) acc += Dc[i] * ts[i];
            acc = warp_sum(acc);
            if (lane == 0) {
                xf[a0 + c + (int64_t)j * s] = acc;
                if (y_dd) y_dd[cperm[a0 + c] + j * ldy] = acc;
            }
        }
        group_sync<NT, GROUPS>();
    }
}

constexpr int kDiagT = 1024;   // threads of the per-level diagonal-block kernels (32 warps)
constexpr int kPanT = 512;     // threads of the per-level forward panel kernels (16 warps)
constexpr int kBPanT = 1024;   // threads of the per-level backward panel kernels (32 warps)

// ---- per-level kernels: one launch per step
template <typename T>
__global__ void __launch_bounds__(32)
k_cfwd_gather(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int32_t* __restrict__ cperm,
              const int64_t* __restrict__ seg_ptr, const int32_t* __restrict__ seg_row, const T* wbuf,
              int64_t nrow, const T* g, int64_t ldg, T* tf, int32_t s, int32_t nrhs) {
    cfwd_gather_warp<T>(tasks[blockIdx.x], threadIdx.x, c0, cperm, seg_ptr, seg_row, wbuf, nrow, g, ldg, tf, s, nrhs);
}

template <typename T>
__global__ void __launch_bounds__(kDiagT)
k_cfwd_diag(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ dinv_off,
            const T* __restrict__ dinv, const T* tf, T* xf, int32_t s, int32_t nrhs) {
    __shared__ T red[kDiagT / 32][33];
    cfwd_diag_cta<T, kDiagT / 32>(tasks[blockIdx.x], red, c0, dinv_off, dinv, tf, xf, s, nrhs);
}

template <typename T>
__global__ void __launch_bounds__(kPanT)
k_cfwd_panel(const int4* __restrict__ ptasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ r_off,
             const int64_t* __restrict__ pan_off, const T* __restrict__ panel, const T* xf, T* wbuf, int64_t nrow,
             int32_t s, int32_t nrhs) {
    extern __shared__ unsigned char csm[];
    cfwd_panel_cta<T, kPanT / 32>(ptasks[blockIdx.x], reinterpret_cast<T*>(csm), c0, r_off, pan_off, panel, xf,
                                  wbuf, nrow, s, nrhs);
}

// one CTA of 32 warps per 32-column task, 16 (FP32) or 8 (FP64) panel loads in flight per lane
template <typename T>
__global__ void __launch_bounds__(kBPanT)
k_cbwd_panel(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ r_off,
             const int32_t* __restrict__ rows, const int64_t* __restrict__ pan_off, const T* __restrict__ panel,
             T* yf, const T* xf, int32_t s, int32_t nrhs) {
    __shared__ T red[kBPanT / 32][33];
    cbwd_panel_cta<T, kBPanT / 32, sizeof(T) == 4 ? 16 : 8>(tasks[blockIdx.x], red, c0, r_off, rows, pan_off, panel,
                                                            yf, xf, s, nrhs);
}

template <typename T>
__global__ void __launch_bounds__(kDiagT)
k_cbwd_diag(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ dinv_off,
            const T* __restrict__ dinv, const int32_t* __restrict__ cperm, const T* tf, T* xf, T* y_dd,
            int64_t ldy, int32_t s, int32_t nrhs) {
    cbwd_diag_cta<T, kDiagT / 32>(tasks[blockIdx.x], c0, dinv_off, dinv, cperm, tf, xf, y_dd, ldy, s, nrhs);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cfwd_small(const int32_t* __restrict__ sns, const int32_t* __restrict__ c0, const int32_t* __restrict__ cperm,
             const int64_t* __restrict__ seg_ptr, const int32_t* __restrict__ seg_row, const int64_t* __restrict__ r_off,
             const int64_t* __restrict__ pan_off, const T* __restrict__ panel, const int64_t* __restrict__ dinv_off,
             const T* __restrict__ dinv, T* wbuf, int64_t nrow, const T* g, int64_t ldg, T* xf, int32_t s,
             int32_t nrhs) {
    __shared__ T ts[kSmallN], xs[kSmallN];
    cfwd_small_cta<T, kThreads, 1>(sns[blockIdx.x], ts, xs, c0, cperm, seg_ptr, seg_row, r_off, pan_off, panel,
                                dinv_off, dinv, wbuf, nrow, g, ldg, xf, s, nrhs);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cbwd_small(const int32_t* __restrict__ sns, const int32_t* __restrict__ c0, const int64_t* __restrict__ r_off,
             const int32_t* __restrict__ rows, const int64_t* __restrict__ pan_off, const T* __restrict__ panel,
             const int64_t* __restrict__ dinv_off, const T* __restrict__ dinv, const int32_t* __restrict__ cperm,
             const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t s, int32_t nrhs) {
    __shared__ T xr[kSmallR], ts[kSmallN];
    __shared__ T red[(kThreads / kSmallN) * kSmallN];
    cbwd_small_cta<T, kThreads, 1>(sns[blockIdx.x], xr, ts, red, c0, r_off, rows, pan_off, panel, dinv_off, dinv, cperm,
                                yf, xf, y_dd, ldy, s, nrhs);
}

// ---- persistent kernels: every level in one cooperative launch
// Plain view of a DevCFactor (device pointers and sizes) passed by value.
template <typename T>
struct CView {
    int32_t s, nlev, nsteps;
    int64_t nrow;
    const int32_t *cperm, *c0, *rows, *seg_row, *lev_sn;
    const int64_t *r_off, *pan_off, *dinv_off, *seg_ptr;
    const T *panel, *dinv;
    T* wbuf;
    const int4 *tasks, *ptasks;
    const int32_t *lev_task_ptr, *lev_ptask_ptr, *lev_sn_ptr;
    const uint8_t* lev_small;
    unsigned* bar;
    int32_t* err;
};

constexpr int kPersT = 1024;                  // 32 warps, one CTA per SM
constexpr int kPersW = kPersT / 32;
constexpr int kSmallT = 256;                  // fused levels: 4 groups of 256 threads, a supernode each
constexpr int kSmallG = kPersT / kSmallT;
constexpr long long kGridSpin = 1ll << 22;    // bounded barrier wait (x 64 ns sleep: about a quarter second)

// All CTAs arrive; the counter (zeroed before the launch) reaches target =
// round x gridDim.x.  A wait that runs out sets the status word and goes on;
// once the status word is set, later waits give up early too.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned target, int32_t* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        long long it = 0;
        while (*reinterpret_cast<volatile unsigned*>(bar) < target) {
            if (++it > kGridSpin) {
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

// shared bytes of the persistent kernels: the larger of the forward panel's
// x_J (max_n values), the fused levels' buffers and the reduction arrays
inline size_t pers_smem_bytes(int32_t max_n, size_t elem) {
    const size_t small_fwd = kSmallG * 2 * kSmallN,
                 small_bwd = kSmallG * (kSmallR + kSmallN + (kSmallT / kSmallN) * kSmallN);
    const size_t red = kPersW * 33;
    return std::max({(size_t)max_n, small_fwd, small_bwd, red}) * elem;
}

template <typename T>
__global__ void __launch_bounds__(kPersT, 1)
k_cfwd_persistent(const CView<T> cf, const T* g, int64_t ldg, T* tf, T* xf, int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char psm[];
    T* sm = reinterpret_cast<T*>(psm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned round = 0;
    int steps_left = cf.nsteps;
    auto sync = [&]() {
        if (--steps_left > 0) grid_barrier(cf.bar, ++round * gridDim.x, cf.err);
    };
    for (int l = 0; l < cf.nlev; ++l) {
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            if (ns == 0) continue;
            const int grp = threadIdx.x / kSmallT;
            T* gs = sm + grp * 2 * kSmallN;
            for (int q = blockIdx.x * kSmallG + grp; q < ns; q += gridDim.x * kSmallG)
                cfwd_small_cta<T, kSmallT, kSmallG>(cf.lev_sn[s0 + q], gs, gs + kSmallN, cf.c0, cf.cperm, cf.seg_ptr,
                                          cf.seg_row, cf.r_off, cf.pan_off, cf.panel, cf.dinv_off, cf.dinv, cf.wbuf,
                                          cf.nrow, g, ldg, xf, cf.s, nrhs);
            sync();
            continue;
        }
        const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
        const int p0 = cf.lev_ptask_ptr[l], np = cf.lev_ptask_ptr[l + 1] - p0;
        if (nt > 0) {
            for (int q = blockIdx.x * kPersW + warp; q < nt; q += gridDim.x * kPersW)
                cfwd_gather_warp<T>(cf.tasks[t0 + q], lane, cf.c0, cf.cperm, cf.seg_ptr, cf.seg_row, cf.wbuf,
                                    cf.nrow, g, ldg, tf, cf.s, nrhs);
            sync();
            for (int q = blockIdx.x; q < nt; q += gridDim.x)
                cfwd_diag_cta<T, kPersW>(cf.tasks[t0 + q], reinterpret_cast<T(*)[33]>(sm), cf.c0, cf.dinv_off,
                                         cf.dinv, tf, xf, cf.s, nrhs);
            sync();
        }
        if (np > 0) {
            for (int q = blockIdx.x; q < np; q += gridDim.x)
                cfwd_panel_cta<T, kPersW>(cf.ptasks[p0 + q], sm, cf.c0, cf.r_off, cf.pan_off, cf.panel, xf, cf.wbuf,
                                          cf.nrow, cf.s, nrhs);
            sync();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kPersT, 1)
k_cbwd_persistent(const CView<T> cf, T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char psm[];
    T* sm = reinterpret_cast<T*>(psm);
    unsigned round = 0;
    int steps_left = cf.nsteps;
    auto sync = [&]() {
        if (--steps_left > 0) grid_barrier(cf.bar, ++round * gridDim.x, cf.err);
    };
    for (int l = cf.nlev - 1; l >= 0; --l) {
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            if (ns == 0) continue;
            const int grp = threadIdx.x / kSmallT;
            T* gs = sm + grp * (kSmallR + kSmallN + (kSmallT / kSmallN) * kSmallN);
            for (int q = blockIdx.x * kSmallG + grp; q < ns; q += gridDim.x * kSmallG)
                cbwd_small_cta<T, kSmallT, kSmallG>(cf.lev_sn[s0 + q], gs, gs + kSmallR, gs + kSmallR + kSmallN, cf.c0,
                                          cf.r_off, cf.rows, cf.pan_off, cf.panel, cf.dinv_off, cf.dinv, cf.cperm,
                                          yf, xf, y_dd, ldy, cf.s, nrhs);
            sync();
            continue;
        }
        const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
        if (nt == 0) continue;
        for (int q = blockIdx.x; q < nt; q += gridDim.x)
            cbwd_panel_cta<T, kPersW>(cf.tasks[t0 + q], reinterpret_cast<T(*)[33]>(sm), cf.c0, cf.r_off, cf.rows,
                                      cf.pan_off, cf.panel, yf, xf, cf.s, nrhs);
        sync();
        for (int q = blockIdx.x; q < nt; q += gridDim.x)
            cbwd_diag_cta<T, kPersW>(cf.tasks[t0 + q], cf.c0, cf.dinv_off, cf.dinv, cf.cperm, yf, xf, y_dd, ldy,
                                     cf.s, nrhs);
        sync();
    }
}

// ------------------------------------------------------------------ K4
// part[(j k + kk) G + b] = partial of U[:, kk] . w[:, j] over block b's rows
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_ut_partial(int32_t s, int32_t k, const T* __restrict__ U, const T* __restrict__ w, T* part) {
    __shared__ T red[kThreads / 32];
    const int kk = blockIdx.y, j = blockIdx.z;
    const T* u = U + (int64_t)kk * s;
    const T* x = w + (int64_t)j * s;
    T acc = T(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (int64_t)gridDim.x * blockDim.x)
        acc += u[i] * x[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        T v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
        v = warp_sum(v);
        if (threadIdx.x == 0) part[((int64_t)j * k + kk) * gridDim.x + blockIdx.x] = v;
    }
}

// vk[kk + j k] = d[kk] * sum_b part[...]   (one warp per (kk, j))
template <typename T>
__global__ void k_ut_final(int32_t k, int32_t nrhs, int32_t G, const T* part, const T* __restrict__ dvec,
                           T* vk) {
    const int id = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (id >= k * nrhs) return;
    const T* pp = part + (int64_t)id * G;
    T acc = T(0);
    for (int b = lane; b < G; b += 32) acc += pp[b];
    acc = warp_sum(acc);
    if (lane == 0) vk[id] = dvec[id % k] * acc;
}

template <typename T>
__global__ void k_lowrank_update(int32_t s, int32_t k, int32_t nrhs, const T* __restrict__ U, const T* vk,
                                 T cinv, T* w) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)s * nrhs) return;
    const int32_t i = (int32_t)(idx % s), j = (int32_t)(idx / s);
    const T* v = vk + (int64_t)j * k;
    T acc = cinv * w[i + (int64_t)j * s];
    for (int kk = 0; kk < k; ++kk) acc += U[i + (int64_t)kk * s] * v[kk];
    w[i + (int64_t)j * s] = acc;
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

inline unsigned blocks_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// every kernel launch of the library goes through this counter
inline void counted(int n = 1) { count_launches(n); }

}  // namespace

// ------------------------------------------------------------------ launchers

template <typename T>
cudaError_t launch_gather_et(const DevOperator<T>& op, int32_t s, const T* g, int64_t ldg, const T* t,
                             int64_t ldt, T* gp, int64_t ldgp, int32_t nrhs, cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    k_gather_et<T><<<blocks_for((int64_t)s * nrhs), kThreads, 0, st>>>(s, nrhs, op.et_rp, op.et_ci, op.et_v, g,
                                                                        ldg, t, ldt, gp, ldgp);
    counted();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmv_e(const DevOperator<T>& op, int32_t nI, const T* y, int64_t ldy, T* out, int64_t ldo,
                          int32_t nrhs, cudaStream_t st) {
    if (nI == 0) return cudaSuccess;
    k_spmv<T><<<blocks_for((int64_t)nI * nrhs), kThreads, 0, st>>>(nI, nrhs, op.e_rp, op.e_ci, op.e_v, y, ldy,
                                                                    out, ldo);
    counted();
    return cudaGetLastError();
}

// Grid of a persistent solve on the current device: one CTA per SM (fewer if
// no step has that many CTA tasks), 0 if the kernel cannot be co-resident.
template <typename K>
int pers_grid(K kern, size_t smem, int32_t max_cta_tasks) {
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
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
    v.nlev = cf.nlev;
    v.nsteps = nsteps;
    v.nrow = cf.nrow;
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
    v.tasks = cf.tasks;
    v.ptasks = cf.ptasks;
    v.lev_task_ptr = cf.d_lev_task_ptr;
    v.lev_ptask_ptr = cf.d_lev_ptask_ptr;
    v.lev_sn_ptr = cf.d_lev_sn_ptr;
    v.lev_small = cf.d_lev_small;
    v.bar = cf.bar;
    v.err = cf.err;
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
cudaError_t launch_c_forward(const DevCFactor<T>& cf, const T* g_dd, int64_t ldg, T* tf, T* xf, int32_t nrhs,
                             cudaStream_t st) {
    if (cf.nsteps_fwd == 0) return cudaSuccess;
    if (!cf.per_level) {
        const size_t smem = pers_smem_bytes(cf.max_n, sizeof(T));
        const int grid = pers_grid(k_cfwd_persistent<T>, smem, cf.max_cta_tasks);
        if (grid > 0)
            return launch_persistent(k_cfwd_persistent<T>, grid, smem, cf.bar, st, make_view(cf, cf.nsteps_fwd), g_dd,
                                     ldg, tf, xf, nrhs);
    }
    for (int l = 0; l < cf.nlev; ++l) {
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            if (ns == 0) continue;
            k_cfwd_small<T><<<ns, kThreads, 0, st>>>(cf.lev_sn + s0, cf.c0, cf.cperm, cf.seg_ptr, cf.seg_row, cf.r_off,
                                                     cf.pan_off, cf.panel, cf.dinv_off, cf.dinv, cf.wbuf, cf.nrow,
                                                     g_dd, ldg, xf, cf.s, nrhs);
            counted();
            continue;
        }
        const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
        const int p0 = cf.lev_ptask_ptr[l], np = cf.lev_ptask_ptr[l + 1] - p0;
        if (nt > 0) {
            k_cfwd_gather<T><<<nt, 32, 0, st>>>(cf.tasks + t0, cf.c0, cf.cperm, cf.seg_ptr, cf.seg_row, cf.wbuf,
                                                cf.nrow, g_dd, ldg, tf, cf.s, nrhs);
            counted();
            k_cfwd_diag<T><<<nt, kDiagT, 0, st>>>(cf.tasks + t0, cf.c0, cf.dinv_off, cf.dinv, tf, xf, cf.s, nrhs);
            counted();
        }
        if (np > 0) {
            k_cfwd_panel<T><<<np, kPanT, cf.max_n * sizeof(T), st>>>(cf.ptasks + p0, cf.c0, cf.r_off, cf.pan_off,
                                                                      cf.panel, xf, cf.wbuf, cf.nrow, cf.s, nrhs);
            counted();
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_c_backward(const DevCFactor<T>& cf, T* yf, T* xf, T* y_dd, int64_t ldy, int32_t nrhs,
                              cudaStream_t st) {
    if (cf.nsteps_bwd == 0) return cudaSuccess;
    if (!cf.per_level) {
        const size_t smem = pers_smem_bytes(cf.max_n, sizeof(T));
        const int grid = pers_grid(k_cbwd_persistent<T>, smem, cf.max_cta_tasks);
        if (grid > 0)
            return launch_persistent(k_cbwd_persistent<T>, grid, smem, cf.bar, st, make_view(cf, cf.nsteps_bwd), yf, xf,
                                     y_dd, ldy, nrhs);
    }
    for (int l = cf.nlev - 1; l >= 0; --l) {
        if (cf.lev_small[l]) {
            const int s0 = cf.lev_sn_ptr[l], ns = cf.lev_sn_ptr[l + 1] - s0;
            if (ns == 0) continue;
            k_cbwd_small<T><<<ns, kThreads, 0, st>>>(cf.lev_sn + s0, cf.c0, cf.r_off, cf.rows, cf.pan_off, cf.panel,
                                                     cf.dinv_off, cf.dinv, cf.cperm, yf, xf, y_dd, ldy, cf.s, nrhs);
            counted();
            continue;
        }
        const int t0 = cf.lev_task_ptr[l], nt = cf.lev_task_ptr[l + 1] - t0;
        if (nt == 0) continue;
        k_cbwd_panel<T><<<nt, kBPanT, 0, st>>>(cf.tasks + t0, cf.c0, cf.r_off, cf.rows, cf.pan_off, cf.panel,
                                              yf, xf, cf.s, nrhs);
        counted();
        k_cbwd_diag<T><<<nt, kDiagT, 0, st>>>(cf.tasks + t0, cf.c0, cf.dinv_off, cf.dinv, cf.cperm, yf, xf,
                                              y_dd, ldy, cf.s, nrhs);
        counted();
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lowrank(const DevOperator<T>& op, int32_t s, int32_t k, T* w, int32_t nrhs, cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    if (k > 0) {
        const int G = kRedBlocks;
        k_ut_partial<T><<<dim3(G, k, nrhs), kThreads, 0, st>>>(s, k, op.U, w, op.part);
        counted();
        k_ut_final<T><<<blocks_for((int64_t)k * nrhs * 32), kThreads, 0, st>>>(k, nrhs, G, op.part, op.dvec, op.vk);
        counted();
    }
    k_lowrank_update<T><<<blocks_for((int64_t)s * nrhs), kThreads, 0, st>>>(s, k, nrhs, op.U, op.vk, op.cinv, w);
    counted();
    return cudaGetLastError();
}

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
    k_spmv<double><<<blocks_for((int64_t)n * nrhs), kThreads, 0, st>>>(n, nrhs, rp, ci, v, x, ldx, y, ldy);
    counted();
    return cudaGetLastError();
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
    template cudaError_t launch_c_forward<T>(const DevCFactor<T>&, const T*, int64_t, T*, T*, int32_t,          \
                                             cudaStream_t);                                                     \
    template cudaError_t launch_c_backward<T>(const DevCFactor<T>&, T*, T*, T*, int64_t, int32_t, cudaStream_t); \
    template cudaError_t launch_lowrank<T>(const DevOperator<T>&, int32_t, int32_t, T*, int32_t, cudaStream_t);
SLR_INST(double)
SLR_INST(float)
#undef SLR_INST
template cudaError_t launch_convert<double, float>(int64_t, int32_t, const double*, int64_t, float*, int64_t,
                                                   cudaStream_t);
template cudaError_t launch_convert<float, double>(int64_t, int32_t, const float*, int64_t, double*, int64_t,
                                                   cudaStream_t);
template cudaError_t launch_convert<double, double>(int64_t, int32_t, const double*, int64_t, double*, int64_t,
                                                    cudaStream_t);

}  // namespace slr

extern "C" int64_t slr_kernel_launches(void) { return slr::g_kernel_launches.load(); }
