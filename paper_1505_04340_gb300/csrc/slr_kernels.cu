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
__device__ __forceinline__ int64_t packed_col(int j, int n) { return (int64_t)j * n - (int64_t)j * (j - 1) / 2; }

// forward, phase 1: t_i = g[cperm[i]] - sum of the panel products w that hold row i
template <typename T>
__global__ void __launch_bounds__(32)
k_cfwd_gather(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int32_t* __restrict__ cperm,
              const int64_t* __restrict__ seg_ptr, const int32_t* __restrict__ seg_row, const T* wbuf,
              int64_t nrow, const T* g, int64_t ldg, T* tf, int32_t s, int32_t nrhs) {
    const int4 tk = tasks[blockIdx.x];
    if ((int)threadIdx.x >= tk.z) return;
    const int32_t i = c0[tk.x] + tk.y + threadIdx.x;
    const int64_t e0 = seg_ptr[i], e1 = seg_ptr[i + 1];
    for (int j = 0; j < nrhs; ++j) {
        const T* w = wbuf + (int64_t)j * nrow;
        T acc = T(0);
        for (int64_t e = e0; e < e1; ++e) acc += w[seg_row[e]];
        tf[i + (int64_t)j * s] = g[cperm[i] + j * ldg] - acc;
    }
}

constexpr int kDiagT = 1024;   // threads of the diagonal-block kernels (32 warps)
constexpr int kPanT = 512;     // threads of the panel kernels (16 warps)

// forward, phase 2: x_J = L_JJ^{-1} t_J for a block of <= 32 rows; 32 warps
// split the reduction over columns (lane = row), 8 loads in flight per lane
template <typename T>
__global__ void __launch_bounds__(kDiagT)
k_cfwd_diag(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ dinv_off,
            const T* __restrict__ dinv, const T* tf, T* xf, int32_t s, int32_t nrhs) {
    constexpr int nw = kDiagT / 32;
    __shared__ T red[nw][33];
    const int4 tk = tasks[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0;
    const int il = tk.y + lane;
    const int ncol = tk.y + tk.z;                  // columns 0 .. ncol-1 reach these rows
    const int chunk = (ncol + nw - 1) / nw;
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
            for (int w = 0; w < nw; ++w) v += red[w][lane];
            if (lane < tk.z) xf[a0 + il + (int64_t)j * s] = v;
        }
        __syncthreads();
    }
}

// forward, phase 3: w[r_off[J] + p] = L[R_J[p], J] . x_J (warp per panel row,
// lanes over columns); x_J staged in shared memory
template <typename T>
__global__ void __launch_bounds__(kPanT)
k_cfwd_panel(const int4* __restrict__ ptasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ r_off,
             const int64_t* __restrict__ pan_off, const T* __restrict__ panel, const T* xf, T* wbuf, int64_t nrow,
             int32_t s, int32_t nrhs) {
    extern __shared__ unsigned char csm[];
    T* xs = reinterpret_cast<T*>(csm);
    const int4 tk = ptasks[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kPanT / 32;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0;
    for (int j = 0; j < nrhs; ++j) {
        for (int c = threadIdx.x; c < nJ; c += kPanT) xs[c] = xf[a0 + c + (int64_t)j * s];
        __syncthreads();
        for (int pr = warp; pr < tk.z; pr += nw) {
            const int64_t p = tk.y + pr;
            const T* P = panel + pan_off[tk.x] + p * nJ;
            T acc0 = T(0), acc1 = T(0);
            int c = lane;
            for (; c + 32 < nJ; c += 64) {
                acc0 += P[c] * xs[c];
                acc1 += P[c + 32] * xs[c + 32];
            }
            if (c < nJ) acc0 += P[c] * xs[c];
            const T acc = warp_sum(acc0 + acc1);
            if (lane == 0) wbuf[r_off[tk.x] + p + (int64_t)j * nrow] = acc;
        }
        __syncthreads();
    }
}

// backward, phase 1: t_j = y_j - sum_p L[R_J[p], j] x[R_J[p]] for <= 32 columns
// (lane = column); 16 warps split the panel rows, 8 loads in flight per lane
template <typename T>
__global__ void __launch_bounds__(kPanT)
k_cbwd_panel(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ r_off,
             const int32_t* __restrict__ rows, const int64_t* __restrict__ pan_off, const T* __restrict__ panel,
             T* yf, const T* xf, int32_t s, int32_t nrhs) {
    constexpr int nw = kPanT / 32;
    __shared__ T red[nw][33];
    const int4 tk = tasks[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0, jl = tk.y + lane;
    const int64_t nr = r_off[tk.x + 1] - r_off[tk.x];
    const int32_t* R = rows + r_off[tk.x];
    const T* Pn = panel + pan_off[tk.x] + jl;
    const int64_t chunk = (nr + nw - 1) / nw, pb = warp * chunk, pe = min(nr, pb + chunk);
    for (int j = 0; j < nrhs; ++j) {
        const T* x = xf + (int64_t)j * s;
        T acc = T(0);
        if (lane < tk.z) {
            int64_t p = pb;
            for (; p + 7 < pe; p += 8) {
                T pv[8], xv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    pv[u] = Pn[(p + u) * nJ];
                    xv[u] = x[R[p + u]];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += pv[u] * xv[u];
            }
            for (; p < pe; ++p) acc += Pn[p * nJ] * x[R[p]];
        }
        red[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && lane < tk.z) {
            T v = T(0);
#pragma unroll
            for (int w = 0; w < nw; ++w) v += red[w][lane];
            yf[a0 + jl + (int64_t)j * s] -= v;
        }
        __syncthreads();
    }
}

// backward, phase 2: x_J = L_JJ^{-T} t_J (warp per column, lanes over the column,
// 8 loads in flight per lane), optional scatter to DD order
template <typename T>
__global__ void __launch_bounds__(kDiagT)
k_cbwd_diag(const int4* __restrict__ tasks, const int32_t* __restrict__ c0, const int64_t* __restrict__ dinv_off,
            const T* __restrict__ dinv, const int32_t* __restrict__ cperm, const T* tf, T* xf, T* y_dd,
            int64_t ldy, int32_t s, int32_t nrhs) {
    const int4 tk = tasks[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int32_t a0 = c0[tk.x], nJ = c0[tk.x + 1] - a0;
    const T* D = dinv + dinv_off[tk.x];
    for (int cc = warp; cc < tk.z; cc += nwarp) {
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

// Fused levels: one CTA per supernode J with n_J <= kSmallN and |R_J| <= kSmallR.
static_assert(kThreads == 2 * kSmallN, "k_cbwd_small pairs two threads per column");
// forward: t_J = g_J - (gathered panel products); x_J = L_JJ^{-1} t_J; w_J = L[R_J, J] x_J
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cfwd_small(const int32_t* __restrict__ sns, const int32_t* __restrict__ c0, const int32_t* __restrict__ cperm,
             const int64_t* __restrict__ seg_ptr, const int32_t* __restrict__ seg_row, const int64_t* __restrict__ r_off,
             const int64_t* __restrict__ pan_off, const T* __restrict__ panel, const int64_t* __restrict__ dinv_off,
             const T* __restrict__ dinv, T* wbuf, int64_t nrow, const T* g, int64_t ldg, T* xf, int32_t s,
             int32_t nrhs) {
    __shared__ T ts[kSmallN], xs[kSmallN];
    const int J = sns[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
    const int32_t a0 = c0[J], nJ = c0[J + 1] - a0;
    const int64_t nr = r_off[J + 1] - r_off[J];
    const T* D = dinv + dinv_off[J];
    const T* Pn = panel + pan_off[J];
    for (int j = 0; j < nrhs; ++j) {
        const T* w = wbuf + (int64_t)j * nrow;
        for (int i = threadIdx.x; i < nJ; i += kThreads) {
            const int32_t pos = a0 + i;
            T acc = T(0);
            for (int64_t e = seg_ptr[pos]; e < seg_ptr[pos + 1]; ++e) acc += w[seg_row[e]];
            ts[i] = g[cperm[pos] + j * ldg] - acc;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nJ; i += kThreads) {
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
        __syncthreads();
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
        __syncthreads();
    }
}

// backward: t_J = y_J - L[R_J, J]^T x_{R_J};  x_J = L_JJ^{-T} t_J (and scatter to DD order)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_cbwd_small(const int32_t* __restrict__ sns, const int32_t* __restrict__ c0, const int64_t* __restrict__ r_off,
             const int32_t* __restrict__ rows, const int64_t* __restrict__ pan_off, const T* __restrict__ panel,
             const int64_t* __restrict__ dinv_off, const T* __restrict__ dinv, const int32_t* __restrict__ cperm,
             const T* yf, T* xf, T* y_dd, int64_t ldy, int32_t s, int32_t nrhs) {
    __shared__ T xr[kSmallR], ts[kSmallN];
    __shared__ T red[2][kSmallN];
    const int J = sns[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
    const int32_t a0 = c0[J], nJ = c0[J + 1] - a0;
    const int64_t nr = r_off[J + 1] - r_off[J];
    const int32_t* R = rows + r_off[J];
    const T* D = dinv + dinv_off[J];
    const T* Pn = panel + pan_off[J];
    for (int j = 0; j < nrhs; ++j) {
        const T* x = xf + (int64_t)j * s;
        for (int64_t p = threadIdx.x; p < nr; p += kThreads) xr[p] = x[R[p]];
        __syncthreads();
        // two halves of the panel rows per column, thread (half, column)
        {
            const int half = threadIdx.x / kSmallN, c = threadIdx.x % kSmallN;
            T acc = T(0);
            if (c < nJ) {
                const int64_t mid = (nr + 1) / 2, pb = half ? mid : 0, pe = half ? nr : mid;
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
            red[half][c] = acc;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < nJ; c += kThreads)
            ts[c] = yf[a0 + c + (int64_t)j * s] - (red[0][c] + red[1][c]);
        __syncthreads();
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
        __syncthreads();
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

template <typename T>
cudaError_t launch_c_forward(const DevCFactor<T>& cf, const T* g_dd, int64_t ldg, T* tf, T* xf, int32_t nrhs,
                             cudaStream_t st) {
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
        k_cbwd_panel<T><<<nt, kPanT, 0, st>>>(cf.tasks + t0, cf.c0, cf.r_off, cf.rows, cf.pan_off, cf.panel,
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
