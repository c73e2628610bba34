// Vector kernels of the preconditioned CG loop of Section 6 for a block of
// right-hand sides (DD order, column j of every vector at offset j n), fused so
// that each iteration streams its n x nrhs vectors as few times as it can:
//
//   q = A p and p.q                       one pass (k_pcg_spmv_dot)
//   x += alpha p, r -= alpha q, r.r, r.z  one pass (k_pcg_xr_dots); with a
//                                         single-precision preconditioner it also
//                                         writes r rounded to FP32, the input of
//                                         the next apply, and r.z is the product
//                                         of the flexible (Polak-Ribiere) beta
//                                         with the z of the apply just done
//   r.z after an apply                    k_pcg_dot with z in the apply's precision
//   p = z + beta p                        k_pcg_update_p with z in that precision
//
// Every dot product has a fixed reduction: block b of a column's G blocks (128;
// 256 in q = Ap) sums the elements i = b*256 + t + m*256G (t its thread,
// m = 0, 1, ...) in that order per thread, then the block's warps by a butterfly
// and the warp sums in order, then a final kernel sums the G block sums (lane l
// the blocks l, l+32, ...; then a butterfly).  A column's dots do not depend on
// the other columns of the block, and an FP32 z enters exactly (widened to FP64
// before the product).
#include <cuda_runtime.h>

#include <cstdint>

#include "slr_device.h"

namespace slr {

namespace {

constexpr int kPcgThreads = 256;
constexpr int kPcgWarps = kPcgThreads / 32;

__device__ __forceinline__ double pcg_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of one value per thread, in the fixed order; valid in thread 0.
__device__ __forceinline__ double pcg_block_sum(double v, double* red) {
    v = pcg_warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < kPcgWarps ? red[threadIdx.x] : 0.0;
        s = pcg_warp_sum(s);
    }
    return s;
}

// Each thread of a dot walks its elements i, i + S, i + 2S, ... (S = 256 G) four
// at a time: the four elements' loads are issued together, their products
// added in element order.
constexpr int kUnroll = 4;
// Blocks per column of the x/r update and of r.z: fewer, longer-running blocks
// than q = Ap takes (measured 7% and 8% faster on 3-D 96^3 with 32 columns)
constexpr int kDotBlocks = 128;

// part[j G + b] = block b's share of sum_i a[i + j n] b[i + j n]
template <typename TB>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_dot(int64_t n, const double* __restrict__ a, const TB* __restrict__ b, double* __restrict__ part) {
    __shared__ double red[kPcgWarps];
    const int j = blockIdx.y;
    const double* x = a + (int64_t)j * n;
    const TB* y = b + (int64_t)j * n;
    const int64_t S = (int64_t)gridDim.x * kPcgThreads;
    int64_t i = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x;
    double acc = 0.0;
    for (; i + (kUnroll - 1) * S < n; i += kUnroll * S) {
        double xv[kUnroll], yv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            xv[u] = x[i + u * S];
            yv[u] = (double)y[i + u * S];
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) acc += xv[u] * yv[u];
    }
    for (; i < n; i += S) acc += x[i] * (double)y[i];
    acc = pcg_block_sum(acc, red);
    if (threadIdx.x == 0) part[(int64_t)j * gridDim.x + blockIdx.x] = acc;
}

// q = A p (CSR) and the block shares of p.q.  A thread takes a row for CG
// columns at once (grid.y = column groups), so the matrix is read once per group
// instead of once per column; each column's row sum runs over the row's entries
// in order.
template <int CG>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_spmv_dot(int64_t n, int32_t nrhs, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
               const double* __restrict__ v, const double* __restrict__ p, double* __restrict__ q,
               double* __restrict__ part) {
    __shared__ double red[CG][kPcgWarps];
    const int j0 = blockIdx.y * CG;
    const int nc = min(CG, nrhs - j0);
    const double* pj = p + (int64_t)j0 * n;
    double* qj = q + (int64_t)j0 * n;
    double acc[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) acc[c] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kPcgThreads) {
        double sum[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) sum[c] = 0.0;
        const int32_t e1 = rp[i + 1];
        for (int32_t e = rp[i]; e < e1; ++e) {
            const double a = v[e];
            const int64_t col = ci[e];
#pragma unroll
            for (int c = 0; c < CG; ++c)
                if (c < nc) sum[c] += a * pj[c * n + col];
        }
#pragma unroll
        for (int c = 0; c < CG; ++c)
            if (c < nc) {
                qj[c * n + i] = sum[c];
                acc[c] += pj[c * n + i] * sum[c];
            }
    }
#pragma unroll
    for (int c = 0; c < CG; ++c) {
        const double t = pcg_block_sum(acc[c], red[c]);
        if (threadIdx.x == 0 && c < nc) part[(int64_t)(j0 + c) * gridDim.x + blockIdx.x] = t;
    }
}

// Active columns: x += alpha p, r -= alpha q (and r32 = fl32(r) when r32 is
// given).  Every column: block shares of r.r (part) and, when z is given, of r.z
// (part + nrhs G).
template <typename TZ>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_xr_dots(int64_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
              const double* __restrict__ q, float* __restrict__ r32, const TZ* __restrict__ z,
              const double* __restrict__ scal, const int32_t* __restrict__ flags, double* __restrict__ part) {
    __shared__ double red[2][kPcgWarps];
    const int j = blockIdx.y;
    const int64_t o = (int64_t)j * n;
    x += o;
    r += o;
    p += o;
    q += o;
    if (r32) r32 += o;
    if (z) z += o;
    const bool active = flags[4 * j] != 0;
    const double a = scal[8 * j + 2];
    const int64_t S = (int64_t)gridDim.x * kPcgThreads;
    int64_t i = (int64_t)blockIdx.x * kPcgThreads + threadIdx.x;
    double rr = 0.0, rz = 0.0;
    for (; i + (kUnroll - 1) * S < n; i += kUnroll * S) {
        double rv[kUnroll], zv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            rv[u] = r[i + u * S];
            zv[u] = z ? (double)z[i + u * S] : 0.0;
        }
        if (active) {
            double xv[kUnroll], pv[kUnroll], qv[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                xv[u] = x[i + u * S];
                pv[u] = p[i + u * S];
                qv[u] = q[i + u * S];
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                x[i + u * S] = xv[u] + a * pv[u];
                rv[u] -= a * qv[u];
                r[i + u * S] = rv[u];
                if (r32) r32[i + u * S] = (float)rv[u];
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            rr += rv[u] * rv[u];
            rz += rv[u] * zv[u];
        }
    }
    for (; i < n; i += S) {
        double rv = r[i];
        if (active) {
            x[i] += a * p[i];
            rv -= a * q[i];
            r[i] = rv;
            if (r32) r32[i] = (float)rv;
        }
        rr += rv * rv;
        if (z) rz += rv * (double)z[i];
    }
    rr = pcg_block_sum(rr, red[0]);
    if (z) rz = pcg_block_sum(rz, red[1]);
    if (threadIdx.x == 0) {
        part[(int64_t)j * gridDim.x + blockIdx.x] = rr;
        if (z) part[((int64_t)gridDim.y + j) * gridDim.x + blockIdx.x] = rz;
    }
}

// out0[j stride] = sum of part[j G ...], and, when out1 is given,
// out1[j stride] = sum of part[(cols + j) G ...]; one warp per sum
__global__ void k_pcg_dot_final(int32_t cols, int32_t G, const double* __restrict__ part, double* out0,
                                double* out1, int32_t stride) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int nsum = out1 ? 2 * cols : cols;
    if (w >= nsum) return;
    double acc = 0.0;
    for (int b = lane; b < G; b += 32) acc += part[(int64_t)w * G + b];
    acc = pcg_warp_sum(acc);
    if (lane == 0) (w < cols ? out0 + (int64_t)w * stride : out1 + (int64_t)(w - cols) * stride)[0] = acc;
}

// p = z + beta p on the active columns; block (b, j) takes column j's elements
// b*1024 + t + 256 u, u < 4, their loads issued together
template <typename TZ>
__global__ void __launch_bounds__(kPcgThreads)
k_pcg_update_p(int64_t n, double* __restrict__ p, const TZ* __restrict__ z, const double* __restrict__ scal,
               const int32_t* __restrict__ flags) {
    const int j = blockIdx.y;
    if (!flags[4 * j]) return;
    const double beta = scal[8 * j + 5];
    const int64_t i0 = (int64_t)blockIdx.x * (kUnroll * kPcgThreads) + threadIdx.x;
    p += (int64_t)j * n;
    z += (int64_t)j * n;
    if (i0 + (kUnroll - 1) * kPcgThreads < n) {
        double pv[kUnroll], zv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            pv[u] = p[i0 + u * kPcgThreads];
            zv[u] = (double)z[i0 + u * kPcgThreads];
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) p[i0 + u * kPcgThreads] = zv[u] + beta * pv[u];
    } else {
        for (int64_t i = i0; i < n; i += kPcgThreads) p[i] = (double)z[i] + beta * p[i];
    }
}

cudaError_t dot_final(int32_t cols, int32_t G, const double* part, double* out0, double* out1, int32_t stride,
                      cudaStream_t st) {
    const int sums = out1 ? 2 * cols : cols;
    const int per = kPcgThreads / 32;
    k_pcg_dot_final<<<(sums + per - 1) / per, kPcgThreads, 0, st>>>(cols, G, part, out0, out1, stride);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

template <typename TB>
cudaError_t launch_pcg_dot(int64_t n, int32_t cols, const double* a, const TB* b, double* part, double* out,
                           int32_t out_stride, cudaStream_t st) {
    if (cols == 0) return cudaSuccess;
    k_pcg_dot<TB><<<dim3(kDotBlocks, cols), kPcgThreads, 0, st>>>(n, a, b, part);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : dot_final(cols, kDotBlocks, part, out, nullptr, out_stride, st);
}

cudaError_t launch_pcg_spmv_dot(int64_t n, int32_t nrhs, const int32_t* rp, const int32_t* ci, const double* v,
                                const double* p, double* q, double* part, double* scal, cudaStream_t st) {
    if (nrhs == 0) return cudaSuccess;
    constexpr int CG = 1;      // a column per block row: measured faster than groups of 8 on A's 7-point rows
    k_pcg_spmv_dot<CG><<<dim3(kRedBlocks, (nrhs + CG - 1) / CG), kPcgThreads, 0, st>>>(n, nrhs, rp, ci, v, p, q,
                                                                                      part);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : dot_final(nrhs, kRedBlocks, part, scal + 1, nullptr, 8, st);
}

template <typename TZ>
cudaError_t launch_pcg_xr_dots(int64_t n, int32_t nrhs, double* x, double* r, const double* p, const double* q,
                               float* r32, const TZ* z, double* scal, const int32_t* flags, double* part,
                               cudaStream_t st) {
    if (nrhs == 0) return cudaSuccess;
    k_pcg_xr_dots<TZ><<<dim3(kDotBlocks, nrhs), kPcgThreads, 0, st>>>(n, x, r, p, q, r32, z, scal, flags, part);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : dot_final(nrhs, kDotBlocks, part, scal + 3, z ? scal + 7 : nullptr, 8, st);
}

template <typename TZ>
cudaError_t launch_pcg_update_pz(int64_t n, int32_t nrhs, double* p, const TZ* z, const double* scal,
                                 const int32_t* flags, cudaStream_t st) {
    if (n == 0 || nrhs == 0) return cudaSuccess;
    const int64_t per = (int64_t)kUnroll * kPcgThreads;
    k_pcg_update_p<TZ><<<dim3((unsigned)((n + per - 1) / per), nrhs), kPcgThreads, 0, st>>>(n, p, z, scal, flags);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_pcg_dot<double>(int64_t, int32_t, const double*, const double*, double*, double*,
                                            int32_t, cudaStream_t);
template cudaError_t launch_pcg_dot<float>(int64_t, int32_t, const double*, const float*, double*, double*,
                                           int32_t, cudaStream_t);
template cudaError_t launch_pcg_xr_dots<double>(int64_t, int32_t, double*, double*, const double*, const double*,
                                                float*, const double*, double*, const int32_t*, double*,
                                                cudaStream_t);
template cudaError_t launch_pcg_xr_dots<float>(int64_t, int32_t, double*, double*, const double*, const double*,
                                               float*, const float*, double*, const int32_t*, double*,
                                               cudaStream_t);
template cudaError_t launch_pcg_update_pz<double>(int64_t, int32_t, double*, const double*, const double*,
                                                  const int32_t*, cudaStream_t);
template cudaError_t launch_pcg_update_pz<float>(int64_t, int32_t, double*, const float*, const double*,
                                                 const int32_t*, cudaStream_t);

}  // namespace slr
