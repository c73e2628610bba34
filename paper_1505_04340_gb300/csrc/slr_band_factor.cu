// Band factorization on the device (Section 5.2: B_i = L_i L_i^T, the factor the
// B solves use), batched over the subdomains, for sm_103a.
//
// With planes of W = w rows, B_i is block tridiagonal: diagonal blocks A_JJ and
// sub-diagonal blocks A_{J+1,J} (upper triangular inside the band).  Its Cholesky
// factor follows plane by plane:
//   S_J    = A_JJ - O_J O_J^T            (O_0 = 0)
//   L_JJ   = chol(S_J),   D_J = L_JJ^{-1}
//   O_{J+1} = L[J+1, J] = A_{J+1,J} L_JJ^{-T} = A_{J+1,J} D_J^T
// which is the same factor the host's column-oriented band Cholesky computes (up
// to rounding).  For a symmetric indefinite A (SPD interface, Section 1) the
// blocks are factored as L_JJ S_J L_JJ^T with S_J the pivot signs (no pivoting):
// S_J = A_JJ - O_J S_{J-1} O_J^T and O_{J+1} = A_{J+1,J} D_J^T S_J; the pack
// kernel folds the signs into the forward blocks (O_J S_{J-1}, S_J D_J).
// One CTA of 512 threads per subdomain walks its planes; the dense W x W blocks
// (W <= 256) live in a global scratch area, worked on in 32 x 32 tiles staged in
// shared memory.  Rows of the last plane past m are identity rows, as in the host
// factor.  A pivot <= 0 (zero when indefinite) records the subdomain in *bad and
// stops that CTA.  A second kernel packs D_J and O_J into the tiled slice layout the band
// solve streams (the same layout the host packer writes, for any split G), in the
// operator's precision.
#include <cuda_runtime.h>

#include <cstdint>

#include "slr_device.h"

namespace slr {

namespace {

constexpr int kFT = 512;   // threads of the factorization CTA (16 warps)

struct Tile {
    double v[32][33];
};

// Loads the 32 x 32 tile at (r0, c0) of the row-major W x W matrix M (zero past W).
__device__ __forceinline__ void load_tile(Tile& t, const double* M, int W, int r0, int c0) {
    for (int i = threadIdx.x; i < 1024; i += kFT) {
        const int r = i >> 5, c = i & 31;
        t.v[r][c] = (r0 + r < W && c0 + c < W) ? M[(int64_t)(r0 + r) * W + c0 + c] : 0.0;
    }
}

// S[ti, tj] -= A diag(sg) B^T summed over the 32-column chunks kc0 .. nt-1 (A: rows
// of tile ti of X, B: rows of tile tj of Y, both row-major W x W; sg: signs of the
// summed columns, or null for all +1), lower entries of S only.
__device__ void tile_sub_abt(double* S, const double* X, const double* Y, int W, int ti, int tj, int kc0, int nt,
                             Tile& ta, Tile& tb, const double* sg = nullptr) {
    const int row = threadIdx.x >> 4, col = (threadIdx.x & 15) * 2;
    double acc0 = 0.0, acc1 = 0.0;
    for (int kc = kc0; kc < nt; ++kc) {
        __syncthreads();
        load_tile(ta, X, W, 32 * ti, 32 * kc);
        load_tile(tb, Y, W, 32 * tj, 32 * kc);
        __syncthreads();
        if (sg) {
            for (int i = threadIdx.x; i < 1024; i += kFT) {
                const int c = 32 * kc + (i & 31);
                if (c < W) ta.v[i >> 5][i & 31] *= sg[c];
            }
            __syncthreads();
        }
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            const double a = ta.v[row][q];
            acc0 = fma(a, tb.v[col][q], acc0);
            acc1 = fma(a, tb.v[col + 1][q], acc1);
        }
    }
    const int r = 32 * ti + row, c = 32 * tj + col;
    if (r < W) {
        if (c < W && c <= r) S[(int64_t)r * W + c] -= acc0;
        if (c + 1 < W && c + 1 <= r) S[(int64_t)r * W + c + 1] -= acc1;
    }
}

// In-place Cholesky of the lower triangle of S (right-looking, 32-column panels):
// S = L L^T, or with indef S = L diag(sg) L^T, the signs of the pivots into sg[W].
// Returns false (uniformly) if a pivot is not positive (SPD) or is zero (indef).
__device__ bool chol_blocked(double* S, int W, int nt, Tile& ta, Tile& tb, int* flag, double* sg, bool indef) {
    __shared__ double tsg[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int kb = 0; kb < nt; ++kb) {
        // diagonal tile: unblocked Cholesky by warp 0 (lane = row); rows past W get 1 on the diagonal
        __syncthreads();
        for (int i = tid; i < 1024; i += kFT) {
            const int r = i >> 5, c = i & 31, gr = 32 * kb + r, gc = 32 * kb + c;
            ta.v[r][c] = (gr < W && gc < W) ? S[(int64_t)gr * W + gc] : (r == c ? 1.0 : 0.0);
        }
        if (tid == 0) *flag = 0;
        __syncthreads();
        if (warp == 0) {
            for (int j = 0; j < 32; ++j) {
                if (lane == j) {
                    const double d = ta.v[j][j];
                    double sj = 1.0;
                    if (indef) {
                        if (!(fabs(d) > 0.0)) *flag = 1;
                        sj = d < 0.0 ? -1.0 : 1.0;
                    } else if (!(d > 0.0)) {
                        *flag = 1;
                    }
                    tsg[j] = sj;
                    ta.v[j][j] = sqrt(fabs(d));
                }
                __syncwarp();
                const double djj = ta.v[j][j] * tsg[j];   // s_j l_jj
                if (lane > j) ta.v[lane][j] = djj != 0.0 ? ta.v[lane][j] / djj : 0.0;
                __syncwarp();
                if (lane > j) {
                    const double lj = ta.v[lane][j] * tsg[j];
                    for (int k = j + 1; k <= lane; ++k) ta.v[lane][k] -= lj * ta.v[k][j];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (*flag) return false;
        for (int i = tid; i < 1024; i += kFT) {
            const int r = i >> 5, c = i & 31, gr = 32 * kb + r, gc = 32 * kb + c;
            if (gr < W && gc < W && c <= r) S[(int64_t)gr * W + gc] = ta.v[r][c];
        }
        if (tid < 32 && 32 * kb + tid < W) sg[32 * kb + tid] = tsg[tid];
        // panel below: row r of L[ib, kb] solves x diag(s) L_kk^T = S[r, kb block] (forward substitution)
        for (int r = 32 * (kb + 1) + tid; r < W; r += kFT) {
            double x[32];
            double* Sr = S + (int64_t)r * W + 32 * kb;
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = (32 * kb + j < W) ? Sr[j] : 0.0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                double s = x[j];
#pragma unroll
                for (int q = 0; q < j; ++q) s -= x[q] * tsg[q] * ta.v[j][q];
                x[j] = s / (tsg[j] * ta.v[j][j]);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (32 * kb + j < W) Sr[j] = x[j];
        }
        __syncthreads();
        // trailing update of the lower tiles: S[ib, jb] -= L[ib, kb] L[jb, kb]^T, kb < jb <= ib
        for (int ib = kb + 1; ib < nt; ++ib)
            for (int jb = kb + 1; jb <= ib; ++jb) tile_sub_abt(S, S, S, W, ib, jb, kb, kb + 1, ta, tb, sg);
    }
    __syncthreads();
    return true;
}

// X = L^{-1} (lower, row-major W x W) for the lower-triangular L in S.
__device__ void trtri_blocked(const double* S, double* X, int W, int nt, Tile& ta, Tile& tb) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < W * W; i += kFT) X[i] = 0.0;
    __syncthreads();
    // diagonal blocks: warp w inverts block w (lane = column; rows past W are identity)
    for (int kb = warp; kb < nt; kb += kFT / 32) {
        const int c0 = 32 * kb;
        auto L = [&](int r, int c) -> double {
            const int gr = c0 + r, gc = c0 + c;
            return (gr < W && gc < W) ? S[(int64_t)gr * W + gc] : (r == c ? 1.0 : 0.0);
        };
        double x[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) x[r] = 0.0;
        for (int r = 0; r < 32; ++r) {
            double s = (r == lane) ? 1.0 : 0.0;
            for (int q = lane; q < r; ++q) s -= L(r, q) * x[q];
            x[r] = r >= lane ? s / L(r, r) : 0.0;
        }
        for (int r = 0; r < 32; ++r)
            if (c0 + r < W && c0 + lane < W) X[(int64_t)(c0 + r) * W + c0 + lane] = x[r];
    }
    __syncthreads();
    // off-diagonal blocks, block row by block row: X[ib, jb] = -X[ib, ib] sum_{kb=jb}^{ib-1} L[ib, kb] X[kb, jb]
    const int row = tid >> 4, col = (tid & 15) * 2;
    for (int ib = 1; ib < nt; ++ib) {
        for (int jb = 0; jb < ib; ++jb) {
            double t0 = 0.0, t1 = 0.0;
            for (int kb = jb; kb < ib; ++kb) {
                __syncthreads();
                load_tile(ta, S, W, 32 * ib, 32 * kb);
                load_tile(tb, X, W, 32 * kb, 32 * jb);
                __syncthreads();
#pragma unroll 8
                for (int q = 0; q < 32; ++q) {
                    const double a = ta.v[row][q];
                    t0 = fma(a, tb.v[q][col], t0);
                    t1 = fma(a, tb.v[q][col + 1], t1);
                }
            }
            __syncthreads();
            tb.v[row][col] = t0;
            tb.v[row][col + 1] = t1;
            load_tile(ta, X, W, 32 * ib, 32 * ib);
            __syncthreads();
            double u0 = 0.0, u1 = 0.0;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                const double a = ta.v[row][q];
                u0 = fma(a, tb.v[q][col], u0);
                u1 = fma(a, tb.v[q][col + 1], u1);
            }
            const int r = 32 * ib + row, c = 32 * jb + col;
            if (r < W) {
                if (c < W) X[(int64_t)r * W + c] = -u0;
                if (c + 1 < W) X[(int64_t)r * W + c + 1] = -u1;
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kFT, 1)
k_band_factor(const BandBlock* __restrict__ band, const int32_t* __restrict__ a_rp, const int32_t* __restrict__ a_ci,
              const double* __restrict__ a_v, double* scr, const int64_t* __restrict__ soff, int32_t* bad, int indef) {
    __shared__ Tile ta, tb;
    __shared__ int flag;
    const BandBlock b = band[blockIdx.x];
    if (b.m == 0) return;
    const int W = b.w, c = b.c, m = b.m, r0 = b.row0, nt = (W + 31) / 32, tid = threadIdx.x;
    const int64_t WW = (int64_t)W * W;
    double* S = scr + soff[b.id];
    double* Dst = S + WW;               // D_J = L_JJ^{-1} at Dst + J W^2
    double* Ost = Dst + (int64_t)c * WW;   // O_J = L[J, J-1] at Ost + J W^2 (O_0 = 0)
    double* Sg = Ost + (int64_t)c * WW;    // pivot signs of plane J at Sg + J W
    for (int J = 0; J < c; ++J) {
        // S = lower part of A_JJ (identity rows past m)
        for (int64_t i = tid; i < WW; i += kFT) S[i] = 0.0;
        __syncthreads();
        for (int r = tid; r < W; r += kFT) {
            const int l = J * W + r;
            if (l >= m) {
                S[(int64_t)r * W + r] = 1.0;
                continue;
            }
            for (int32_t q = a_rp[r0 + l]; q < a_rp[r0 + l + 1]; ++q) {
                const int k = a_ci[q] - r0 - J * W;
                if (k >= 0 && k <= r) S[(int64_t)r * W + k] = a_v[q];
            }
        }
        __syncthreads();
        // S -= O_J O_J^T (O_J upper triangular: column chunks from the row tile on)
        if (J > 0) {
            const double* O = Ost + (int64_t)J * WW;
            const double* sgp = indef ? Sg + (int64_t)(J - 1) * W : nullptr;
            for (int ti = 0; ti < nt; ++ti)
                for (int tj = 0; tj <= ti; ++tj) tile_sub_abt(S, O, O, W, ti, tj, ti, nt, ta, tb, sgp);
            __syncthreads();
        }
        if (!chol_blocked(S, W, nt, ta, tb, &flag, Sg + (int64_t)J * W, indef != 0)) {
            if (tid == 0) atomicCAS(bad, -1, (int32_t)blockIdx.x);
            return;
        }
        double* D = Dst + (int64_t)J * WW;
        trtri_blocked(S, D, W, nt, ta, tb);
        // O_{J+1}[r][k] = sum over the couplings q of row (J+1) W + r into plane J: A[r][q] D[k][q]
        if (J + 1 < c) {
            double* On = Ost + (int64_t)(J + 1) * WW;
            for (int64_t i = tid; i < WW; i += kFT) {
                const int r = (int)(i / W), k = (int)(i % W), l = (J + 1) * W + r;
                double s = 0.0;
                if (l < m)
                    for (int32_t q = a_rp[r0 + l]; q < a_rp[r0 + l + 1]; ++q) {
                        const int qq = a_ci[q] - r0 - J * W;
                        if (qq >= 0 && qq < W && qq <= k) s += a_v[q] * D[(int64_t)k * W + qq];
                    }
                On[i] = indef ? s * Sg[(int64_t)J * W + k] : s;
            }
            __syncthreads();
        }
    }
}

// One CTA per (subdomain, plane, slice): the four blocks of the slice, as the
// host packer writes them (slr_internal.h: [O_J | D_J | O_J^T | D_J^T]).
template <typename T>
__global__ void __launch_bounds__(256)
k_band_pack(const BandBlock* __restrict__ band, int32_t cmax, int32_t G, const double* __restrict__ scr,
            const int64_t* __restrict__ soff, T* bfac, int indef) {
    const int i = blockIdx.x / (cmax * G), J = (blockIdx.x / G) % cmax, g = blockIdx.x % G;
    const BandBlock b = band[i];
    if (b.m == 0 || J >= b.c) return;
    const int W = b.w, m = b.m;
    const int64_t WW = (int64_t)W * W;
    const double* S0 = scr + soff[b.id];                            // the blocks of subdomain b.id
    const double* X = S0 + WW + (int64_t)J * WW;                    // D_J
    const double* O = S0 + WW + (int64_t)(b.c + J) * WW;            // O_J
    const double* Sg = S0 + WW + 2 * (int64_t)b.c * WW;             // pivot signs, plane by plane
    auto sgn = [&](int plane, int r) -> double { return indef ? Sg[(int64_t)plane * W + r] : 1.0; };
    T* plane = bfac + b.foff + (int64_t)J * G * 2 * (b.SU + b.SL) + (int64_t)g * 2 * (b.SU + b.SL);
    T* Uf = plane;          // O_J      (upper)
    T* Lf = Uf + b.SU;      // D_J      (lower)
    T* Lb = Lf + b.SL;      // O_J^T    (lower)
    T* Ub = Lb + b.SL;      // D_J^T    (upper)
    int64_t su = 0, sl = 0;
    for (int rb = 0; rb < b.nrb[g]; ++rb) {
        const int R0 = 32 * b.rbmap[g][rb];
        const int cu0 = min(W, R0), cl1 = min(W, min(R0 + 31, W - 1) + 1);
        const int nu = W - cu0;
        for (int e = threadIdx.x; e < 32 * nu; e += blockDim.x) {   // upper: rows r <= cc
            const int cc = cu0 + e / 32, r = R0 + (e & 31), l = J * W + r;
            const bool in = r < W && r <= cc;
            Uf[(su * 32) + e] = in && J > 0 && l < m ? (T)(O[(int64_t)r * W + cc] * sgn(J - 1, cc)) : T(0);
            Ub[(su * 32) + e] = in ? (T)X[(int64_t)cc * W + r] : T(0);
        }
        for (int e = threadIdx.x; e < 32 * cl1; e += blockDim.x) {  // lower: rows r >= cc
            const int cc = e / 32, r = R0 + (e & 31), lc = J * W + cc;
            const bool in = r < W && r >= cc;
            Lf[(sl * 32) + e] = in ? (T)(X[(int64_t)r * W + cc] * sgn(J, r)) : T(0);
            Lb[(sl * 32) + e] = in && J > 0 && lc < m ? (T)O[(int64_t)cc * W + r] : T(0);
        }
        su += nu;
        sl += cl1;
    }
}

}  // namespace

cudaError_t launch_band_factor(const BandBlock* band, int32_t p, const int32_t* a_rp, const int32_t* a_ci,
                               const double* a_v, double* scr, const int64_t* soff, int32_t* bad, bool indef,
                               cudaStream_t st) {
    if (p == 0) return cudaSuccess;
    k_band_factor<<<p, kFT, 0, st>>>(band, a_rp, a_ci, a_v, scr, soff, bad, indef ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_band_pack(const BandBlock* band, int32_t p, int32_t cmax, int32_t G, const double* scr,
                             const int64_t* soff, T* bfac, bool indef, cudaStream_t st) {
    if (p == 0 || cmax == 0) return cudaSuccess;
    k_band_pack<T><<<(unsigned)p * cmax * G, 256, 0, st>>>(band, cmax, G, scr, soff, bfac, indef ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_band_pack<double>(const BandBlock*, int32_t, int32_t, int32_t, const double*,
                                              const int64_t*, double*, bool, cudaStream_t);
template cudaError_t launch_band_pack<float>(const BandBlock*, int32_t, int32_t, int32_t, const double*,
                                             const int64_t*, float*, bool, cudaStream_t);

}  // namespace slr
