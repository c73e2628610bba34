// K4 on the tensor cores: the two products of the low-rank correction of
// Eq. 4.7 (U-form), w' = cinv w + U_k (d o (U_k^T w)), for a block of right-hand
// sides of the FP32 apply, with U and w rounded to TF32 or BF16 and the products
// accumulated in FP32 in tensor memory (tcgen05.mma, cta_group::1, M = 128).
//
//   pass 1  V = U^T W        M = k (at most 128, padded), N = right-hand sides
//                            (padded to 16), K = the rows of the CTA's slice of s;
//                            A = U column-major (K-major as it is), B = W column-major
//   pass 2  W' = cinv W + U (d o V)   M = 128 rows of s, N = right-hand sides,
//                            K = k; A = a row-major copy of U, B = d o V
//
// Each CTA is 128 threads; thread 0 issues the MMAs, all threads stage operands
// (rounding them) into shared memory in the K-major core-matrix layout of
// slr_tc.cuh, and warp w reads accumulator lanes 32 w .. 32 w + 31.  Waits on the
// MMA completion barriers are bounded: one that runs out sets the operator's
// status word (3), the CTA stops issuing, waits (bounded) for what it issued,
// frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "slr_device.h"
#include "slr_tc.cuh"

namespace slr {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcKc = 32;                  // rows of s per stage of pass 1
constexpr long long kTcSpin = 1ll << 24;   // polls of a completion wait

template <int AB>
struct TcType;
template <>
struct TcType<2> {                          // TF32: FP32 storage, rounded when staged
    using U = float;
    static constexpr int E = 4;
    __device__ static float pack(float x) { return tc::to_tf32(x); }
};
template <>
struct TcType<1> {                          // BF16
    using U = __nv_bfloat16;
    static constexpr int E = 2;
    __device__ static __nv_bfloat16 pack(float x) { return __float2bfloat16_rn(x); }
};

template <int AB>
__device__ __forceinline__ float load_u(const typename TcType<AB>::U* p) {
    if constexpr (AB == 2) return *p;
    else return __bfloat162float(*p);
}

// row blocks of pass 1: the CUDA-core pass's partition of s (so both write the
// same partial-sum layout)
__host__ __device__ inline int tc_blocks(int32_t s) {
    const int b = (s + 127) / 128;
    return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

// UK, WK: columns of U (k <= 4 UK) and of W (nrhs <= 4 WK) a thread holds per chunk
template <int AB, int UK, int WK>
__global__ void __launch_bounds__(kTcThreads, 1)
k_lr_vt_tc(int32_t s, int32_t k, int32_t nrhs, int32_t np, const typename TcType<AB>::U* __restrict__ Ucm,
           const float* __restrict__ w, float* part, int32_t* err) {
    using Tp = TcType<AB>;
    using Te = typename Tp::U;
    constexpr int E = Tp::E;
    constexpr int M = 128;
    constexpr uint32_t kA = M * kTcKc * E, kB = 64 * kTcKc * E;   // bytes of one stage's A and B tiles
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sA = sm;                         // [2][kA]
    unsigned char* sB = sm + 2 * kA;                // [2][kB]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kA + 2 * kB);   // [2] stage free, [2] final
    uint32_t* tbase = reinterpret_cast<uint32_t*>(bar + 3);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t ncol = np <= 32 ? 32 : 64;
    if (warp == 0) {
        tc::tmem_alloc(tbase, ncol);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::mbar_init(&bar[2], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // rows k .. 127 of A and nrhs .. np-1 of B stay zero in both stages
    for (int i = t; i < (int)(2 * kA + 2 * kB) / 16; i += kTcThreads)
        reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tbase;
    const int R = (s + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * R, r1 = min(s, r0 + R);
    const uint32_t idesc = tc::instr_desc(AB, M, np);
    bool ok = true;
    int nchunks = 0;
    // a thread's share of a chunk: row q of s, columns m = m0 + 4 i of U (i < UK) and
    // n = m0 + 4 i of W (i < WK); its values are loaded into registers one chunk ahead,
    // so the loads of the next chunk are in flight while this one's MMAs run
    constexpr int kStep = kTcThreads / kTcKc;
    const int q = t % kTcKc, m0 = t / kTcKc;        // consecutive threads: consecutive rows (coalesced)
    static_assert(kStep == 4, "four rows of U and W per thread step");
    float ur[UK], wr[WK];
    auto fetch = [&](int c0) {
        const int rows = min(kTcKc, r1 - c0);
#pragma unroll
        for (int i = 0; i < UK; ++i) {
            const int m = m0 + kStep * i;
            ur[i] = (q < rows && m < k) ? load_u<AB>(Ucm + (c0 + q) + (int64_t)m * s) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < WK; ++i) {
            const int n = m0 + kStep * i;
            wr[i] = (q < rows && n < nrhs) ? w[(c0 + q) + (int64_t)n * s] : 0.0f;
        }
    };
    if (r0 < r1) fetch(r0);
    for (int c0 = r0; c0 < r1; c0 += kTcKc, ++nchunks) {
        const int st = nchunks & 1;
        if (nchunks >= 2 && ok) ok = tc::mbar_wait(&bar[st], (uint32_t)(((nchunks - 2) >> 1) & 1), kTcSpin);
        ok = __syncthreads_and(ok);
        if (!ok) break;
        unsigned char* a = sA + st * kA;
        unsigned char* b = sB + st * kB;
#pragma unroll
        for (int i = 0; i < UK; ++i) {
            const int m = m0 + kStep * i;
            if (m < k) *reinterpret_cast<Te*>(a + tc::kmajor_off<E>(m, q, kTcKc)) = Tp::pack(ur[i]);
        }
#pragma unroll
        for (int i = 0; i < WK; ++i) {
            const int n = m0 + kStep * i;
            if (n < nrhs) *reinterpret_cast<Te*>(b + tc::kmajor_off<E>(n, q, kTcKc)) = Tp::pack(wr[i]);
        }
        if (c0 + kTcKc < r1) fetch(c0 + kTcKc);
        tc::fence_async_smem();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_addr(a), sb = tc::smem_addr(b);
#pragma unroll
            for (int step = 0; step < kTcKc * E / 32; ++step)
                tc::mma<AB>(tmem, tc::smem_desc(sa + 256 * step, 128, 8 * kTcKc * E),
                            tc::smem_desc(sb + 256 * step, 128, 8 * kTcKc * E), idesc, nchunks > 0 || step > 0);
            tc::commit(&bar[st]);
        }
    }
    // every MMA issued has completed (bounded even after a failure, so nothing is in flight)
    if (t == 0) tc::commit(&bar[2]);
    bool fin = tc::mbar_wait(&bar[2], 0, kTcSpin);
    fin = __syncthreads_and(fin);
    if (!(ok && fin)) {
        if (t == 0) atomicExch(err, 3);
    } else {
        tc::fence_after_sync();
        const int kk = 32 * warp + lane;
        for (int c = 0; c < np; c += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            if (kk < k) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c + j < nrhs)
                        part[((int64_t)blockIdx.x * k + kk) * nrhs + c + j] = nchunks > 0 ? v[j] : 0.0f;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc::tmem_dealloc(tmem, ncol);
    }
}

template <int AB>
__global__ void __launch_bounds__(kTcThreads, 1)
k_lr_update_tc(int32_t s, int32_t k, int32_t kp, int32_t nrhs, int32_t np, const typename TcType<AB>::U* __restrict__ Urm,
               const float* __restrict__ vk, float cinv, float* w, int32_t* err) {
    using Tp = TcType<AB>;
    using Te = typename Tp::U;
    constexpr int E = Tp::E;
    constexpr int M = 128;
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t kA = M * kp * E, kB = 64 * kp * E;
    unsigned char* sA = sm;
    unsigned char* sB = sm + kA;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kA + kB);
    uint32_t* tbase = reinterpret_cast<uint32_t*>(bar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t ncol = np <= 32 ? 32 : 64;
    if (warp == 0) {
        tc::tmem_alloc(tbase, ncol);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(&bar[0], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int64_t i0 = (int64_t)blockIdx.x * M;
    const int rows = (int)((s - i0) < M ? (s - i0) : M);
    // rows of U: sixteen loads in flight per thread before any is stored
    for (int e0 = t; e0 < M * kp; e0 += 16 * kTcThreads) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = e0 + u * kTcThreads, r = e / kp, q = e % kp;
            v[u] = (e < M * kp && r < rows && q < k) ? load_u<AB>(Urm + (i0 + r) * k + q) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = e0 + u * kTcThreads, r = e / kp, q = e % kp;
            if (e < M * kp) *reinterpret_cast<Te*>(sA + tc::kmajor_off<E>(r, q, kp)) = Tp::pack(v[u]);
        }
    }
    for (int e = t; e < np * kp; e += kTcThreads) {
        const int n = e / kp, q = e % kp;
        const float v = (n < nrhs && q < k) ? vk[q + (int64_t)n * k] : 0.0f;
        *reinterpret_cast<Te*>(sB + tc::kmajor_off<E>(n, q, kp)) = Tp::pack(v);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tbase;
    if (t == 0) {
        const uint32_t sa = tc::smem_addr(sA), sb = tc::smem_addr(sB), idesc = tc::instr_desc(AB, M, np);
        for (int step = 0; step < kp * E / 32; ++step)
            tc::mma<AB>(tmem, tc::smem_desc(sa + 256 * step, 128, 8 * kp * E), tc::smem_desc(sb + 256 * step, 128, 8 * kp * E),
                        idesc, step > 0);
        tc::commit(&bar[0]);
    }
    bool fin = tc::mbar_wait(&bar[0], 0, kTcSpin);
    fin = __syncthreads_and(fin);
    if (!fin) {
        if (t == 0) atomicExch(err, 3);
    } else {
        tc::fence_after_sync();
        const int r = 32 * warp + lane;
        for (int c = 0; c < np; c += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            if (r < rows) {
                float o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) o[j] = c + j < nrhs ? w[i0 + r + (int64_t)(c + j) * s] : 0.0f;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c + j < nrhs) w[i0 + r + (int64_t)(c + j) * s] = cinv * o[j] + v[j];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc::tmem_dealloc(tmem, ncol);
    }
}

// V = d o (sum over the pass-1 blocks of their partial products), in a fixed order:
// block (kk, j-group) has kFinSeg segments of the G blocks, each summed in order by
// its threads (the right-hand sides j fastest: coalesced), then the segment sums
// added in order
constexpr int kFinSeg = 16, kFinJ = 16;
__global__ void __launch_bounds__(kFinSeg * kFinJ)
k_lr_fin_tc(int32_t k, int32_t nrhs, int32_t G, const float* __restrict__ part, const float* __restrict__ dvec,
            float* vk) {
    __shared__ float seg[kFinSeg][kFinJ];
    const int kk = blockIdx.x, j = blockIdx.y * kFinJ + (threadIdx.x % kFinJ), q = threadIdx.x / kFinJ;
    const int len = (G + kFinSeg - 1) / kFinSeg, b0 = q * len, b1 = min(G, b0 + len);
    float acc = 0.0f;
    if (j < nrhs) {
        int b = b0;
        for (; b + 4 <= b1; b += 4) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = part[((int64_t)(b + u) * k + kk) * nrhs + j];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += v[u];
        }
        for (; b < b1; ++b) acc += part[((int64_t)b * k + kk) * nrhs + j];
    }
    seg[q][threadIdx.x % kFinJ] = acc;
    __syncthreads();
    if (q == 0 && j < nrhs) {
        float v = 0.0f;
        for (int qq = 0; qq < kFinSeg; ++qq) v += seg[qq][threadIdx.x];
        vk[kk + (int64_t)j * k] = dvec[kk] * v;
    }
}

template <typename Te>
__global__ void k_lr_pack(int32_t s, int32_t k, const double* __restrict__ U, Te* Urm, Te* Ucm) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)s * k) return;
    const int64_t i = e % s, kk = e / s;
    const float v = (float)U[e];
    if constexpr (sizeof(Te) == 2) {
        Urm[i * k + kk] = __float2bfloat16_rn(v);
        if (Ucm) Ucm[e] = __float2bfloat16_rn(v);
    } else {
        Urm[i * k + kk] = v;
        if (Ucm) Ucm[e] = v;
    }
}

template <int AB>
cudaError_t launch_tc(const DevOperator<float>& op, int32_t s, int32_t k, float* w, int32_t nrhs, cudaStream_t st) {
    using Te = typename TcType<AB>::U;
    constexpr int E = TcType<AB>::E;
    const int np = (nrhs + 15) / 16 * 16;
    const int G = tc_blocks(s);
    const Te* Ucm = AB == 2 ? reinterpret_cast<const Te*>(op.U) : reinterpret_cast<const Te*>(op.U_tc_cm);
    const size_t sm1 = 2 * (128 + 64) * kTcKc * E + 64;
    // registers per thread for the chunk prefetch: as many as k and nrhs need
    auto vt = k <= 64 ? (np <= 32 ? k_lr_vt_tc<AB, 16, 8> : k_lr_vt_tc<AB, 16, 16>)
                      : (np <= 32 ? k_lr_vt_tc<AB, 32, 8> : k_lr_vt_tc<AB, 32, 16>);
    cudaError_t e = cudaFuncSetAttribute(vt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    vt<<<G, kTcThreads, sm1, st>>>(s, k, nrhs, np, Ucm, w, op.part, op.err);
    k_lr_fin_tc<<<dim3(k, (nrhs + kFinJ - 1) / kFinJ), kFinSeg * kFinJ, 0, st>>>(k, nrhs, G, op.part, op.dvec, op.vk);
    const int kp = AB == 2 ? (k + 7) / 8 * 8 : (k + 15) / 16 * 16;
    const size_t sm2 = (size_t)(128 + 64) * kp * E + 64;
    // the limit is process-wide state of the kernel: always the same (largest) value,
    // so concurrent launches for different k never race between setting and launching
    e = cudaFuncSetAttribute(k_lr_update_tc<AB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((128 + 64) * 128 * E + 64));
    if (e != cudaSuccess) return e;
    k_lr_update_tc<AB><<<(s + 127) / 128, kTcThreads, sm2, st>>>(s, k, kp, nrhs, np,
                                                                 reinterpret_cast<const Te*>(op.U_tc_rm), op.vk,
                                                                 op.cinv, w, op.err);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace

bool lowrank_tc_usable(const DevOperator<float>& op, int32_t k, int32_t nrhs) {
    return op.u_dtype != SLR_U_FP32 && op.U_tc_rm && nrhs >= 8 && nrhs <= 64 && k > 0 && k <= 128;
}

cudaError_t launch_lowrank_tc(const DevOperator<float>& op, int32_t s, int32_t k, float* w, int32_t nrhs,
                              cudaStream_t st) {
    if (s == 0) return cudaSuccess;
    return op.u_dtype == SLR_U_TF32 ? launch_tc<2>(op, s, k, w, nrhs, st) : launch_tc<1>(op, s, k, w, nrhs, st);
}

size_t lowrank_tc_elem(int32_t u_dtype) { return u_dtype == SLR_U_BF16 ? 2 : 4; }

cudaError_t launch_lowrank_tc_pack(int32_t u_dtype, int32_t s, int32_t k, const double* U, void* Urm, void* Ucm,
                                   cudaStream_t st) {
    const int64_t n = (int64_t)s * k;
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (u_dtype == SLR_U_BF16)
        k_lr_pack<__nv_bfloat16><<<blocks, 256, 0, st>>>(s, k, U, static_cast<__nv_bfloat16*>(Urm),
                                                          static_cast<__nv_bfloat16*>(Ucm));
    else
        k_lr_pack<float><<<blocks, 256, 0, st>>>(s, k, U, static_cast<float*>(Urm), nullptr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace slr
