// K1: batched banded solves t = B^{-1} f with B = diag(B_i) (Section 5.2),
// one subdomain per thread-block cluster of G CTAs, for sm_103a.
//
// Factor layout (built by host_band_factor): the Cholesky factor L_i is banded
// with half-bandwidth w; rows are grouped in planes of W rows.  For plane J
//   O_J = L_i[plane J, plane J-1]  upper triangular incl. diagonal,
//   D_J = L_i[plane J, plane J]^{-1} lower triangular incl. diagonal (inverted on the host).
// Rows r of a plane are dealt to cluster ranks g = r mod G ("slices"); slice g
// of each block is stored column-major and packed: column c of O holds the
// slice's rows r <= c, column q of D holds its rows r >= q.  Plane stride is
// G (SO + SD) elements: slice g's O block at g (SO + SD), its D block SO later.
//
//   forward  (L y = f):    t_J = f_J - O_J y_{J-1};       y_J = D_J t_J
//   backward (L^T x = y):  t_J = y_J - O_{J+1}^T x_{J+1};  x_J = D_J^T t_J
//
// Each CTA streams the blocks of its slice through a ring of NBUF shared
// buffers with 1-D bulk asynchronous copies completed on mbarriers (one
// thread issues, everyone waits with a bounded spin).  Forward phases use
// lanes = rows, warps = columns round-robin; backward phases use one warp per
// column.  Vectors move between the CTAs of a cluster through distributed
// shared memory, ordered by cluster barriers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "slr_device.h"

namespace cg = cooperative_groups;

namespace slr {

extern std::atomic<int64_t> g_kernel_launches;

namespace {

constexpr int kT = 256;            // threads per CTA
constexpr int kW = kT / 32;        // warps per CTA
constexpr int kNBuf = 3;           // ring slots
constexpr int kChunk = 48 * 1024;  // bytes per ring slot
constexpr int kMaxCh = 64;         // chunks per block
constexpr int kRB = 8;             // row blocks of 32: at most 256 rows per slice
constexpr long long kSpin = 1ll << 24;   // bounded mbarrier wait (about a second)

// ---- slice geometry (the host packer uses the same rules: band_* in slr_internal.h)
__device__ __forceinline__ int slice_rows(int W, int G, int g) { return g < W ? (W - 1 - g) / G + 1 : 0; }
__device__ __forceinline__ int cnt_O(int c, int G, int g) { return c >= g ? (c - g) / G + 1 : 0; }
__device__ __forceinline__ int lr0_D(int q, int G, int g) { return q <= g ? 0 : (q - g + G - 1) / G; }

// ---- mbarrier / bulk copy PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T warp_sum_band(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ void cluster_barrier() {
    if constexpr (G > 1) {
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

struct Geom {
    int W, c, g, nrg;
    int nO, nD;
    int64_t base, PS, SO;
};

// Position of chunk k in the stream: forward  D_0, (O_J, D_J) J = 1..c-1,
// then backward D_{c-1}, (O_{J+1}, D_J) J = c-2..0.  part: 0 = O, 1 = D.
__device__ __forceinline__ void chunk_pos(const Geom& q, int k, int& part, int& plane, int& idx) {
    const int per = q.nO + q.nD, fwd = q.nD + (q.c - 1) * per;
    int kk = k < fwd ? k : k - fwd;
    if (kk < q.nD) {
        part = 1;
        plane = k < fwd ? 0 : q.c - 1;
        idx = kk;
        return;
    }
    kk -= q.nD;
    const int pr = kk / per, r = kk % per;
    if (k < fwd) {
        plane = 1 + pr;
        part = r < q.nO ? 0 : 1;
        idx = r < q.nO ? r : r - q.nO;
    } else {
        part = r < q.nO ? 0 : 1;
        plane = r < q.nO ? q.c - 1 - pr : q.c - 2 - pr;
        idx = r < q.nO ? r : r - q.nO;
    }
}

}  // namespace

template <typename T, int NR, int G>
__global__ void __launch_bounds__(kT, 1)
k_band_solve2(const BandBlock* __restrict__ blocks, const T* __restrict__ fac, const T* in, int64_t ldi, T* out,
              int64_t ldo, const T* base, int64_t ldb, int32_t* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int sub = blockIdx.x / G;
    const int g = (G > 1) ? (int)cg::this_cluster().block_rank() : 0;
    const BandBlock b = blocks[sub];
    if (b.m == 0) return;                       // uniform across the cluster
    const int W = b.w, c = b.c, m = b.m;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- shared memory carve-up
    unsigned char* ring = smem;                                     // kNBuf x kChunk
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kNBuf * kChunk);
    int* colO = reinterpret_cast<int*>(full + kNBuf);              // [W+1]
    int* colD = colO + (W + 1);                                    // [W+1]
    int* chO = colD + (W + 1);                                     // [kMaxCh+1]
    int* chD = chO + (kMaxCh + 1);                                 // [kMaxCh+1]
    int* hdr = chD + (kMaxCh + 1);                                 // nO, nD
    uintptr_t vp = reinterpret_cast<uintptr_t>(hdr + 4);
    vp = (vp + 15) & ~uintptr_t(15);
    T* yfull = reinterpret_cast<T*>(vp);            // [NR][W]  y_{J-1} (forward)
    T* tfull = yfull + NR * W;                      // [NR][W]  t_J (forward)
    T* part = tfull + NR * W;                       // [kW][NR][256] per-warp partial sums
    T* recvA = part + kW * NR * 256;                // [G][NR][W]
    T* recvB = recvA + G * NR * W;                  // [2][G][NR][W]
    T* xown = recvB + 2 * G * NR * W;               // [NR][256]
    T* town = xown + NR * 256;                      // [NR][256]

    Geom q;
    q.W = W;
    q.c = c;
    q.g = g;
    q.nrg = slice_rows(W, G, g);
    q.PS = (int64_t)G * (b.SO + b.SD);
    q.SO = b.SO;
    q.base = b.foff + (int64_t)g * (b.SO + b.SD);

    if (tid == 0) {
        int a = 0, d = 0;
        for (int cc = 0; cc < W; ++cc) {
            colO[cc] = a;
            colD[cc] = d;
            a += cnt_O(cc, G, g);
            d += q.nrg - min(q.nrg, lr0_D(cc, G, g));
        }
        colO[W] = a;
        colD[W] = d;
        // greedy column chunks of at most kChunk - 32 bytes (room for 16-byte alignment)
        const int budget = (kChunk - 32) / (int)sizeof(T);
        int n = 0, acc = 0;
        chO[0] = 0;
        for (int cc = 0; cc < W; ++cc) {
            const int e = colO[cc + 1] - colO[cc];
            if (acc > 0 && acc + e > budget) { chO[++n] = cc; acc = 0; }
            acc += e;
        }
        chO[++n] = W;
        hdr[0] = n;
        n = 0;
        acc = 0;
        chD[0] = 0;
        for (int cc = 0; cc < W; ++cc) {
            const int e = colD[cc + 1] - colD[cc];
            if (acc > 0 && acc + e > budget) { chD[++n] = cc; acc = 0; }
            acc += e;
        }
        chD[++n] = W;
        hdr[1] = n;
        for (int i = 0; i < kNBuf; ++i) mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    q.nO = hdr[0];
    q.nD = hdr[1];
    const int total = 2 * (q.nD + (c - 1) * (q.nO + q.nD));

    // chunk k -> (source, bytes, element shift) ; issued by thread 0 only
    auto issue = [&](int k) {
        int pt, pl, ix;
        chunk_pos(q, k, pt, pl, ix);
        const int* col = pt ? colD : colO;
        const int* ch = pt ? chD : chO;
        const int64_t e0 = q.base + (int64_t)pl * q.PS + (pt ? q.SO : 0) + col[ch[ix]];
        const int64_t e1 = e0 + (col[ch[ix + 1]] - col[ch[ix]]);
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(fac + e0), a1 = reinterpret_cast<uintptr_t>(fac + e1);
        const uintptr_t al0 = a0 & ~uintptr_t(15), al1 = (a1 + 15) & ~uintptr_t(15);
        uint64_t* bar = &full[k % kNBuf];
        if (al1 > al0) {
            mbar_arrive_expect_tx(bar, (uint32_t)(al1 - al0));
            bulk_g2s(ring + (k % kNBuf) * kChunk, reinterpret_cast<const void*>(al0), (uint32_t)(al1 - al0), bar);
        } else {
            mbar_arrive(bar);
        }
    };
    // consumer view of chunk k: pointer p with p[col[cc] + local] = element
    auto view = [&](int k, int pt, int ix) -> const T* {
        int ptc, pl, ixc;
        chunk_pos(q, k, ptc, pl, ixc);
        const int* col = pt ? colD : colO;
        const int* ch = pt ? chD : chO;
        const int64_t e0 = q.base + (int64_t)pl * q.PS + (pt ? q.SO : 0) + col[ch[ix]];
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(fac + e0);
        const int shift = (int)((a0 & 15) / sizeof(T));
        return reinterpret_cast<const T*>(ring + (k % kNBuf) * kChunk) + shift - col[ch[ix]];
    };
    auto wait_full = [&](int k) {
        uint64_t* bar = &full[k % kNBuf];
        const uint32_t par = (uint32_t)((k / kNBuf) & 1);
        long long it = 0;
        while (!mbar_try_wait(bar, par)) {
            if (++it > kSpin) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
        }
    };
    auto release = [&](int k) {   // everyone is done with chunk k's slot: refill it
        __syncthreads();
        if (tid == 0 && k + kNBuf < total) {
            fence_proxy_async();
            issue(k + kNBuf);
        }
    };

    if (tid == 0)
        for (int k = 0; k < kNBuf && k < total; ++k) issue(k);
    // every CTA of the cluster is running before anyone stores into a peer's shared memory
    cluster_barrier<G>();

    auto peer = [&](T* p, int r) -> T* {
        if constexpr (G > 1) return cg::this_cluster().map_shared_rank(p, r);
        return p;
    };

    int k = 0;
    T acc[kRB][NR];
    // =================================================================== forward
    for (int J = 0; J < c; ++J) {
        // ---- t_J = f_J - O_J y_{J-1}: lanes = rows, warps take columns round-robin
#pragma unroll
        for (int rb = 0; rb < kRB; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[rb][j] = T(0);
        if (J > 0) {
            for (int ix = 0; ix < q.nO; ++ix, ++k) {
                wait_full(k);
                const T* P = view(k, 0, ix);
                for (int cc = chO[ix] + warp; cc < chO[ix + 1]; cc += kW) {
                    const int n = cnt_O(cc, G, g);
                    const T* Pc = P + colO[cc];
                    T yv[NR];
#pragma unroll
                    for (int j = 0; j < NR; ++j) yv[j] = yfull[j * W + cc];
#pragma unroll
                    for (int rb = 0; rb < kRB; ++rb) {
                        const int lr = rb * 32 + lane;
                        if (rb * 32 < n && lr < n) {
                            const T a = Pc[lr];
#pragma unroll
                            for (int j = 0; j < NR; ++j) acc[rb][j] += a * yv[j];
                        }
                    }
                }
                release(k);
            }
        }
#pragma unroll
        for (int rb = 0; rb < kRB; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) part[(warp * NR + j) * 256 + rb * 32 + lane] = acc[rb][j];
        __syncthreads();
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                T s = T(0);
#pragma unroll
                for (int w = 0; w < kW; ++w) s += part[(w * NR + j) * 256 + lr];
                const T f = row < m ? in[b.row0 + row + j * ldi] : T(0);
                const T t = f - s;
#pragma unroll
                for (int pr = 0; pr < G; ++pr) peer(tfull, pr)[j * W + r] = t;
            }
        }
        cluster_barrier<G>();
        // ---- y_J = D_J t_J
#pragma unroll
        for (int rb = 0; rb < kRB; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[rb][j] = T(0);
        for (int ix = 0; ix < q.nD; ++ix, ++k) {
            wait_full(k);
            const T* P = view(k, 1, ix);
            for (int cc = chD[ix] + warp; cc < chD[ix + 1]; cc += kW) {
                const int l0 = min(q.nrg, lr0_D(cc, G, g));
                const T* Pc = P + colD[cc] - l0;
                T tv[NR];
#pragma unroll
                for (int j = 0; j < NR; ++j) tv[j] = tfull[j * W + cc];
#pragma unroll
                for (int rb = 0; rb < kRB; ++rb) {
                    const int lr = rb * 32 + lane;
                    if (rb * 32 + 31 >= l0 && rb * 32 < q.nrg && lr >= l0 && lr < q.nrg) {
                        const T a = Pc[lr];
#pragma unroll
                        for (int j = 0; j < NR; ++j) acc[rb][j] += a * tv[j];
                    }
                }
            }
            release(k);
        }
#pragma unroll
        for (int rb = 0; rb < kRB; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) part[(warp * NR + j) * 256 + rb * 32 + lane] = acc[rb][j];
        __syncthreads();
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                T s = T(0);
#pragma unroll
                for (int w = 0; w < kW; ++w) s += part[(w * NR + j) * 256 + lr];
                if (row < m) out[b.row0 + row + j * ldo] = s;
#pragma unroll
                for (int pr = 0; pr < G; ++pr) peer(yfull, pr)[j * W + r] = s;
            }
        }
        cluster_barrier<G>();
    }
    // =================================================================== backward
    for (int J = c - 1; J >= 0; --J) {
        const int par = J & 1;
        // ---- column partials of O_{J+1}^T x_{J+1} over this slice's rows
        if (J < c - 1) {
            for (int ix = 0; ix < q.nO; ++ix, ++k) {
                wait_full(k);
                const T* P = view(k, 0, ix);
                for (int cc = chO[ix] + warp; cc < chO[ix + 1]; cc += kW) {
                    const int n = cnt_O(cc, G, g);
                    const T* Pc = P + colO[cc];
                    T s[NR];
#pragma unroll
                    for (int j = 0; j < NR; ++j) s[j] = T(0);
                    for (int lr = lane; lr < n; lr += 32) {
                        const T a = Pc[lr];
#pragma unroll
                        for (int j = 0; j < NR; ++j) s[j] += a * xown[j * 256 + lr];
                    }
#pragma unroll
                    for (int j = 0; j < NR; ++j) s[j] = warp_sum_band(s[j]);
                    if (lane < G) {
#pragma unroll
                        for (int j = 0; j < NR; ++j) peer(recvA, lane)[(g * NR + j) * W + cc] = s[j];
                    }
                }
                release(k);
            }
        }
        cluster_barrier<G>();
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                T s = T(0);
                if (J < c - 1) {
#pragma unroll
                    for (int pr = 0; pr < G; ++pr) s += recvA[(pr * NR + j) * W + r];
                }
                const T y = row < m ? out[b.row0 + row + j * ldo] : T(0);
                town[j * 256 + lr] = y - s;
            }
        }
        __syncthreads();
        // ---- column partials of D_J^T t_J
        T* rB = recvB + par * G * NR * W;
        for (int ix = 0; ix < q.nD; ++ix, ++k) {
            wait_full(k);
            const T* P = view(k, 1, ix);
            for (int cc = chD[ix] + warp; cc < chD[ix + 1]; cc += kW) {
                const int l0 = min(q.nrg, lr0_D(cc, G, g));
                const T* Pc = P + colD[cc] - l0;
                T s[NR];
#pragma unroll
                for (int j = 0; j < NR; ++j) s[j] = T(0);
                for (int lr = l0 + lane; lr < q.nrg; lr += 32) {
                    const T a = Pc[lr];
#pragma unroll
                    for (int j = 0; j < NR; ++j) s[j] += a * town[j * 256 + lr];
                }
#pragma unroll
                for (int j = 0; j < NR; ++j) s[j] = warp_sum_band(s[j]);
                if (lane < G) {
#pragma unroll
                    for (int j = 0; j < NR; ++j) peer(rB, lane)[(g * NR + j) * W + cc] = s[j];
                }
            }
            release(k);
        }
        cluster_barrier<G>();
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                T x = T(0);
#pragma unroll
                for (int pr = 0; pr < G; ++pr) x += rB[(pr * NR + j) * W + r];
                xown[j * 256 + lr] = x;
                if (row < m) {
                    const int64_t gi = b.row0 + row;
                    out[gi + j * ldo] = base ? base[gi + j * ldb] - x : x;
                }
            }
        }
        __syncthreads();
    }
}

size_t band_smem_bytes(int32_t wmax, int32_t G, int32_t nr, size_t elem) {
    size_t fixed = (size_t)kNBuf * kChunk + kNBuf * 8 + 2 * (wmax + 1) * 4 + 2 * (kMaxCh + 1) * 4 + 16 + 16;
    size_t vec = (size_t)(2 * nr * wmax + kW * nr * 256 + G * nr * wmax + 2 * G * nr * wmax + 2 * nr * 256) * elem;
    return fixed + vec;
}

namespace {
template <typename T, int NR, int G>
cudaError_t band_launch(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                        int64_t ldo, const T* base, int64_t ldb, cudaStream_t st) {
    const size_t smem = band_smem_bytes(wmax, G, NR, sizeof(T));
    auto kern = k_band_solve2<T, NR, G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p * G);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = G > 1 ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, kern, op.band, op.bfac, in, ldi, out, ldo, base, ldb, op.err);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename T, int NR>
cudaError_t band_launch_g(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                          int64_t ldo, const T* base, int64_t ldb, cudaStream_t st) {
    switch (op.band_G) {
        case 2: return band_launch<T, NR, 2>(op, p, wmax, in, ldi, out, ldo, base, ldb, st);
        case 4: return band_launch<T, NR, 4>(op, p, wmax, in, ldi, out, ldo, base, ldb, st);
        default: return band_launch<T, NR, 1>(op, p, wmax, in, ldi, out, ldo, base, ldb, st);
    }
}
}  // namespace

template <typename T>
cudaError_t launch_band_solve(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                              int64_t ldo, const T* base, int64_t ldb, int32_t nrhs, cudaStream_t st) {
    if (p == 0 || wmax == 0) return cudaSuccess;
    const size_t cap = 227 * 1024;
    for (int32_t c = 0; c < nrhs;) {
        const int32_t left = nrhs - c;
        int nr = 1;
        if (left >= 4 && band_smem_bytes(wmax, op.band_G, 4, sizeof(T)) <= cap) nr = 4;
        else if (left >= 2 && band_smem_bytes(wmax, op.band_G, 2, sizeof(T)) <= cap) nr = 2;
        const T* bs = base ? base + c * ldb : nullptr;
        cudaError_t e;
        if (nr == 4) e = band_launch_g<T, 4>(op, p, wmax, in + c * ldi, ldi, out + c * ldo, ldo, bs, ldb, st);
        else if (nr == 2) e = band_launch_g<T, 2>(op, p, wmax, in + c * ldi, ldi, out + c * ldo, ldo, bs, ldb, st);
        else e = band_launch_g<T, 1>(op, p, wmax, in + c * ldi, ldi, out + c * ldo, ldo, bs, ldb, st);
        if (e != cudaSuccess) return e;
        c += nr;
    }
    return cudaSuccess;
}

template cudaError_t launch_band_solve<double>(const DevOperator<double>&, int32_t, int32_t, const double*, int64_t,
                                               double*, int64_t, const double*, int64_t, int32_t, cudaStream_t);
template cudaError_t launch_band_solve<float>(const DevOperator<float>&, int32_t, int32_t, const float*, int64_t,
                                              float*, int64_t, const float*, int64_t, int32_t, cudaStream_t);

}  // namespace slr
