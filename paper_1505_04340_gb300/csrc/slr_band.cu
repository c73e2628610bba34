// K1: batched banded solves t = B^{-1} f with B = diag(B_i) (Section 5.2),
// one subdomain per thread-block cluster of G CTAs, for sm_103a.
//
// Factor layout (built by host_band_factor): the Cholesky factor L_i is banded
// with half-bandwidth w; rows are grouped in planes of W rows.  For plane J
//   O_J = L_i[plane J, plane J-1]    upper triangular incl. diagonal,
//   D_J = L_i[plane J, plane J]^{-1} lower triangular incl. diagonal (inverted on the host),
//   forward  (L y = f):    t = f_J - O_J y_{J-1};          y_J = D_J t
//   backward (L^T x = y):  t = y_J - O_{J+1}^T x_{J+1};    x_J = D_J^T t
// All four products are "output row = sum over columns" of a triangular
// matrix (O_J, D_J^T upper; D_J, O_J^T lower), each stored on its own.  Output
// rows are dealt to the G CTAs of a cluster (r mod G = rank); each CTA's
// slice of a block is packed column-major (column c: its rows r <= c for an
// upper block, r >= c for a lower one), so a CTA streams exactly its bytes.
//
// Each CTA streams its slices through a ring of kNBuf shared buffers with 1-D
// bulk asynchronous copies completed on mbarriers (one thread issues,
// everyone waits with a bounded spin that sets a device status word instead of
// hanging).  Lanes own output rows, warps take columns round-robin, and the
// per-warp partial sums are added once per phase.  The full input vector of a
// phase is assembled in every CTA through distributed shared memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "slr_device.h"

namespace cg = cooperative_groups;

namespace slr {

namespace {

constexpr int kT = 512;            // threads per CTA (4 warps per SM sub-partition hide the load->FMA latency)
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
    int nU, nL;
    int64_t base, PS, SU, SL;
};

// Block types: 0 O_J (upper, fwd), 1 D_J (lower, fwd), 2 O_J^T (lower, bwd), 3 D_J^T (upper, bwd).
// Stream: forward D_0, (O_J, D_J) J = 1..c-1; backward D_{c-1}^T, (O_{J+1}^T, D_J^T) J = c-2..0.
__device__ __forceinline__ void chunk_pos(const Geom& q, int k, int& type, int& plane, int& idx) {
    const int per = q.nU + q.nL, half = q.nL + (q.c - 1) * per;
    if (k < half) {
        if (k < q.nL) { type = 1; plane = 0; idx = k; return; }
        const int kk = k - q.nL, pr = kk / per, r = kk % per;
        plane = 1 + pr;
        if (r < q.nU) { type = 0; idx = r; } else { type = 1; idx = r - q.nU; }
        return;
    }
    const int k2 = k - half;
    if (k2 < q.nU) { type = 3; plane = q.c - 1; idx = k2; return; }
    const int kk = k2 - q.nU, pr = kk / per, r = kk % per;
    if (r < q.nL) { type = 2; plane = q.c - 1 - pr; idx = r; } else { type = 3; plane = q.c - 2 - pr; idx = r - q.nL; }
}

__device__ __forceinline__ int64_t block_off(const Geom& q, int type) {
    return type == 0 ? 0 : type == 1 ? q.SU : type == 2 ? q.SU + q.SL : q.SU + 2 * q.SL;
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
    int* colU = reinterpret_cast<int*>(full + kNBuf);              // [W+1]
    int* colL = colU + (W + 1);                                    // [W+1]
    int* chU = colL + (W + 1);                                     // [kMaxCh+1]
    int* chL = chU + (kMaxCh + 1);                                 // [kMaxCh+1]
    int* hdr = chL + (kMaxCh + 1);                                 // nU, nL
    uintptr_t vp = reinterpret_cast<uintptr_t>(hdr + 4);
    vp = (vp + 15) & ~uintptr_t(15);
    T* vst = reinterpret_cast<T*>(vp);              // [NR][W] y_{J-1} (fwd) / x_{J+1} (bwd), whole plane
    T* vt = vst + NR * W;                           // [NR][W] t, whole plane
    T* part = vt + NR * W;                          // [kW][NR][256] per-warp partial sums

    Geom q;
    q.W = W;
    q.c = c;
    q.g = g;
    q.nrg = slice_rows(W, G, g);
    q.SU = b.SU;
    q.SL = b.SL;
    q.PS = (int64_t)G * 2 * (b.SU + b.SL);
    q.base = b.foff + (int64_t)g * 2 * (b.SU + b.SL);

    if (tid == 0) {
        int a = 0, d = 0;
        for (int cc = 0; cc < W; ++cc) {
            colU[cc] = a;
            colL[cc] = d;
            a += cnt_O(cc, G, g);
            d += q.nrg - min(q.nrg, lr0_D(cc, G, g));
        }
        colU[W] = a;
        colL[W] = d;
        // greedy column chunks of at most kChunk - 32 bytes (room for 16-byte alignment)
        const int budget = (kChunk - 32) / (int)sizeof(T);
        for (int t = 0; t < 2; ++t) {
            const int* col = t ? colL : colU;
            int* ch = t ? chL : chU;
            int n = 0, acc = 0;
            ch[0] = 0;
            for (int cc = 0; cc < W; ++cc) {
                const int e = col[cc + 1] - col[cc];
                if (acc > 0 && acc + e > budget) { ch[++n] = cc; acc = 0; }
                acc += e;
            }
            ch[++n] = W;
            hdr[t] = n;
        }
        for (int i = 0; i < kNBuf; ++i) mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    q.nU = hdr[0];
    q.nL = hdr[1];
    const int total = 2 * (q.nL + (c - 1) * (q.nU + q.nL));

    auto src_of = [&](int k, int& type, int& ix, int64_t& e0, int64_t& e1) {
        int pl;
        chunk_pos(q, k, type, pl, ix);
        const bool up = (type == 0 || type == 3);
        const int* col = up ? colU : colL;
        const int* ch = up ? chU : chL;
        e0 = q.base + (int64_t)pl * q.PS + block_off(q, type) + col[ch[ix]];
        e1 = e0 + (col[ch[ix + 1]] - col[ch[ix]]);
    };
    auto issue = [&](int k) {   // thread 0 only
        int type, ix;
        int64_t e0, e1;
        src_of(k, type, ix, e0, e1);
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
    auto peer = [&](T* p, int r) -> T* {
        if constexpr (G > 1) return cg::this_cluster().map_shared_rank(p, r);
        return p;
    };

    if (tid == 0)
        for (int k = 0; k < kNBuf && k < total; ++k) issue(k);
    // every CTA of the cluster is running before anyone stores into a peer's shared memory
    cluster_barrier<G>();

    int k = 0;
    T acc[kRB][NR];
    // acc[rb][j] += sum over the chunks of one block of M[lr][cc] * vin[j][cc], lanes = rows
    auto run_block = [&](bool upper, const T* vin) {
#pragma unroll
        for (int rb = 0; rb < kRB; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[rb][j] = T(0);
        const int nch = upper ? q.nU : q.nL;
        const int* col = upper ? colU : colL;
        const int* ch = upper ? chU : chL;
        for (int ix = 0; ix < nch; ++ix, ++k) {
            wait_full(k);
            int type, ixx;
            int64_t e0, e1;
            src_of(k, type, ixx, e0, e1);
            const int shift = (int)((reinterpret_cast<uintptr_t>(fac + e0) & 15) / sizeof(T));
            const T* P = reinterpret_cast<const T*>(ring + (k % kNBuf) * kChunk) + shift - col[ch[ix]];
            const int ca = ch[ix], cb = ch[ix + 1];
            if constexpr (sizeof(T) == 8) {
                // FP64: row block outer.  Row block rb (own rows 32 rb .. 32 rb + 31)
                // meets column cc of an upper block iff cc >= G (32 rb) + g; a lower
                // block holds rows >= lr0(cc), so rb meets columns cc <= G (32 rb + 31) + g.
                // Separate loops per rb keep every DFMA unpredicated (an if-converted
                // rb loop would issue all kRB of them per column on the slow FP64 pipe,
                // which serves each SM sub-partition at a fixed rate).
#pragma unroll
                for (int rb = 0; rb < kRB; ++rb) {
                    if (rb * 32 >= q.nrg) break;
                    const int lr = rb * 32 + lane;
                    const int c0 = max(ca, upper ? G * (rb * 32) + g : ca);
                    const int c1 = upper ? cb : min(cb, G * (rb * 32 + 31) + g + 1);
                    int cc = ca + warp + ((c0 > ca + warp) ? ((c0 - ca - warp + kW - 1) / kW) * kW : 0);
                    auto term = [&](int c) {
                        const int lo = upper ? 0 : min(q.nrg, lr0_D(c, G, g));
                        const int hi = upper ? cnt_O(c, G, g) : q.nrg;
                        const T a = (lr >= lo && lr < hi) ? P[col[c] - lo + lr] : T(0);
#pragma unroll
                        for (int j = 0; j < NR; ++j) acc[rb][j] = fma(a, vin[j * W + c], acc[rb][j]);
                    };
                    for (; cc + kW < c1; cc += 2 * kW) {
                        term(cc);
                        term(cc + kW);
                    }
                    if (cc < c1) term(cc);
                }
            } else {
                // FP32: column outer, row blocks inner (the FP32 pipe absorbs the
                // predicated-off lanes; this order issues the fewest instructions)
                for (int cc = ca + warp; cc < cb; cc += kW) {
                    const int lo = upper ? 0 : min(q.nrg, lr0_D(cc, G, g));
                    const int hi = upper ? cnt_O(cc, G, g) : q.nrg;
                    const T* Pc = P + col[cc] - lo;
                    T v[NR];
#pragma unroll
                    for (int j = 0; j < NR; ++j) v[j] = vin[j * W + cc];
#pragma unroll
                    for (int rb = 0; rb < kRB; ++rb) {
                        if (rb * 32 + 32 > lo && rb * 32 < hi) {
                            const int lr = rb * 32 + lane;
                            if (lr >= lo && lr < hi) {
                                const T a = Pc[lr];
#pragma unroll
                                for (int j = 0; j < NR; ++j) acc[rb][j] += a * v[j];
                            }
                        }
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
    };
    auto zero_part = [&]() {
        for (int i = tid; i < kW * NR * 256; i += kT) part[i] = T(0);
        __syncthreads();
    };
    auto part_sum = [&](int lr, int j) -> T {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < kW; ++w) s += part[(w * NR + j) * 256 + lr];
        return s;
    };

    // =================================================================== forward
    for (int J = 0; J < c; ++J) {
        if (J > 0) run_block(true, vst); else zero_part();                 // O_J y_{J-1}
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const T f = row < m ? in[b.row0 + row + j * ldi] : T(0);
                const T t = f - part_sum(lr, j);
#pragma unroll
                for (int pr = 0; pr < G; ++pr) peer(vt, pr)[j * W + r] = t;
            }
        }
        cluster_barrier<G>();
        run_block(false, vt);                                              // D_J t
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const T y = part_sum(lr, j);
                if (row < m) out[b.row0 + row + j * ldo] = y;
#pragma unroll
                for (int pr = 0; pr < G; ++pr) peer(vst, pr)[j * W + r] = y;
            }
        }
        cluster_barrier<G>();
    }
    // =================================================================== backward
    for (int J = c - 1; J >= 0; --J) {
        if (J < c - 1) run_block(false, vst); else zero_part();            // O_{J+1}^T x_{J+1}
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const T y = row < m ? out[b.row0 + row + j * ldo] : T(0);
                const T t = y - part_sum(lr, j);
#pragma unroll
                for (int pr = 0; pr < G; ++pr) peer(vt, pr)[j * W + r] = t;
            }
        }
        cluster_barrier<G>();
        run_block(true, vt);                                               // D_J^T t
        for (int lr = tid; lr < q.nrg; lr += kT) {
            const int r = lr * G + g, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const T x = part_sum(lr, j);
                if (row < m) {
                    const int64_t gi = b.row0 + row;
                    out[gi + j * ldo] = base ? base[gi + j * ldb] - x : x;
                }
#pragma unroll
                for (int pr = 0; pr < G; ++pr) peer(vst, pr)[j * W + r] = x;
            }
        }
        cluster_barrier<G>();
    }
}

size_t band_smem_bytes(int32_t wmax, int32_t G, int32_t nr, size_t elem) {
    (void)G;
    size_t fixed = (size_t)kNBuf * kChunk + kNBuf * 8 + 2 * (wmax + 1) * 4 + 2 * (kMaxCh + 1) * 4 + 16 + 16;
    size_t vec = (size_t)(2 * nr * wmax + kW * nr * 256) * elem;
    return fixed + vec;
}

namespace {
template <typename T, int NR, int G>
cudaError_t band_launch(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                        int64_t ldo, const T* base, int64_t ldb, cudaStream_t st) {
    const size_t smem = band_smem_bytes(wmax, G, NR, sizeof(T));
    auto kern = k_band_solve2<T, NR, G>;
    // The dynamic shared-memory limit of a kernel is process-wide state on its
    // device.  It is raised once, to the device's opt-in maximum, so that
    // threads launching this kernel for operators of different widths never
    // race between one thread's setting and another's launch.
    static std::mutex mu;
    static uint64_t raised = 0;                     // bit d: done on device d
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu);
        if (!(raised >> dev & 1)) {
            int optin = 0;
            e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            if (e != cudaSuccess) return e;
            raised |= 1ull << dev;
        }
    }
    cudaError_t e;
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
    count_launches(1);
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
