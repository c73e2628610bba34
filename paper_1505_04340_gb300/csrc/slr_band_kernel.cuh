// The band-solve kernel K1 and its launch helpers, shared by the translation
// units that instantiate its 512- and 256-thread variants (slr_band.cu,
// slr_band_half.cu); the layout and pipeline are described in slr_band.cu.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "slr_device.h"

namespace cg = cooperative_groups;

namespace slr {

namespace {

constexpr int kMaxBuf = 8;         // ring slots at most
constexpr int kMinBuf = 2;         // ring slots at least
constexpr int kDefBuf = 2;         // ring slots unless the operator asks for another count
                                   // (two large slots measured fastest: per-chunk latency dominates)
constexpr int kMinSlot = 16 * 1024;   // bytes per ring slot at least
// Shared memory a CTA may use: the opt-in maximum for 512-thread CTAs (one per
// SM); for 256-thread CTAs, half an SM's 228 KB less its per-CTA reserve, so
// two CTAs (two subdomains) share each SM.
inline size_t band_cap(int nt) { return nt == 512 ? 227 * 1024 : 112 * 1024; }
constexpr int kRB = 8;             // row blocks of 32: at most 256 rows per slice
constexpr long long kSpin = 1ll << 24;   // bounded mbarrier wait (about a second)

// ---- slice geometry (the host packer uses the same rules: band_* in slr_internal.h)
// local row block with first plane row R0: columns it meets in an upper block
// start at seg_cU0, in a lower block end before seg_cL1
__device__ __forceinline__ int seg_cU0(int W, int R0) { return min(W, R0); }
__device__ __forceinline__ int seg_cL1(int W, int R0) { return min(W, min(R0 + 31, W - 1) + 1); }

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
// Wait with acquire at cluster scope: the bytes it waits for were stored by
// peers with st.async, whose complete_tx releases at cluster scope.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Address of the same shared-memory location in cluster CTA `rank`.
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// Store one value into another cluster CTA's shared memory; its bytes complete
// on that CTA's mbarrier `bar` (both addresses in the shared::cluster window, in
// the same CTA, which must not be the executing one).
__device__ __forceinline__ void st_async(uint32_t addr, float v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
                 "l"(__double_as_longlong(v)), "r"(bar)
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

// Column c of every block goes to warp c mod KW whatever the chunk boundaries,
// so each warp's partial sums, and the result, do not depend on the ring's
// slot size (which varies with the right-hand sides per CTA).
template <int KW>
__device__ __forceinline__ int first_col(int lo, int warp) { return lo + ((warp - lo % KW) + KW) % KW; }

struct Geom {
    int W, c, g;
    int nU, nL;
    int64_t base, PS, SU, SL;
};

// Block types: 0 O_J (upper, fwd), 1 D_J (lower, fwd), 2 O_J^T (lower, bwd), 3 D_J^T (upper, bwd).
// Stream order: forward D_0, (O_J, D_J) J = 1..c-1; backward D_{c-1}^T, then
// (O_{J+1}^T, D_J^T) J = c-2..0 (O_{J+1}^T is stored with plane J+1).
// next_block advances (type, plane) along that order; plane < 0 ends it.
__device__ __forceinline__ void next_block(int c, int& type, int& plane) {
    switch (type) {
        case 1: if (plane + 1 < c) { type = 0; ++plane; } else { type = 3; plane = c - 1; } break;
        case 0: type = 1; break;
        case 3: if (plane > 0) type = 2; else plane = -1; break;
        default: type = 3; --plane; break;
    }
}

__device__ __forceinline__ int64_t block_off(const Geom& q, int type) {
    return type == 0 ? 0 : type == 1 ? q.SU : type == 2 ? q.SU + q.SL : q.SU + 2 * q.SL;
}

}  // namespace

// NT threads per CTA: 512 (one CTA per SM, 4 warps per SM sub-partition to hide
// the load->FMA latency) or 256 (two CTAs, two subdomains, per SM).
template <typename T, int NR, int G, int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
k_band_solve2(const BandBlock* __restrict__ blocks, const T* __restrict__ fac, const T* in, int64_t ldi, T* out,
              int64_t ldo, const T* base, int64_t ldb, int32_t* err, int nbuf, int slot) {
    constexpr int kT = NT;         // threads per CTA
    constexpr int kW = NT / 32;    // warps per CTA
    extern __shared__ __align__(128) unsigned char smem[];
    const int sub = blockIdx.x / G;
    const int g = (G > 1) ? (int)cg::this_cluster().block_rank() : 0;
    const BandBlock b = blocks[sub];
    if (b.m == 0) return;                       // uniform across the cluster
    const int W = b.w, c = b.c, m = b.m;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- shared memory carve-up: barriers, tables and vectors, then the ring
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);              // [kMaxBuf]
    uint64_t* empty = full + kMaxBuf;                                 // [kMaxBuf]
    uint64_t* vbar = empty + kMaxBuf;                                 // [3] t (two buffers), y/x
    int* segU = reinterpret_cast<int*>(vbar + 4);                    // [kRB+1] first segment of row block rb
    int* segL = segU + (kRB + 1);                                    // [kRB+1]
    int* hdr = segL + (kRB + 1);                                     // nU, nL, segments per chunk, abort
    uintptr_t vp = reinterpret_cast<uintptr_t>(hdr + 4);
    vp = (vp + 15) & ~uintptr_t(15);
    T* vst = reinterpret_cast<T*>(vp);              // [NR][W] y_{J-1} (fwd) / x_{J+1} (bwd), whole plane
    T* vt = vst + NR * W;                           // [2][NR][W] t, whole plane, by phase parity
    T* part = vt + 2 * NR * W;                      // [kW][NR][256] per-warp partial sums
    uintptr_t rp = reinterpret_cast<uintptr_t>(part + kW * NR * 256);
    unsigned char* ring = reinterpret_cast<unsigned char*>((rp + 127) & ~uintptr_t(127));   // nbuf x slot bytes

    Geom q;
    q.W = W;
    q.c = c;
    q.g = g;
    q.SU = b.SU;
    q.SL = b.SL;
    q.PS = (int64_t)G * 2 * (b.SU + b.SL);
    q.base = b.foff + (int64_t)g * 2 * (b.SU + b.SL);

    // this slice's row blocks: first plane row of each (past W: none)
    const int nrb = b.nrb[g];
    int R0[kRB];
#pragma unroll
    for (int rb = 0; rb < kRB; ++rb) R0[rb] = rb < nrb ? 32 * b.rbmap[g][rb] : W;
    // Every row of a plane has one owner in the cluster.  A phase of a vector
    // barrier completes with 1 + nrb arrivals (thread 0 arming it, and each of
    // this slice's owner warps once its rows are stored here) and the bytes of
    // the other slices' rows, stored by their owners with st.async.
    int my_rows = 0;
#pragma unroll
    for (int rb = 0; rb < kRB; ++rb)
        if (rb < nrb) my_rows += min(32, W - R0[rb]);
    const uint32_t rbytes = (uint32_t)((W - my_rows) * NR * (int)sizeof(T));
    if (tid == 0) {
        int a = 0, d = 0;
        for (int rb = 0; rb <= kRB; ++rb) {
            segU[rb] = a;
            segL[rb] = d;
            if (rb < nrb) {
                a += W - seg_cU0(W, R0[rb]);
                d += seg_cL1(W, R0[rb]);
            }
        }
        const int per = max(1, slot / (32 * (int)sizeof(T)));   // whole segments per chunk
        hdr[0] = (a + per - 1) / per;
        hdr[1] = (d + per - 1) / per;
        hdr[2] = per;
        hdr[3] = 0;                                // set once a bounded wait of this CTA expires
        for (int i = 0; i < nbuf; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kW);
        }
        for (int i = 0; i < 3; ++i) mbar_init(&vbar[i], 1 + nrb);
        for (int i = 0; i < 3; ++i) {
            if (rbytes) mbar_arrive_expect_tx(&vbar[i], rbytes);
            else mbar_arrive(&vbar[i]);
        }
        fence_mbar_init();
    }
    __syncthreads();
    q.nU = hdr[0];
    q.nL = hdr[1];
    const int per = hdr[2];
    // forward: D_0 (lower), then (O_J upper, D_J lower); backward: D_{c-1}^T (upper), then (O^T lower, D^T upper)
    const int total = q.nL + q.nU + 2 * (c - 1) * (q.nU + q.nL);

    // first and one-past-last element of chunk ix of a block: segments [ix per, ...)
    auto chunk_src = [&](int type, int plane, int ix, int64_t& e0, int64_t& e1) {
        const bool up = (type == 0 || type == 3);
        const int nseg = up ? segU[kRB] : segL[kRB];
        e0 = q.base + (int64_t)plane * q.PS + block_off(q, type) + (int64_t)ix * per * 32;
        e1 = e0 + (int64_t)(min(per, nseg - ix * per)) * 32;
    };
    // thread 0 issues chunks in stream order; its cursor is the next chunk to issue
    int cur_type = 1, cur_plane = 0, cur_ix = 0, issued = 0;
    auto issue_next = [&]() {
        if (cur_plane < 0) return;                 // past the end of the stream: nothing to copy
        int64_t e0, e1;
        chunk_src(cur_type, cur_plane, cur_ix, e0, e1);
        // whole segments of 32 values: start and size are multiples of 128 bytes
        const uint32_t bytes = (uint32_t)((e1 - e0) * (int64_t)sizeof(T));
        const int sl = issued % nbuf;
        uint64_t* bar = &full[sl];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(ring + (size_t)sl * slot, fac + e0, bytes, bar);
        ++issued;
        const int nch = (cur_type == 0 || cur_type == 3) ? q.nU : q.nL;
        if (++cur_ix == nch) {
            cur_ix = 0;
            next_block(c, cur_type, cur_plane);
        }
    };
    // After a bounded wait expires the CTA aborts: the status word and the
    // CTA's abort flag (hdr[3]) are set, no further copy is issued, the block
    // products and the vector waits are skipped, and before it exits thread 0
    // waits for the copies it issued.
    volatile int* abort_flag = hdr + 3;
    auto wait_bar = [&](uint64_t* bar, uint32_t par) -> bool {
        long long it = 0;
        while (!mbar_try_wait(bar, par)) {
            if (++it > kSpin) {
                atomicExch(err, 1);
                *abort_flag = 1;
                return false;
            }
        }
        return true;
    };
    // chunk k's data has landed (the (k / nbuf)-th fill of its slot); false once the CTA
    // aborted.  The answer is the same for the whole warp (all lanes saw the data land).
    auto wait_full = [&](int k) -> bool {
        bool ok = !*abort_flag && wait_bar(&full[k % nbuf], (uint32_t)((k / nbuf) & 1));
        return __all_sync(0xffffffffu, ok);
    };
    // this warp is done with chunk k's slot (its release is ordered after a store
    // of the abort flag, so the refilling thread sees the flag once it has the slot)
    auto release = [&](int k) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[k % nbuf]);
    };
    // thread 0, before consuming chunk k: once every warp has released chunk
    // k - 1, its slot takes the next chunk of the stream (unless the CTA aborted:
    // a warp whose wait for chunk k - 1 expired may have left that copy in flight)
    auto refill = [&](int k) {
        if (tid == 0 && k >= 1 && issued < total && !*abort_flag) {
            if (wait_bar(&empty[(k - 1) % nbuf], (uint32_t)(((k - 1) / nbuf) & 1)) && !*abort_flag) {
                fence_proxy_async();
                issue_next();
            }
        }
    };
    // thread 0 at exit after an abort: the last copy issued into each slot has
    // landed (the fills of a slot are issued one after another, each once the
    // previous one was consumed, so the last one completing means all did)
    auto drain = [&]() {
        if (tid != 0 || !*abort_flag) return;
        for (int sl = 0; sl < nbuf && sl < issued; ++sl) {
            const int last = sl + ((issued - 1 - sl) / nbuf) * nbuf;
            long long it = 0;
            while (!mbar_try_wait(&full[sl], (uint32_t)((last / nbuf) & 1)) && ++it <= kSpin) {
            }
        }
    };
    // The plane vector of a phase reaches every CTA of the cluster: each owner
    // stores its rows into this CTA's copy (then its warp arrives on the local
    // vector barrier) and, by st.async, into every peer's copy, where the bytes
    // complete on the peer's vector barrier, armed by the peer's thread 0 with
    // the bytes it receives.  No cluster-wide barrier is taken per phase.  A CTA re-arms a barrier for
    // its next phase as soon as it has seen the current one complete: the next
    // phase's stores into it come only after the peers have received this CTA's
    // own next rows, which it sends after consuming the current phase.  For the
    // same reason the t vector has two buffers (by phase parity): the forward
    // pass's last t and the backward pass's first t have no exchange of y
    // between them, so a fast peer can send the second before a slow CTA has
    // read the first.  y/x needs one buffer (an exchange of t always lies between
    // two of its phases).  A wait that expires sets the abort flag; the barrier
    // is then left un-armed (thread 0 never arrives twice in one phase).
    auto wait_vec = [&](uint64_t* bar, uint32_t par) -> bool {
        bool ok = false;
        if (!*abort_flag) {
            long long it = 0;
            ok = true;
            while (!mbar_try_wait_cluster(bar, par)) {
                if (++it > kSpin) {
                    atomicExch(err, 1);
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
            }
            if (ok && tid == 0) {
                if (rbytes) mbar_arrive_expect_tx(bar, rbytes);
                else mbar_arrive(bar);
            }
        }
        return __all_sync(0xffffffffu, ok);
    };
    // owner rows of a phase into vector vec (element j W + own_r) of every CTA.
    // An aborted CTA sends nothing more: its peers' waits for its rows then
    // expire and they abort in turn, so at most a phase or two of bytes reach a
    // barrier this CTA no longer arms.
    auto send = [&](T* vec, uint64_t* bar, int j, int r, T v) {
        if (*abort_flag) return;
        vec[j * W + r] = v;
        if constexpr (G > 1) {
            const uint32_t a = smem_u32(vec + j * W + r), mb = smem_u32(bar);
#pragma unroll
            for (int pr = 0; pr < G; ++pr)
                if (pr != g) st_async(peer_addr(a, pr), v, peer_addr(mb, pr));
        }
    };
    // an owner warp, once all its rows of a phase are stored here (all of its lanes)
    auto arrive_local = [&](uint64_t* bar) {
        if (warp < nrb) {
            __syncwarp();
            if (lane == 0 && !*abort_flag) mbar_arrive(bar);
        }
    };

    if (tid == 0)
        while (issued < nbuf && issued < total) issue_next();
    // every CTA of the cluster has armed its barriers before any st.async reaches it
    cluster_barrier<G>();

    int k = 0;
    T acc[kRB][NR];
    // acc[rb][j] = sum over the block's segments of row block rb of seg[lane] * vin[j][column];
    // vin is complete once phase `par` of vector barrier `vb` has
    auto run_block = [&](int type, int plane, const T* vin, uint64_t* vb, uint32_t par) {
        const bool upper = (type == 0 || type == 3);
#pragma unroll
        for (int rb = 0; rb < kRB; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[rb][j] = T(0);
        const int nch = upper ? q.nU : q.nL;
        const int* seg = upper ? segU : segL;
        bool vok = true, waited = false;
        for (int ix = 0; ix < nch; ++ix, ++k) {
            refill(k);
            const bool landed = wait_full(k);
            if (!waited) {                 // the input vector (after the block's first data)
                vok = wait_vec(vb, par);
                waited = true;
            }
            if (!landed || !vok) {         // aborted: no product
                release(k);
                continue;
            }
            const int s0 = ix * per, s1 = min(s0 + per, seg[kRB]);
            const T* P = reinterpret_cast<const T*>(ring + (size_t)(k % nbuf) * slot);
#pragma unroll
            for (int rb = 0; rb < kRB; ++rb) {
                if (rb >= nrb) break;
                const int sa = max(s0, seg[rb]), sb = min(s1, seg[rb + 1]);
                if (sa >= sb) continue;
                const int cb0 = upper ? seg_cU0(W, R0[rb]) : 0;         // column of segment seg[rb]
                const int ca = cb0 + (sa - seg[rb]), ce = cb0 + (sb - seg[rb]);
                int cc = first_col<kW>(ca, warp);
                const T* Ps = P + (sa - s0 + (cc - ca)) * 32 + lane;
#pragma unroll 2
                for (; cc < ce; cc += kW, Ps += kW * 32) {
                    const T a = *Ps;
#pragma unroll
                    for (int j = 0; j < NR; ++j) acc[rb][j] = fma(a, vin[j * W + cc], acc[rb][j]);
                }
            }
            release(k);
        }
        if (!waited) wait_vec(vb, par);    // a block without chunks (a slice without rows)
#pragma unroll
        for (int rb = 0; rb < kRB; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) part[(warp * NR + j) * 256 + rb * 32 + lane] = acc[rb][j];
        __syncthreads();
    };
    // (the barrier first: owners may still be reading the previous phase's sums)
    auto zero_part = [&]() {
        __syncthreads();
        for (int i = tid; i < kW * NR * 256; i += kT) part[i] = T(0);
        __syncthreads();
    };
    auto part_sum = [&](int lr, int j) -> T {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < kW; ++w) s += part[(w * NR + j) * 256 + lr];
        return s;
    };

    // Each thread owns at most one output row per plane (a slice has at most
    // 256 rows): its right-hand side (forward) or forward result (backward) is
    // loaded before the block product so the load is off the plane-to-plane chain.
    int own_r = W;
#pragma unroll
    for (int rb = 0; rb < kRB; ++rb)
        if ((tid >> 5) == rb) own_r = R0[rb] + (tid & 31);
    const bool owner = tid < 32 * nrb && own_r < W;
    int ut = 0, uy = 0;        // phases of the t vector and of the y/x vector so far
    // =================================================================== forward
    for (int J = 0; J < c; ++J) {
        const int row = J * W + own_r;
        T pre[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) pre[j] = (owner && row < m) ? in[b.row0 + row + j * ldi] : T(0);
        if (J > 0) run_block(0, J, vst, &vbar[2], (uint32_t)(uy++ & 1));        // O_J y_{J-1}
        else zero_part();
        T* vtb = vt + (ut & 1) * NR * W;
        if (owner) {
#pragma unroll
            for (int j = 0; j < NR; ++j) send(vtb, &vbar[ut & 1], j, own_r, pre[j] - part_sum(tid, j));
        }
        arrive_local(&vbar[ut & 1]);
        run_block(1, J, vtb, &vbar[ut & 1], (uint32_t)((ut >> 1) & 1));        // D_J t
        ++ut;
        if (owner) {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const T y = part_sum(tid, j);
                if (row < m) out[b.row0 + row + j * ldo] = y;
                if (J + 1 < c) send(vst, &vbar[2], j, own_r, y);                 // read by O_{J+1}
            }
        }
        if (J + 1 < c) arrive_local(&vbar[2]);
    }
    // =================================================================== backward
    for (int J = c - 1; J >= 0; --J) {
        const int row = J * W + own_r;
        const int64_t gi = b.row0 + row;
        T pre[NR], bs[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            pre[j] = (owner && row < m) ? out[gi + j * ldo] : T(0);
            bs[j] = (owner && row < m && base) ? base[gi + j * ldb] : T(0);
        }
        if (J < c - 1) run_block(2, J + 1, vst, &vbar[2], (uint32_t)(uy++ & 1));   // O_{J+1}^T x_{J+1}
        else zero_part();
        T* vtb = vt + (ut & 1) * NR * W;
        if (owner) {
#pragma unroll
            for (int j = 0; j < NR; ++j) send(vtb, &vbar[ut & 1], j, own_r, pre[j] - part_sum(tid, j));
        }
        arrive_local(&vbar[ut & 1]);
        run_block(3, J, vtb, &vbar[ut & 1], (uint32_t)((ut >> 1) & 1));           // D_J^T t
        ++ut;
        if (owner) {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const T x = part_sum(tid, j);
                if (row < m) out[gi + j * ldo] = base ? bs[j] - x : x;
                if (J > 0) send(vst, &vbar[2], j, own_r, x);                      // read by O_J^T
            }
        }
        if (J > 0) arrive_local(&vbar[2]);
    }
    cluster_barrier<G>();    // no CTA leaves while a peer may still store into it
    drain();                 // nor with a bulk copy still writing its shared memory
}

// Shared memory besides the ring (barriers, column tables, vectors, partials,
// the ring's alignment), for planes of at most wmax rows.
inline size_t band_fixed_bytes(int32_t wmax, int32_t nr, size_t elem, int nt) {
    const size_t head = 2 * kMaxBuf * 8 + 4 * 8 + 2 * (kRB + 1) * 4 + 16 + 16;
    const size_t vec = (size_t)(3 * nr * wmax + (nt / 32) * nr * 256) * elem;
    return head + vec + 128;
}

// The ring of a CTA of nt threads: the slot count (nbuf_req, 0 for the default,
// clamped to what fits) and the bytes per slot that fill the shared memory left
// beside the tables and vectors; false if no ring fits.
inline bool band_ring(int32_t wmax, int32_t nr, size_t elem, int32_t nbuf_req, int nt, int32_t* nbuf, int32_t* slot) {
    const size_t fx = band_fixed_bytes(wmax, nr, elem, nt), cap = band_cap(nt);
    if (fx + (size_t)kMinBuf * kMinSlot > cap) return false;
    const size_t avail = cap - fx;
    int32_t n = nbuf_req > 0 ? nbuf_req : kDefBuf;
    n = std::max(kMinBuf, std::min<int32_t>(n, kMaxBuf));
    while (n > kMinBuf && avail / n < (size_t)kMinSlot) --n;
    *nbuf = n;
    *slot = (int32_t)((avail / n) & ~size_t(127));
    return true;
}

inline size_t band_smem_bytes(int32_t wmax, int32_t nr, size_t elem, int nt, int32_t nbuf, int32_t slot) {
    return band_fixed_bytes(wmax, nr, elem, nt) + (size_t)nbuf * slot;
}

namespace {
template <typename T, int NR, int G, int NT>
cudaError_t band_launch(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                        int64_t ldo, const T* base, int64_t ldb, cudaStream_t st) {
    auto kern = k_band_solve2<T, NR, G, NT>;
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
    int32_t nbuf = 0, slot = 0;
    if (!band_ring(wmax, NR, sizeof(T), op.band_nbuf, NT, &nbuf, &slot)) return cudaErrorInvalidValue;
    const size_t smem = band_smem_bytes(wmax, NR, sizeof(T), NT, nbuf, slot);
    cudaError_t e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p * G);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = G > 1 ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, kern, op.band, op.bfac, in, ldi, out, ldo, base, ldb, op.err, (int)nbuf, (int)slot);
    count_launches(1);
    return e;
}

template <typename T, int NR, int NT>
cudaError_t band_launch_g(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                          int64_t ldo, const T* base, int64_t ldb, cudaStream_t st) {
    switch (op.band_G) {
        case 2: return band_launch<T, NR, 2, NT>(op, p, wmax, in, ldi, out, ldo, base, ldb, st);
        case 4: return band_launch<T, NR, 4, NT>(op, p, wmax, in, ldi, out, ldo, base, ldb, st);
        default: return band_launch<T, NR, 1, NT>(op, p, wmax, in, ldi, out, ldo, base, ldb, st);
    }
}
}  // namespace

// The 256-thread variants (instantiated in their own translation unit).
template <typename T, int NR>
cudaError_t band_launch_half(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                             int64_t ldo, const T* base, int64_t ldb, cudaStream_t st);


}  // namespace slr
