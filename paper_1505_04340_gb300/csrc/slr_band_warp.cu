// K1 for narrow planes (W <= 64, the 2-D workloads): one warp per subdomain.
//
// With one slice per subdomain the factor layout is the one slr_band.cu describes:
// row blocks 0 and 1 (rows 32 rb .. 32 rb + 31), and per block of a plane the
// segments of 32 values (one per row) of every column that meets the triangle, row
// blocks one after the other, columns ascending.  A lane owns rows R0 + lane of the
// (at most two) row blocks and the warp walks every segment of a block in stream
// order, one multiply-add per segment, row and right-hand side.  A plane step thus
// needs no cross-warp sum and no CTA barrier: the plane vectors live in the warp's
// shared buffer, stored by their owners and read back by broadcast after
// __syncwarp.  Lane 0 streams the factor through the warp's ring of nbuf slots with
// 1-D bulk copies completed on per-slot mbarriers and refills a slot as soon as the
// warp has read it.  Every wait is bounded: one that runs out sets the status word
// and the warp stops issuing copies and computing, waits (bounded) for the copies it
// issued and returns.
#include "slr_band_kernel.cuh"

namespace slr {
namespace {

constexpr int kWarpBuf = 8;                 // ring slots at most
constexpr size_t kWarpCap = 100 * 1024;     // shared memory of a warp's CTA: two per SM

template <typename T, int NR>
__global__ void __launch_bounds__(32)
k_band_warp(const BandBlock* __restrict__ blocks, const T* __restrict__ fac, const T* in, int64_t ldi, T* out,
            int64_t ldo, const T* base, int64_t ldb, int32_t* err, int nbuf, int slot) {
    extern __shared__ __align__(128) unsigned char smem[];
    const BandBlock b = blocks[blockIdx.x];
    if (b.m == 0) return;
    const int W = b.w, c = b.c, m = b.m, lane = threadIdx.x;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);                      // [kWarpBuf]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(full + kWarpBuf);
    T* vst = reinterpret_cast<T*>(smem + 128);                               // [NR][64] y_{J-1} / x_{J+1}
    T* vt = vst + NR * 64;                                                   // [NR][64] t
    unsigned char* ring = smem + 128 + ((2 * NR * 64 * sizeof(T) + 127) & ~size_t(127));

    // the slice's row blocks (one or two) and their segment counts per block
    const int nrb = b.nrb[0];
    int R0[2], segU[3], segL[3];
#pragma unroll
    for (int rb = 0; rb < 2; ++rb) R0[rb] = rb < nrb ? 32 * b.rbmap[0][rb] : W;
    segU[0] = segL[0] = 0;
#pragma unroll
    for (int rb = 0; rb < 2; ++rb) {
        segU[rb + 1] = segU[rb] + (rb < nrb ? W - seg_cU0(W, R0[rb]) : 0);
        segL[rb + 1] = segL[rb] + (rb < nrb ? seg_cL1(W, R0[rb]) : 0);
    }
    const int per = max(1, slot / (32 * (int)sizeof(T)));                   // whole segments per chunk
    Geom q;
    q.W = W;
    q.c = c;
    q.g = 0;
    q.SU = b.SU;
    q.SL = b.SL;
    q.PS = 2 * (b.SU + b.SL);
    q.base = b.foff;
    q.nU = (segU[2] + per - 1) / per;
    q.nL = (segL[2] + per - 1) / per;
    const int total = q.nL + q.nU + 2 * (c - 1) * (q.nU + q.nL);

    if (lane == 0) {
        for (int i = 0; i < nbuf; ++i) mbar_init(&full[i], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    // the vectors' rows past W stay zero (they meet only zero factor entries)
    for (int i = lane; i < 2 * NR * 64; i += 32) vst[i] = T(0);
    __syncwarp();

    // lane 0 issues the chunks in stream order (forward: D_0, then (O_J, D_J); backward:
    // D_{c-1}^T, then (O_{J+1}^T, D_J^T)); chunk k goes to slot k mod nbuf
    int cur_type = 1, cur_plane = 0, cur_ix = 0, issued = 0;
    auto issue_next = [&]() {
        if (cur_plane < 0) return;
        const bool up = (cur_type == 0 || cur_type == 3);
        const int nseg = up ? segU[2] : segL[2];
        const int64_t e0 = q.base + (int64_t)cur_plane * q.PS + block_off(q, cur_type) + (int64_t)cur_ix * per * 32;
        const int64_t e1 = e0 + (int64_t)min(per, nseg - cur_ix * per) * 32;
        const uint32_t bytes = (uint32_t)((e1 - e0) * (int64_t)sizeof(T));
        uint64_t* bar = &full[issued % nbuf];
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(ring + (size_t)(issued % nbuf) * slot, fac + e0, bytes, bar);
        ++issued;
        if (++cur_ix == (up ? q.nU : q.nL)) {
            cur_ix = 0;
            next_block(c, cur_type, cur_plane);
        }
    };
    if (lane == 0)
        while (issued < nbuf && issued < total) issue_next();
    __syncwarp();

    int k = 0;
    T acc[2][NR];
    // acc[rb][j] = sum over the block's segments of row block rb of seg[lane] * vin[j][column]
    auto run_block = [&](int type, const T* vin) {
        const bool upper = (type == 0 || type == 3);
#pragma unroll
        for (int rb = 0; rb < 2; ++rb)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[rb][j] = T(0);
        const int nch = upper ? q.nU : q.nL;
        const int* seg = upper ? segU : segL;
        for (int ix = 0; ix < nch; ++ix, ++k) {
            bool ok = !*abort_flag;
            if (ok) {
                long long it = 0;
                while (!mbar_try_wait(&full[k % nbuf], (uint32_t)((k / nbuf) & 1))) {
                    if (++it > kSpin) {
                        ok = false;
                        break;
                    }
                }
            }
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0 && !*abort_flag) {
                    atomicExch(err, 1);
                    *abort_flag = 1;
                }
                __syncwarp();
                continue;
            }
            const int s0 = ix * per, s1 = min(s0 + per, seg[2]);
            const T* P = reinterpret_cast<const T*>(ring + (size_t)(k % nbuf) * slot);
#pragma unroll
            for (int rb = 0; rb < 2; ++rb) {
                if (rb >= nrb) break;
                const int sa = max(s0, seg[rb]), sb = min(s1, seg[rb + 1]);
                if (sa >= sb) continue;
                const int cb0 = upper ? seg_cU0(W, R0[rb]) : 0;          // column of segment seg[rb]
                const T* Ps = P + (sa - s0) * 32 + lane;
                int cc = cb0 + (sa - seg[rb]);
                const int ce = cb0 + (sb - seg[rb]);
#pragma unroll 4
                for (; cc < ce; ++cc, Ps += 32) {
                    const T a = *Ps;
#pragma unroll
                    for (int j = 0; j < NR; ++j) acc[rb][j] = fma(a, vin[j * 64 + cc], acc[rb][j]);
                }
            }
            __syncwarp();                       // every lane has read the slot: lane 0 refills it
            if (lane == 0 && issued < total && !*abort_flag) {
                fence_proxy_async();
                issue_next();
            }
        }
    };

    // =================================================================== forward
    for (int J = 0; J < c; ++J) {
        T pre[2][NR];
#pragma unroll
        for (int rb = 0; rb < 2; ++rb) {
            const int r = R0[rb] + lane, row = J * W + r;
#pragma unroll
            for (int j = 0; j < NR; ++j) pre[rb][j] = (rb < nrb && r < W && row < m) ? in[b.row0 + row + j * ldi] : T(0);
        }
        if (J > 0) {
            run_block(0, vst);                                                 // O_J y_{J-1}
        } else {
#pragma unroll
            for (int rb = 0; rb < 2; ++rb)
#pragma unroll
                for (int j = 0; j < NR; ++j) acc[rb][j] = T(0);
        }
#pragma unroll
        for (int rb = 0; rb < 2; ++rb) {
            const int r = R0[rb] + lane;
            if (rb < nrb && r < W)
#pragma unroll
                for (int j = 0; j < NR; ++j) vt[j * 64 + r] = pre[rb][j] - acc[rb][j];
        }
        __syncwarp();
        run_block(1, vt);                                                      // D_J t
#pragma unroll
        for (int rb = 0; rb < 2; ++rb) {
            const int r = R0[rb] + lane, row = J * W + r;
            if (rb < nrb && r < W)
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    if (row < m) out[b.row0 + row + j * ldo] = acc[rb][j];
                    vst[j * 64 + r] = acc[rb][j];
                }
        }
        __syncwarp();
    }
    // =================================================================== backward
    for (int J = c - 1; J >= 0; --J) {
        T pre[2][NR], bs[2][NR];
#pragma unroll
        for (int rb = 0; rb < 2; ++rb) {
            const int r = R0[rb] + lane, row = J * W + r;
            const bool own = rb < nrb && r < W && row < m;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                pre[rb][j] = own ? out[b.row0 + row + j * ldo] : T(0);
                bs[rb][j] = (own && base) ? base[b.row0 + row + j * ldb] : T(0);
            }
        }
        if (J < c - 1) {
            run_block(2, vst);                                                 // O_{J+1}^T x_{J+1}
        } else {
#pragma unroll
            for (int rb = 0; rb < 2; ++rb)
#pragma unroll
                for (int j = 0; j < NR; ++j) acc[rb][j] = T(0);
        }
#pragma unroll
        for (int rb = 0; rb < 2; ++rb) {
            const int r = R0[rb] + lane;
            if (rb < nrb && r < W)
#pragma unroll
                for (int j = 0; j < NR; ++j) vt[j * 64 + r] = pre[rb][j] - acc[rb][j];
        }
        __syncwarp();
        run_block(3, vt);                                                      // D_J^T t
#pragma unroll
        for (int rb = 0; rb < 2; ++rb) {
            const int r = R0[rb] + lane, row = J * W + r;
            if (rb < nrb && r < W)
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    if (row < m) out[b.row0 + row + j * ldo] = base ? bs[rb][j] - acc[rb][j] : acc[rb][j];
                    vst[j * 64 + r] = acc[rb][j];
                }
        }
        __syncwarp();
    }
    // after an abort: the last copy issued into each slot has landed before the warp leaves
    if (lane == 0 && *abort_flag) {
        for (int sl = 0; sl < nbuf && sl < issued; ++sl) {
            const int last = sl + ((issued - 1 - sl) / nbuf) * nbuf;
            long long it = 0;
            while (!mbar_try_wait(&full[sl], (uint32_t)((last / nbuf) & 1)) && ++it <= kSpin) {
            }
        }
    }
}

template <typename T, int NR>
cudaError_t warp_launch(const DevOperator<T>& op, int32_t p, const T* in, int64_t ldi, T* out, int64_t ldo,
                        const T* base, int64_t ldb, cudaStream_t st) {
    auto kern = k_band_warp<T, NR>;
    static std::mutex mu;
    static uint64_t raised = 0;                     // bit d: the limit is raised on device d
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu);
        if (!(raised >> dev & 1)) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpCap);
            if (e != cudaSuccess) return e;
            raised |= 1ull << dev;
        }
    }
    const size_t fixed = 128 + ((2 * NR * 64 * sizeof(T) + 127) & ~size_t(127));
    // slots of whole 128-byte multiples filling the rest, nbuf of them (2 .. 8)
    const int nbuf = kWarpBuf;
    const int32_t slot = (int32_t)(((kWarpCap - fixed) / nbuf) & ~size_t(127));
    if (slot < 32 * (int32_t)sizeof(T)) return cudaErrorInvalidValue;
    k_band_warp<T, NR><<<p, 32, fixed + (size_t)nbuf * slot, st>>>(op.band, op.bfac, in, ldi, out, ldo, base, ldb,
                                                                    op.err, nbuf, slot);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

// The warp-per-subdomain band solve (planes of at most 64 rows, one slice per
// subdomain), 1, 2 or 4 right-hand sides per launch as the block kernel takes them.
template <typename T>
cudaError_t launch_band_warp(const DevOperator<T>& op, int32_t p, const T* in, int64_t ldi, T* out, int64_t ldo,
                             const T* base, int64_t ldb, int32_t nrhs, cudaStream_t st) {
    for (int32_t c = 0; c < nrhs;) {
        const int32_t left = nrhs - c;
        const int nr = left >= 4 ? 4 : left >= 2 ? 2 : 1;
        const T* bs = base ? base + c * ldb : nullptr;
        cudaError_t e = nr == 4 ? warp_launch<T, 4>(op, p, in + c * ldi, ldi, out + c * ldo, ldo, bs, ldb, st)
                        : nr == 2 ? warp_launch<T, 2>(op, p, in + c * ldi, ldi, out + c * ldo, ldo, bs, ldb, st)
                                  : warp_launch<T, 1>(op, p, in + c * ldi, ldi, out + c * ldo, ldo, bs, ldb, st);
        if (e != cudaSuccess) return e;
        c += nr;
    }
    return cudaSuccess;
}

template cudaError_t launch_band_warp<float>(const DevOperator<float>&, int32_t, const float*, int64_t, float*,
                                             int64_t, const float*, int64_t, int32_t, cudaStream_t);
template cudaError_t launch_band_warp<double>(const DevOperator<double>&, int32_t, const double*, int64_t, double*,
                                              int64_t, const double*, int64_t, int32_t, cudaStream_t);

}  // namespace slr
