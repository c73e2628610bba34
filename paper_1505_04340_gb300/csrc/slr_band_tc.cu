// K1 for blocks of right-hand sides on the tensor cores: t = B^{-1} F with
// B = diag(B_i) (Section 5.2), F an n_I x r block (8 <= r <= 64), in the mixed
// path, with the band factor and the plane vectors rounded to TF32 or BF16 and
// every product accumulated in FP32 in tensor memory (tcgen05.mma, M = 128).
//
// The factor of B_i is the plane chain of slr_band.cu (planes of W <= 256 rows):
//   forward   t = F_J - O_J Y_{J-1},        Y_J = D_J t
//   backward  t = Y_J - O_{J+1}^T X_{J+1},  X_J = D_J^T t
// Each of the four products per plane is a dense W x W (triangular) block times
// a W x r block, i.e. an MMA with M = W (one or two tiles of 128 rows), K = W
// (steps of KS columns: 8 TF32 or 16 BF16) and N = r (padded to NP = 16, 32, 48
// or 64).  The factor is packed once (k_band_tc_pack) as "sub-tiles" of 128 rows
// x KS columns, 4096 bytes each, already in the K-major core-matrix layout of
// slr_tc.cuh (SBO = 256, LBO = 128), keeping only the sub-tiles that meet the
// triangle: per plane [O_J | D_J | O_J^T | D_J^T], each block M-tile by M-tile,
// K-steps ascending.  The vectors Y / X and t live in shared memory as the MMA's
// B operand (NP x WK, K-major, WK = W rounded up to KS, zero past W).
//
// One CTA of 256 threads per subdomain, three roles:
//   thread 0 (warp 0)  streams the sub-tiles through a ring of shared slots with
//                      1-D bulk copies (cp.async.bulk) on "full" mbarriers;
//   thread 32 (warp 1) issues the MMAs of a block once its vector operand is in
//                      shared memory, returns each slot by tcgen05.commit on its
//                      "empty" mbarrier and signals the accumulator on "acc";
//   warps 4-7          read the accumulator (thread e owns rows e and 128 + e),
//                      form t, Y or X, write the next operand into shared memory
//                      and the results to global memory, and arrive on "opnd".
// Every wait is bounded: one that runs out sets the status word (1) and the CTA's
// abort flag; every role then stops, thread 0 waits (bounded) for the copies it
// issued, thread 32 for the MMAs it issued, and the tensor memory is freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "slr_device.h"
#include "slr_tc.cuh"

namespace slr {
namespace {

constexpr int kBtThreads = 256;
constexpr int kSub = 4096;                 // bytes of one sub-tile (128 rows x 32 bytes)
constexpr long long kBtSpin = 1ll << 24;   // polls of a bounded wait

template <int AB>
struct BtType;
template <>
struct BtType<2> {   // TF32 in FP32 containers
    using Te = float;
    static constexpr int E = 4, KS = 8;
    __device__ static float pack(float x) { return tc::to_tf32(x); }
};
template <>
struct BtType<1> {   // BF16
    using Te = __nv_bfloat16;
    static constexpr int E = 2, KS = 16;
    __device__ static __nv_bfloat16 pack(float x) { return __float2bfloat16_rn(x); }
};

// K-steps of the sub-tiles that meet the triangle, for M-tile mt of a W x W block
// with ks steps of KS columns: upper (row <= column) or lower (row >= column)
__host__ __device__ inline int bt_nk(int W, int KS) { return (W + KS - 1) / KS; }
__host__ __device__ inline int bt_k0(bool upper, int mt, int KS) { return upper ? 128 * mt / KS : 0; }
__host__ __device__ inline int bt_k1(bool upper, int mt, int W, int KS) {
    const int hi = 128 * mt + 128 < W ? 128 * mt + 128 : W;
    return upper ? bt_nk(W, KS) : (hi + KS - 1) / KS;
}
__host__ __device__ inline int bt_tiles(bool upper, int W, int KS) {
    int n = 0;
    for (int mt = 0; mt * 128 < W; ++mt) n += bt_k1(upper, mt, W, KS) - bt_k0(upper, mt, KS);
    return n;
}

// ------------------------------------------------------------------ packing
// one CTA per (subdomain, plane, block type); scr holds the subdomain's dense
// plane blocks (slr_band_factor.cu): D_J then O_J, row-major W x W, then the pivot
// signs, which go into the forward blocks as in the CUDA-core layout
template <int AB>
__global__ void __launch_bounds__(256)
k_band_tc_pack(const BandTcBlock* __restrict__ band, int32_t cmax, const double* __restrict__ scr,
               const int64_t* __restrict__ soff, unsigned char* fac, int indef) {
    using Tp = BtType<AB>;
    using Te = typename Tp::Te;
    constexpr int E = Tp::E, KS = Tp::KS;
    const int i = blockIdx.x / (cmax * 4), J = (blockIdx.x / 4) % cmax, type = blockIdx.x % 4;
    const BandTcBlock b = band[i];
    if (b.m == 0 || J >= b.c) return;
    const int W = b.w, m = b.m;
    const int64_t WW = (int64_t)W * W;
    const double* S0 = scr + soff[b.id];
    const double* X = S0 + WW + (int64_t)J * WW;                    // D_J
    const double* O = S0 + WW + (int64_t)(b.c + J) * WW;            // O_J
    const double* Sg = S0 + WW + 2 * (int64_t)b.c * WW;             // pivot signs
    auto sgn = [&](int plane, int r) -> double { return indef ? Sg[(int64_t)plane * W + r] : 1.0; };
    const bool upper = type == 0 || type == 3;
    const int64_t boff = type == 0 ? 0 : type == 1 ? b.nU : type == 2 ? b.nU + b.nL : b.nU + 2 * b.nL;
    unsigned char* blk = fac + b.foff + ((int64_t)J * (2 * b.nU + 2 * b.nL) + boff) * kSub;
    int tile = 0;
    for (int mt = 0; mt * 128 < W; ++mt)
        for (int ks = bt_k0(upper, mt, KS); ks < bt_k1(upper, mt, W, KS); ++ks, ++tile) {
            unsigned char* st = blk + (int64_t)tile * kSub;
            for (int e = threadIdx.x; e < 128 * KS; e += blockDim.x) {
                const int rl = e / KS, q = e % KS, r = 128 * mt + rl, cc = ks * KS + q;
                double v = 0.0;
                if (r < W && cc < W) {
                    if (type == 0 && r <= cc && J > 0 && J * W + r < m) v = O[(int64_t)r * W + cc] * sgn(J - 1, cc);
                    else if (type == 1 && r >= cc) v = X[(int64_t)r * W + cc] * sgn(J, r);
                    else if (type == 2 && r >= cc && J > 0 && J * W + cc < m) v = O[(int64_t)cc * W + r];
                    else if (type == 3 && r <= cc) v = X[(int64_t)cc * W + r];
                }
                *reinterpret_cast<Te*>(st + tc::kmajor_off<E>(rl, q, KS)) = Tp::pack((float)v);
            }
        }
}

// ------------------------------------------------------------------ the solve
// The block sequence of one subdomain: forward D_0, (O_J, D_J) for J = 1 .. c-1;
// backward D_{c-1}^T, (O_{J+1}^T, D_J^T) for J = c-2 .. 0.  Block q of the
// sequence: its plane (where its sub-tiles are stored), type, and the plane of
// the vector it produces.
struct BtBlock {
    int plane, type, vplane;
};
__device__ __forceinline__ BtBlock bt_block(int q, int c) {
    if (q < 2 * c - 1) {                               // forward
        if (q == 0) return {0, 1, 0};
        const int J = (q + 1) / 2;
        return (q & 1) ? BtBlock{J, 0, J} : BtBlock{J, 1, J};
    }
    const int u = q - (2 * c - 1);                     // backward
    if (u == 0) return {c - 1, 3, c - 1};
    const int J = c - 1 - (u + 1) / 2;
    return (u & 1) ? BtBlock{J + 1, 2, J} : BtBlock{J, 3, J};
}

// Operand rows of 32 columns c0 .. c0 + 31 from the lanes' values v (lane = row
// rbase + lane): a butterfly transpose inside groups of RPQ = 16 / E lanes (the rows
// that share 16 bytes of a core-matrix row) leaves lane u of a group holding
// column c0 + jc RPQ + u of the group's RPQ rows, stored as one 16-byte word.
template <int AB>
__device__ __forceinline__ void bt_put_rows(unsigned char* vdst, int rbase, int c0, const float (&v)[32],
                                            uint32_t sbo_v, int nrhs, int W, int lane) {
    using Tp = BtType<AB>;
    using Te = typename Tp::Te;
    constexpr int RPQ = 16 / Tp::E;
    const int grp = lane / RPQ, u = lane % RPQ;
#pragma unroll
    for (int jc = 0; jc < 32 / RPQ; ++jc) {
        float a[RPQ];
#pragma unroll
        for (int i = 0; i < RPQ; ++i) a[i] = v[jc * RPQ + i];
#pragma unroll
        for (int m = 1; m < RPQ; m <<= 1) {
            const bool upper = (u & m) != 0;
#pragma unroll
            for (int i = 0; i < RPQ; ++i) {
                if (i & m) continue;
                const float send = upper ? a[i] : a[i | m];
                const float recv = __shfl_xor_sync(0xffffffffu, send, m);
                if (upper) a[i] = recv;
                else a[i | m] = recv;
            }
        }
        const int j = c0 + jc * RPQ + u;
        const int r0 = rbase + grp * RPQ;              // first of the group's rows (a multiple of RPQ)
        if (j < nrhs && r0 < W) {
            uint32_t w32[4];
            if constexpr (RPQ == 4) {
#pragma unroll
                for (int k = 0; k < 4; ++k) w32[k] = __float_as_uint(Tp::pack(r0 + k < W ? a[k] : 0.0f));
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(r0 + 2 * k < W ? a[2 * k] : 0.0f,
                                                                    r0 + 2 * k + 1 < W ? a[2 * k + 1] : 0.0f);
                    w32[k] = *reinterpret_cast<const uint32_t*>(&h2);
                }
            }
            *reinterpret_cast<uint4*>(vdst + (j >> 3) * sbo_v + (r0 / RPQ) * 128 + (j & 7) * 16) =
                make_uint4(w32[0], w32[1], w32[2], w32[3]);
        }
    }
}

template <int AB, int NP>
__global__ void __launch_bounds__(kBtThreads, NP <= 32 ? 2 : 1)
k_band_tc(const BandTcBlock* __restrict__ blocks, const unsigned char* __restrict__ fac, const float* in,
          int64_t ldi, float* out, int64_t ldo, const float* base, int64_t ldb, int32_t nrhs, int32_t nslot,
          int32_t stiles, int32_t* err) {
    using Tp = BtType<AB>;
    using Te = typename Tp::Te;
    constexpr int E = Tp::E, KS = Tp::KS;
    extern __shared__ __align__(1024) unsigned char sm[];
    const BandTcBlock b = blocks[blockIdx.x];
    if (b.m == 0) return;
    const int W = b.w, c = b.c, m = b.m;
    const int WK = bt_nk(W, KS) * KS;
    const uint32_t vbytes = (uint32_t)NP * WK * E, sbo_v = 8u * WK * E;
    // One operand buffer: a block's MMAs all complete (acc_bar) before its epilogue
    // overwrites the operand with the next block's, and the next block's MMAs wait
    // for that epilogue (opnd_bar), so the two never overlap.
    unsigned char* ring = sm;                                      // nslot x stiles sub-tiles
    unsigned char* vbuf = ring + (size_t)nslot * stiles * kSub;    // the vector operand
    uint64_t* full = reinterpret_cast<uint64_t*>(vbuf + (size_t)vbytes);
    uint64_t* empty = full + nslot;
    uint64_t* acc_bar = empty + nslot;
    uint64_t* opnd_bar = acc_bar + 1;
    uint64_t* fin_bar = opnd_bar + 1;
    uint32_t* tbase = reinterpret_cast<uint32_t*>(fin_bar + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tbase + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nM = (W + 127) / 128;
    // tensor memory: the accumulators (M-tile mt at column mt CS), then as many columns
    // holding the epilogue's global operand of a block (F_J, Y_J or the base), written
    // by the epilogue threads while the block's MMAs run.  The epilogue moves 32
    // columns at a time, so an M-tile's columns are at least 32 wide (CS): with N = 16
    // and two M-tiles, a stride of 16 would put the second tile's staged operand past
    // the allocation, into the columns of the SM's other CTA.
    constexpr uint32_t CS = NP < 32 ? 32 : NP;
    const uint32_t acols = nM * CS <= 32 ? 32 : nM * CS <= 64 ? 64 : 128, ncol = 2 * acols;
    if (warp == 0) {
        tc::tmem_alloc(tbase, ncol);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < nslot; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(acc_bar, 1);
        tc::mbar_init(opnd_bar, 128);
        tc::mbar_init(fin_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (uint32_t e = tid; e < vbytes / 16; e += kBtThreads)                // K and N padding stay zero
        reinterpret_cast<uint4*>(vbuf)[e] = make_uint4(0, 0, 0, 0);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tbase;
    const int nU = b.nU, nL = b.nL;
    const int nblk = 4 * c - 2;
    auto tiles_of = [&](int type) { return (type == 0 || type == 3) ? nU : nL; };
    auto fills_of = [&](int type) { return (tiles_of(type) + stiles - 1) / stiles; };
    auto fail = [&]() {
        atomicExch(err, 1);
        *abort_flag = 1;
    };

    if (tid == 0) {
        // ---------------------------------------------------------------- producer
        int f = 0;
        for (int q = 0; q < nblk && !*abort_flag; ++q) {
            const BtBlock bk = bt_block(q, c);
            const int nt = tiles_of(bk.type);
            const int64_t boff = bk.type == 0 ? 0 : bk.type == 1 ? nU : bk.type == 2 ? nU + nL : nU + 2 * nL;
            const unsigned char* src = fac + b.foff + ((int64_t)bk.plane * (2 * nU + 2 * nL) + boff) * kSub;
            for (int t0 = 0; t0 < nt; t0 += stiles, ++f) {
                const int s = f % nslot;
                if (f >= nslot && !tc::mbar_wait(&empty[s], (uint32_t)(((f / nslot) - 1) & 1), kBtSpin)) {
                    fail();
                    break;
                }
                if (*abort_flag) break;
                const uint32_t bytes = (uint32_t)(min(stiles, nt - t0) * kSub);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(&full[s])),
                             "r"(bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        tc::smem_addr(ring + (size_t)s * stiles * kSub)),
                    "l"(src + (int64_t)t0 * kSub), "r"(bytes), "r"(tc::smem_addr(&full[s]))
                    : "memory");
            }
        }
        // no copy of this CTA still writes its shared memory when it leaves: the last
        // fill of each slot has landed (fills of a slot complete in order)
        for (int s = 0; s < nslot && s < f; ++s) {
            const int last = s + ((f - 1 - s) / nslot) * nslot;
            tc::mbar_wait(&full[s], (uint32_t)((last / nslot) & 1), kBtSpin);
        }
    } else if (tid == 32) {
        // ---------------------------------------------------------------- MMA issuer
        const uint32_t idesc = tc::instr_desc(AB, 128, NP);
        int f = 0;
        for (int q = 0; q < nblk; ++q) {
            if (!tc::mbar_wait(opnd_bar, (uint32_t)(q & 1), kBtSpin)) fail();
            if (*abort_flag) break;
            tc::fence_after_sync();
            const BtBlock bk = bt_block(q, c);
            const bool upper = bk.type == 0 || bk.type == 3;
            // the operand: t (D blocks) or Y / X (O blocks), written by the last epilogue
            const uint32_t vb = tc::smem_addr(vbuf);
            int t = 0;
            bool ok = true;
            for (int mt = 0; mt < nM && ok; ++mt)
                for (int ks = bt_k0(upper, mt, KS); ks < bt_k1(upper, mt, W, KS); ++ks, ++t) {
                    const int fl = f + t / stiles, s = fl % nslot, in_slot = t % stiles;
                    if (in_slot == 0 && !tc::mbar_wait(&full[s], (uint32_t)((fl / nslot) & 1), kBtSpin)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const uint32_t sa = tc::smem_addr(ring + ((size_t)s * stiles + in_slot) * kSub);
                    tc::mma<AB>(tmem + (uint32_t)(mt * CS), tc::smem_desc(sa, 128, 256),
                                tc::smem_desc(vb + 256u * ks, 128, sbo_v), idesc, ks > bt_k0(upper, mt, KS));
                    const bool last_of_fill = in_slot == stiles - 1 || t == tiles_of(bk.type) - 1;
                    if (last_of_fill) tc::commit(&empty[s]);
                }
            if (!ok) break;
            f += fills_of(bk.type);
            tc::commit(acc_bar);
        }
        tc::commit(fin_bar);                            // every MMA issued has completed
        tc::mbar_wait(fin_bar, 0, kBtSpin);
    } else if (warp >= 4) {
        // ---------------------------------------------------------------- epilogue
        const int e = tid - 128, quarter = warp - 4;
        const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
        unsigned char* v0 = vbuf;                       // Y / X
        unsigned char* v1 = vbuf;                       // t (the same buffer, in turn)
        // byte of (column j, row r) of an operand (K index r)
        auto opos = [&](int j, int r) -> uint32_t {
            return (uint32_t)((j >> 3) * sbo_v + (r / (16 / E)) * 128 + (j & 7) * 16 + (r % (16 / E)) * E);
        };
        auto arrive = [&]() {
            tc::fence_async_smem();
            tc::fence_before_sync();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(opnd_bar)) : "memory");
        };
        auto row_of = [&](int J, int r) -> int64_t { return (int64_t)b.row0 + (int64_t)J * W + r; };
        auto valid = [&](int J, int r) { return r < W && J * W + r < m; };
        // forward pre-step: t = F_0 into buffer 1
        for (int mt = 0; mt < nM; ++mt) {
            const int r = 128 * mt + e;
            if (r >= W) continue;
            const bool ok = valid(0, r);
            for (int j = 0; j < nrhs; ++j)
                *reinterpret_cast<Te*>(v1 + opos(j, r)) = Tp::pack(ok ? in[row_of(0, r) + j * ldi] : 0.0f);
        }
        arrive();
        auto put_rows = [&](unsigned char* vdst, int rbase, int c0, const float (&v)[32]) {
            bt_put_rows<AB>(vdst, rbase, c0, v, sbo_v, nrhs, W, tid & 31);
        };
        for (int q = 0; q < nblk; ++q) {
            const BtBlock bk = bt_block(q, c);
            const int J = bk.vplane;
            // this block's global operand into tensor memory while its MMAs run (the
            // previous block's epilogue, by these threads, has read the columns)
            const bool need_pre = bk.type == 0 || bk.type == 2 || (bk.type == 3 && base);
            if (need_pre) {
                const float* srcb = bk.type == 0 ? in : bk.type == 2 ? out : base;
                const int64_t lds = bk.type == 0 ? ldi : bk.type == 2 ? ldo : ldb;
                for (int mt = 0; mt < nM; ++mt) {
                    const int r = 128 * mt + e;
                    const bool ok = valid(J, r);
                    const int64_t row = row_of(J, r);
#pragma unroll
                    for (int c0 = 0; c0 < NP; c0 += 32) {
                        float pv[32];
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            pv[jj] = (ok && c0 + jj < nrhs) ? srcb[row + (c0 + jj) * lds] : 0.0f;
                        tc::tmem_st32(tmem + lane_addr + acols + (uint32_t)(mt * CS + c0), pv);
                    }
                }
            }
            // the warp decides together (tcgen05.ld below is warp-collective)
            bool ok = tc::mbar_wait(acc_bar, (uint32_t)(q & 1), kBtSpin);
            if (!__all_sync(0xffffffffu, ok)) {
                if ((tid & 31) == 0) fail();
                break;
            }
            if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
            tc::fence_after_sync();
            for (int mt = 0; mt < nM; ++mt) {
                const int r = 128 * mt + e;
                const bool in_w = r < W, ok_r = valid(J, r);
                const int64_t row = row_of(J, r);
                const int rbase = 128 * mt + 32 * quarter;      // first row of the warp
#pragma unroll
                for (int c0 = 0; c0 < NP; c0 += 32) {
                    float v[32];
                    tc::tmem_ld32(tmem + lane_addr + (uint32_t)(mt * CS + c0), v);
                    const uint32_t pre_col = tmem + lane_addr + acols + (uint32_t)(mt * CS + c0);
                    // v := pre - v (the operand's columns past nrhs were stored as zeros)
                    auto pre_minus = [&]() {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float p[16];
                            tc::tmem_ld16(pre_col + 16 * h, p);
#pragma unroll
                            for (int i = 0; i < 16; ++i) v[16 * h + i] = p[i] - v[16 * h + i];
                        }
                    };
                    if (bk.type == 0 || bk.type == 2) {          // t = F_J - O_J Y_{J-1}  /  Y_J - O^T X
                        pre_minus();
                        put_rows(v1, rbase, c0, v);
                    } else if (bk.type == 1) {                   // Y_J = D_J t
                        if (in_w && ok_r) {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj)
                                if (c0 + jj < nrhs) out[row + (c0 + jj) * ldo] = v[jj];
                        }
                        put_rows(v0, rbase, c0, v);             // also the backward's first t (J = c - 1)
                    } else {                                     // X_J = D_J^T t (out: base - X_J with a base)
                        if (base) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                float p[16];
                                tc::tmem_ld16(pre_col + 16 * h, p);    // warp-collective: every lane
                                if (in_w && ok_r) {
#pragma unroll
                                    for (int i = 0; i < 16; ++i)
                                        if (c0 + 16 * h + i < nrhs) out[row + (c0 + 16 * h + i) * ldo] = p[i] - v[16 * h + i];
                                }
                            }
                        } else if (in_w && ok_r) {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj)
                                if (c0 + jj < nrhs) out[row + (c0 + jj) * ldo] = v[jj];
                        }
                        put_rows(v0, rbase, c0, v);
                    }
                }
            }
            if (q + 1 < nblk) arrive();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc::tmem_dealloc(tmem, ncol);
    }
}

template <int AB, int NP>
cudaError_t bt_launch(const DevOperator<float>& op, int32_t p, const float* in, int64_t ldi, float* out, int64_t ldo,
                      const float* base, int64_t ldb, int32_t nrhs, cudaStream_t st) {
    constexpr int E = BtType<AB>::E, KS = BtType<AB>::KS;
    const int WK = bt_nk(op.band_tc_wmax, KS) * KS;
    const size_t vbytes = (size_t)NP * WK * E;
    const size_t fixed = vbytes + 8 * (2 * 8 + 3) + 16;
    // ring: as many 8-sub-tile slots (32 KB) as fit, 2 .. 8, in the opt-in maximum or,
    // with more subdomains than SMs, in half an SM (113 KB: two CTAs per SM, one wave).
    // Fewer, larger copies measured faster: on 3-D 96^3 with 32 columns two 32 KB slots
    // took 1014 us per B-solve, five of 16 KB 1039 us, ten of 8 KB 1114 us.
    const int stiles = 8;
    const size_t cap = (NP <= 32 && p > op.cf.nsm) ? 113 * 1024 : 227 * 1024;
    int nslot = fixed < cap ? (int)((cap - fixed) / ((size_t)stiles * kSub)) : 0;
    nslot = nslot > 8 ? 8 : nslot;
    if (nslot < 2) return cudaErrorInvalidValue;
    const size_t smem = (size_t)nslot * stiles * kSub + fixed;
    cudaError_t e = cudaFuncSetAttribute(k_band_tc<AB, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    k_band_tc<AB, NP><<<p, kBtThreads, smem, st>>>(op.band_tc, op.band_tc_fac, in, ldi, out, ldo, base, ldb, nrhs,
                                                  nslot, stiles, op.err);
    count_launches(1);
    return cudaGetLastError();
}

template <int AB>
cudaError_t bt_launch_np(const DevOperator<float>& op, int32_t p, const float* in, int64_t ldi, float* out,
                         int64_t ldo, const float* base, int64_t ldb, int32_t nrhs, cudaStream_t st) {
    if (nrhs <= 16) return bt_launch<AB, 16>(op, p, in, ldi, out, ldo, base, ldb, nrhs, st);
    if (nrhs <= 32) return bt_launch<AB, 32>(op, p, in, ldi, out, ldo, base, ldb, nrhs, st);
    return bt_launch<AB, 64>(op, p, in, ldi, out, ldo, base, ldb, nrhs, st);
}

}  // namespace

int bt_ks(int32_t mma_dtype) { return mma_dtype == SLR_U_BF16 ? 16 : 8; }

std::vector<BandTcBlock> band_tc_layout(const std::vector<BandBlock>& run_order, int32_t mma_dtype, int64_t* bytes) {
    const int KS = bt_ks(mma_dtype);
    std::vector<BandTcBlock> out(run_order.size());
    // sub-tiles stored subdomain by subdomain in subdomain order, whatever the run order
    std::vector<int64_t> off(run_order.size() + 1, 0);
    std::vector<const BandBlock*> by_id(run_order.size());
    for (const BandBlock& b : run_order) by_id[b.id] = &b;
    for (size_t i = 0; i < by_id.size(); ++i) {
        const BandBlock& b = *by_id[i];
        const int64_t per_plane = b.m ? 2 * (int64_t)bt_tiles(true, b.w, KS) + 2 * (int64_t)bt_tiles(false, b.w, KS) : 0;
        off[i + 1] = off[i] + per_plane * b.c * kSub;
    }
    for (size_t q = 0; q < run_order.size(); ++q) {
        const BandBlock& b = run_order[q];
        BandTcBlock t;
        t.m = b.m;
        t.w = b.w;
        t.c = b.c;
        t.row0 = b.row0;
        t.id = b.id;
        t.foff = off[b.id];
        t.nU = b.m ? bt_tiles(true, b.w, KS) : 0;
        t.nL = b.m ? bt_tiles(false, b.w, KS) : 0;
        out[q] = t;
    }
    *bytes = off.back();
    return out;
}

cudaError_t launch_band_tc_pack(int32_t mma_dtype, const BandTcBlock* band, int32_t p, int32_t cmax,
                                const double* scr, const int64_t* soff, unsigned char* fac, bool indef,
                                cudaStream_t st) {
    if (p == 0 || cmax == 0) return cudaSuccess;
    const unsigned grid = (unsigned)p * cmax * 4;
    if (mma_dtype == SLR_U_BF16) k_band_tc_pack<1><<<grid, 256, 0, st>>>(band, cmax, scr, soff, fac, indef ? 1 : 0);
    else k_band_tc_pack<2><<<grid, 256, 0, st>>>(band, cmax, scr, soff, fac, indef ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_band_solve_tc(const DevOperator<float>& op, int32_t p, const float* in, int64_t ldi, float* out,
                                 int64_t ldo, const float* base, int64_t ldb, int32_t nrhs, cudaStream_t st) {
    if (p == 0) return cudaSuccess;
    for (int32_t c0 = 0; c0 < nrhs; c0 += 64) {
        const int32_t nr = nrhs - c0 < 64 ? nrhs - c0 : 64;
        const float* bs = base ? base + c0 * ldb : nullptr;
        cudaError_t e = op.band_mma == SLR_U_BF16
                            ? bt_launch_np<1>(op, p, in + c0 * ldi, ldi, out + c0 * ldo, ldo, bs, ldb, nr, st)
                            : bt_launch_np<2>(op, p, in + c0 * ldi, ldi, out + c0 * ldo, ldo, bs, ldb, nr, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace slr
