// The C ABI of include/slr.h: setup orchestration (host analysis, upload,
// device Lanczos), the SLR apply, SLR-preconditioned CG and the accessors.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <shared_mutex>
#include <string>
#include <type_traits>
#include <tuple>
#include <vector>

#include "slr_device.h"

using namespace slr;

namespace {

#define CK(...)                                                                            \
    do {                                                                                   \
        cudaError_t e_ = (__VA_ARGS__);                                                    \
        if (e_ != cudaSuccess) {                                                           \
            set_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));          \
            return SLR_ERR_CUDA;                                                           \
        }                                                                                  \
    } while (0)
#define CS(...)                                    \
    do {                                           \
        slr_status s_ = (__VA_ARGS__);             \
        if (s_ != SLR_OK) return s_;               \
    } while (0)

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Graph captures and device frees exclude each other.  A stream capture in one
// thread fails if another thread meanwhile makes a call that must wait for the
// capturing stream; a free may wait for the whole device.  Captures share the
// lock, frees take it alone.  (Captures take milliseconds and happen once per
// handle and right-hand-side count.)
std::shared_mutex g_capture_mu;

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&old);
        if (old != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (old >= 0 && cur != old) cudaSetDevice(old);
    }
};

// slr_inject_alloc_failure: allocations left until the injected failure (0: off)
std::atomic<int64_t> g_fail_alloc{0};

template <typename T>
slr_status dalloc(slr_handle h, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return SLR_OK;
    if (g_fail_alloc.load(std::memory_order_relaxed) > 0 && g_fail_alloc.fetch_sub(1) == 1) {
        set_error("cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: injected failure");
        return SLR_ERR_OOM;
    }
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e));
        return SLR_ERR_OOM;
    }
    h->allocs.push_back((void*)*p);
    h->device_bytes += (int64_t)(count * sizeof(T));
    return SLR_OK;
}

template <typename T>
void dfree(slr_handle h, T*& p, size_t count) {
    if (!p) return;
    auto it = std::find(h->allocs.begin(), h->allocs.end(), (void*)p);
    if (it != h->allocs.end()) h->allocs.erase(it);
    {
        std::unique_lock<std::shared_mutex> lk(g_capture_mu);
        cudaFree(p);
    }
    h->device_bytes -= (int64_t)(count * sizeof(T));
    p = nullptr;
}

// A device buffer of the handle freed when it goes out of scope (also on an early
// error return).
template <typename T>
struct ScopedBuf {
    slr_handle h;
    T* p = nullptr;
    size_t n = 0;
    explicit ScopedBuf(slr_handle hh) : h(hh) {}
    ScopedBuf(const ScopedBuf&) = delete;
    ScopedBuf& operator=(const ScopedBuf&) = delete;
    ~ScopedBuf() {
        if (p) dfree(h, p, n);
    }
    slr_status alloc(size_t count) {
        n = count;
        return dalloc(h, &p, count);
    }
};

template <typename TD, typename TS>
slr_status upload(slr_handle h, TD** p, const std::vector<TS>& v) {
    CS(dalloc(h, p, v.size()));
    if (v.empty()) return SLR_OK;
    // from pageable memory: the call returns once the data is staged, so the
    // source may go away afterwards
    if constexpr (std::is_same<TD, TS>::value) {
        CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(TD), cudaMemcpyHostToDevice, h->stream));
    } else {
        std::vector<TD> tmp(v.begin(), v.end());
        CK(cudaMemcpyAsync(*p, tmp.data(), tmp.size() * sizeof(TD), cudaMemcpyHostToDevice, h->stream));
    }
    return SLR_OK;
}

// The band blocks on the device, in the order their clusters are launched
// (opts.band_order; every order gives the same result, bit for bit).
slr_status upload_band(slr_handle h, BandBlock** p) {
    return upload(h, p, band_run_order(h->hs.band, h->opts.band_order ? h->opts.band_order : kBandOrderAuto));
}

template <typename T>
slr_status upload_operator(slr_handle h, DevOperator<T>& op, bool with_band) {
    const HostSetup& hs = h->hs;
    const int32_t r = std::max(1, h->opts.nrhs_max);
    CS(upload_band(h, &op.band));
    if (with_band) CS(upload(h, &op.bfac, hs.bfac));
    op.band_G = hs.band_G;
    op.band_nbuf = h->opts.band_slots;
    op.band_nt = hs.band_nt;
    CS(dalloc(h, &op.err, 1));
    CK(cudaMemsetAsync(op.err, 0, sizeof(int32_t), h->stream));
    CS(upload(h, &op.e_rp, hs.e_rp));
    CS(upload(h, &op.e_ci, hs.e_ci));
    CS(upload(h, &op.e_v, hs.e_v));
    CS(upload(h, &op.et_rp, hs.et_rp));
    CS(upload(h, &op.et_ci, hs.et_ci));
    CS(upload(h, &op.et_v, hs.et_v));
    const CFactorHost& c = hs.cf;
    DevCFactor<T>& d = op.cf;
    d.s = c.s;
    d.ns = c.ns;
    d.nlev = c.nlev;
    d.lev_task_ptr = c.lev_task_ptr;
    CS(upload(h, &d.cperm, c.cperm));
    {
        std::vector<int32_t> ip(c.cperm.size());
        for (size_t q = 0; q < c.cperm.size(); ++q) ip[c.cperm[q]] = (int32_t)q;
        CS(upload(h, &d.ciperm, ip));
    }
    CS(upload(h, &d.c0, c.c0));
    CS(upload(h, &d.r_off, c.r_off));
    CS(upload(h, &d.rows, c.rows));
    CS(upload(h, &d.pan_off, c.pan_off));
    CS(upload(h, &d.panel, c.panel));
    CS(upload(h, &d.dinv_off, c.dinv_off));
    CS(upload(h, &d.dinv, c.dinv));
    CS(upload(h, &d.seg_ptr, c.seg_ptr));
    CS(upload(h, &d.seg_row, c.seg_row));
    d.lev_ptask_ptr = c.lev_ptask_ptr;
    d.lev_sn_ptr = c.lev_sn_ptr;
    d.lev_small = c.lev_small;
    CS(upload(h, &d.lev_sn, c.lev_sn));
    // the persistent solves read the level tables on the device; they run
    // nsteps dependent steps (a grid barrier between consecutive ones)
    CS(upload(h, &d.d_lev_task_ptr, c.lev_task_ptr));
    CS(upload(h, &d.d_lev_ptask_ptr, c.lev_ptask_ptr));
    CS(upload(h, &d.d_lev_sn_ptr, c.lev_sn_ptr));
    CS(upload(h, &d.d_lev_small, c.lev_small));
    d.nsteps_fwd = d.nsteps_bwd = 0;
    d.max_cta_tasks = 1;
    for (int32_t l = 0; l < c.top_lev; ++l) {   // the top zone is not level-stepped
        const int32_t nt = c.lev_task_ptr[l + 1] - c.lev_task_ptr[l], np = c.lev_ptask_ptr[l + 1] - c.lev_ptask_ptr[l];
        const int32_t ns = c.lev_sn_ptr[l + 1] - c.lev_sn_ptr[l];
        if (c.lev_small[l]) {
            d.nsteps_fwd += ns > 0;
            d.nsteps_bwd += ns > 0;
            d.max_cta_tasks = std::max(d.max_cta_tasks, ns);
            continue;
        }
        d.nsteps_fwd += nt + np > 0;
        d.nsteps_bwd += nt > 0;
        d.max_cta_tasks = std::max(d.max_cta_tasks, nt + np);
    }
    // fused levels stage a supernode's [L_JJ^{-1}; M_J] in shared memory when it fits
    // 36 KB (the rest of the 48 KB default holds the kernels' static arrays); the
    // forward stages the panel with an odd row stride (n_J | 1), so sizes count it
    {
        const int64_t capmax = 36 * 1024 / (int64_t)sizeof(T);
        d.lev_stage.assign(c.nlev, 0);
        d.stage_cap = 0;
        for (int32_t l = 0; l < c.nlev; ++l) {
            if (!c.lev_small[l]) continue;
            int64_t mx = 0;
            for (int32_t q = c.lev_sn_ptr[l]; q < c.lev_sn_ptr[l + 1]; ++q) {
                const int32_t J = c.lev_sn[q];
                const int64_t nJ = c.c0[J + 1] - c.c0[J], nr = c.r_off[J + 1] - c.r_off[J];
                mx = std::max(mx, nJ * (nJ + 1) / 2 + nr * (nJ | 1));
            }
            d.lev_stage[l] = (int32_t)std::min(mx, capmax);
            d.stage_cap = std::max(d.stage_cap, d.lev_stage[l]);
        }
    }
    CS(dalloc(h, &d.bar, 1));
    d.err = op.err;
    if (h->opts.spin_limit > 0) d.grid_spin = h->opts.spin_limit;
    d.per_level = h->opts.c_persistent != 1;   // per-level launches unless the persistent solve is asked for
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            d.nsm = nsm;
    }
    d.nrow = (int64_t)c.rows.size();
    d.max_n = 1;
    for (int32_t J = 0; J < c.ns; ++J) d.max_n = std::max(d.max_n, c.c0[J + 1] - c.c0[J]);
    // a forward task holds t_J (max_n values) and a 32 x 33 reduction array in shared memory
    if (((size_t)d.max_n + 32 * 33) * sizeof(T) > 48 * 1024) {
        set_error("a separator of C has " + std::to_string(d.max_n) + " nodes, beyond the C-solve kernels' limit");
        return SLR_ERR_UNSUPPORTED;
    }
    CS(dalloc(h, &d.tasks, c.tasks.size() / 4));
    if (!c.tasks.empty())
        CK(cudaMemcpyAsync(d.tasks, c.tasks.data(), c.tasks.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CS(dalloc(h, &d.ptasks, c.ptasks.size() / 4));
    if (!c.ptasks.empty())
        CK(cudaMemcpyAsync(d.ptasks, c.ptasks.data(), c.ptasks.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                           h->stream));
    CS(dalloc(h, &d.wbuf, (size_t)std::max<int64_t>(d.nrow, 1) * r));
    CS(dalloc(h, &d.tws, (size_t)std::max<int64_t>(c.s, 1) * r));
    CS(dalloc(h, &d.gfs, (size_t)std::max<int64_t>(c.s, 1) * r));
    d.lev_maxn.assign(c.nlev, 0);
    for (int32_t l = 0; l < c.nlev; ++l) {
        if (c.lev_small[l]) continue;
        for (int32_t q = c.lev_sn_ptr[l]; q < c.lev_sn_ptr[l + 1]; ++q) {
            const int32_t J = c.lev_sn[q];
            d.lev_maxn[l] = std::max(d.lev_maxn[l], c.c0[J + 1] - c.c0[J]);
        }
    }
    d.ws_cols = r;
    // top zone: explicit inverse in both layouts, task tables and workspaces
    d.top_lev = c.top_lev;
    d.nT = c.nT;
    if (c.nT > 0) {
        CS(upload(h, &d.tpos, c.tpos));
        CS(upload(h, &d.tseg_ptr, c.tseg_ptr));
        CS(upload(h, &d.tseg_row, c.tseg_row));
        CS(upload(h, &d.tsk_off, c.tsk_off));
        CS(upload(h, &d.tsk_lo, c.tsk_lo));
        CS(upload(h, &d.tsk, c.tsk));
        CS(upload(h, &d.tb_off, c.tb_off));
        CS(upload(h, &d.tb, c.tb));
        CS(upload(h, &d.tp_off, c.tp_off));
        CS(upload(h, &d.tp_pos, c.tp_pos));
        CS(upload(h, &d.tb_cb_part, c.tb_cb_part));
        auto upload4 = [&](int4** p, const std::vector<int32_t>& v, int32_t* count) -> slr_status {
            *count = (int32_t)(v.size() / 4);
            CS(dalloc(h, p, v.size() / 4));
            if (!v.empty())
                CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
            return SLR_OK;
        };
        CS(upload4(&d.tf_rb, c.tf_rb, &d.n_tf_rb));
        CS(upload4(&d.tf_tasks, c.tf_tasks, &d.n_tf_tasks));
        CS(upload4(&d.tb_cb, c.tb_cb, &d.n_tb_cb));
        CS(upload4(&d.tb_tasks, c.tb_tasks, &d.n_tb_tasks));
        d.tf_parts = c.tf_parts;
        d.tb_parts = c.tb_parts;
        CS(dalloc(h, &d.tT, (size_t)c.nT * r));
        CS(dalloc(h, &d.tf_part, (size_t)c.tf_parts * r));
        CS(dalloc(h, &d.tb_part, (size_t)c.tb_parts * r));
        CS(dalloc(h, &d.tf_cnt, (size_t)d.n_tf_rb));
        CS(dalloc(h, &d.tb_cnt, (size_t)d.n_tb_cb));
        CK(cudaMemsetAsync(d.tf_cnt, 0, sizeof(int32_t) * d.n_tf_rb, h->stream));
        CK(cudaMemsetAsync(d.tb_cnt, 0, sizeof(int32_t) * d.n_tb_cb, h->stream));
    }
    const int64_t n = hs.n, nI = hs.nI, s = hs.s;
    if constexpr (!std::is_same<T, double>::value) {
        CS(dalloc(h, &op.wr, (size_t)n * r));
        CS(dalloc(h, &op.wz, (size_t)n * r));
    }
    CS(dalloc(h, &op.tB, (size_t)std::max<int64_t>(nI, 1) * r));
    CS(dalloc(h, &op.eb, (size_t)std::max<int64_t>(nI, 1) * r));
    CS(dalloc(h, &op.gp, (size_t)std::max<int64_t>(s, 1) * r));
    CS(dalloc(h, &op.wf, (size_t)std::max<int64_t>(s, 1) * r));
    CS(dalloc(h, &op.xf, (size_t)std::max<int64_t>(s, 1) * r));
    return SLR_OK;
}

// Low-rank data of one operator: U (s x k, factor order), d, 1/(1-theta).
template <typename T>
slr_status set_operator_lowrank(slr_handle h, DevOperator<T>& op, const double* U64_dev, int32_t k_old,
                                int32_t k, const std::vector<double>& lam, double theta) {
    const int64_t s = h->hs.s;
    const int32_t r = std::max(1, h->opts.nrhs_max);
    if (op.U_tc_rm) {   // the tensor-core copies are rebuilt below
        const size_t eb = lowrank_tc_elem(op.u_dtype) * (size_t)s * k_old;
        dfree(h, reinterpret_cast<char*&>(op.U_tc_rm), eb);
        if (op.U_tc_cm) dfree(h, reinterpret_cast<char*&>(op.U_tc_cm), eb);
    }
    if (op.Zdd) dfree(h, op.Zdd, (size_t)s * k_old);
    if (op.U && k_old != k) {
        dfree(h, op.U, (size_t)s * k_old);
        dfree(h, op.dvec, (size_t)k_old);
        dfree(h, op.vk, (size_t)k_old * r);
        dfree(h, op.part, (size_t)lowrank_part_elems((int32_t)s, k_old, r));
    }
    if (!op.U && k > 0) {
        CS(dalloc(h, &op.U, (size_t)s * k));
        CS(dalloc(h, &op.dvec, (size_t)k));
        CS(dalloc(h, &op.vk, (size_t)k * r));
        CS(dalloc(h, &op.part, (size_t)lowrank_part_elems((int32_t)s, k, r)));
    }
    if (k > 0) {
        if constexpr (std::is_same<T, double>::value) {
            if ((void*)op.U != (void*)U64_dev)
                CK(cudaMemcpyAsync(op.U, U64_dev, sizeof(double) * s * k, cudaMemcpyDeviceToDevice, h->stream));
        } else {
            CK(launch_convert<double, float>(s, k, U64_dev, s, op.U, s, h->stream));
            op.u_dtype = h->opts.u_dtype;
            if (op.u_dtype != SLR_U_FP32 && k <= 128) {
                const size_t eb = lowrank_tc_elem(op.u_dtype) * (size_t)s * k;
                char *rm = nullptr, *cm = nullptr;
                CS(dalloc(h, &rm, eb));
                if (op.u_dtype == SLR_U_BF16) CS(dalloc(h, &cm, eb));
                op.U_tc_rm = rm;
                op.U_tc_cm = cm;
                CK(launch_lowrank_tc_pack(op.u_dtype, (int32_t)s, k, U64_dev, rm, cm, h->stream));
            }
        }
        if (h->opts.zform) {
            // Z_k = L^{-T} U_k (Proposition 4.3) with the FP64 factor, scattered to DD order,
            // at most nrhs_max columns at a time (the solves' workspaces hold that many)
            double* Z64 = nullptr;
            CS(dalloc(h, &Z64, (size_t)s * k));
            for (int32_t c0 = 0; c0 < k; c0 += r)
                CK(launch_c_backward<double>(h->op64.cf, U64_dev + (int64_t)c0 * s, h->op64.xf, Z64 + (int64_t)c0 * s,
                                             s, std::min(r, k - c0), h->stream));
            if constexpr (std::is_same<T, double>::value) {
                op.Zdd = Z64;
            } else {
                CS(dalloc(h, &op.Zdd, (size_t)s * k));
                CK(launch_convert<double, float>(s, k, Z64, s, op.Zdd, s, h->stream));
                CK(cudaStreamSynchronize(h->stream));
                dfree(h, Z64, (size_t)s * k);
            }
        }
        // d_i = (1 - lambda_i)^{-1} - (1 - theta)^{-1}, formed in FP64 (cancellation near 1)
        std::vector<double> d(k);
        for (int32_t i = 0; i < k; ++i) d[i] = 1.0 / (1.0 - lam[i]) - 1.0 / (1.0 - theta);
        std::vector<T> dt(d.begin(), d.end());
        CK(cudaMemcpyAsync(op.dvec, dt.data(), sizeof(T) * k, cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    op.cinv = (T)(1.0 / (1.0 - theta));
    return SLR_OK;
}

// z = M^{-1} r in precision T; r, z in DD order (Eq. 4.1 with the block LU of Eq. 2.4)
template <typename T>
slr_status run_apply(slr_handle h, DevOperator<T>& op, const T* r, int64_t ldr, T* z, int64_t ldz,
                     int32_t nrhs, cudaStream_t st) {
    const HostSetup& hs = h->hs;
    const int32_t nI = hs.nI, s = hs.s;
    CK(launch_band_solve<T>(op, hs.p, hs.wmax, r, ldr, op.tB, nI, nullptr, 0, nrhs, st));   // t = B^{-1} f
    CK(launch_gather_et<T>(op, s, r + nI, ldr, op.tB, nI, op.gp, s, nrhs, st));              // g' = g - E^T t
    if (op.Zdd && h->k > 0) {
        // Z-form (Proposition 4.3, Eq. 4.15): v = d o Z_k^T g' on the side stream while
        // y = C^{-1} g' runs, then y = (1-theta)^{-1} y + Z_k v
        CK(cudaEventRecord(h->ev_fork, st));
        CK(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
        CK(launch_lowrank_v<T>(op, s, h->k, op.Zdd, op.gp, s, nrhs, h->aux));
        CK(cudaEventRecord(h->ev_join, h->aux));
        CK(launch_c_forward<T>(op.cf, op.gp, s, op.wf, nrhs, st));                           // L^{-1} g'
        CK(launch_c_backward<T>(op.cf, op.wf, op.xf, z + nI, ldz, nrhs, st));                // C^{-1} g'
        CK(cudaStreamWaitEvent(st, h->ev_join, 0));
        CK(launch_lowrank_update<T>(op, s, h->k, op.Zdd, z + nI, ldz, nrhs, st));
    } else {
        CK(launch_c_forward<T>(op.cf, op.gp, s, op.wf, nrhs, st));                           // w = L^{-1} g'
        CK(launch_lowrank<T>(op, s, h->k, op.wf, nrhs, st));                                 // w' (Eq. 4.7)
        CK(launch_c_backward<T>(op.cf, op.wf, op.xf, z + nI, ldz, nrhs, st));                // y = L^{-T} w'
    }
    CK(launch_spmv_e<T>(op, nI, z + nI, ldz, op.eb, nI, nrhs, st));                          // E y
    CK(launch_band_solve<T>(op, hs.p, hs.wmax, op.eb, nI, z, ldz, op.tB, nI, nrhs, st));    // u = t - B^{-1} E y
    return SLR_OK;
}

slr_status apply_any(slr_handle h, const double* r, int64_t ldr, double* z, int64_t ldz, int32_t nrhs,
                     cudaStream_t st) {
    if (h->opts.precision == SLR_PREC_FP64) return run_apply<double>(h, h->op64, r, ldr, z, ldz, nrhs, st);
    DevOperator<float>& op = h->op32;
    const int64_t n = h->hs.n;
    CK(launch_convert<double, float>(n, nrhs, r, ldr, op.wr, n, st));
    CS(run_apply<float>(h, op, op.wr, n, op.wz, n, nrhs, st));
    CK(launch_convert<float, double>(n, nrhs, op.wz, n, z, ldz, st));
    return SLR_OK;
}

// w = H v, H = L^{-1} E^T B^{-1} E L^{-T} (Eq. 3.2), FP64, v and w in factor order (length s)
slr_status h_apply(slr_handle h, const double* v, double* w, cudaStream_t st) {
    DevOperator<double>& op = h->op64;
    const int32_t nI = h->hs.nI, s = h->hs.s;
    CK(launch_c_backward<double>(op.cf, v, op.xf, op.gp, s, 1, st));       // y = L^{-T} v (DD in gp)
    CK(launch_spmv_e<double>(op, nI, op.gp, s, op.eb, nI, 1, st));         // E y
    CK(launch_band_solve<double>(op, h->hs.p, h->hs.wmax, op.eb, nI, op.tB, nI, nullptr, 0, 1, st));
    CK(launch_gather_et<double>(op, s, nullptr, 0, op.tB, nI, op.gp, s, 1, st));  // E^T B^{-1} E y
    CK(launch_c_forward<double>(op.cf, op.gp, s, w, 1, st));         // L^{-1} (...)
    return SLR_OK;
}

double read_scalar(const double* dev, cudaStream_t st, slr_status* err) {
    double v = 0.0;
    if (cudaMemcpyAsync(&v, dev, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *err = SLR_ERR_CUDA;
        set_error("device to host copy failed");
    }
    return v;
}

// The operator's device status word: cleared on the call's stream before its
// kernels, read (synchronising) after them.
int32_t* status_word(slr_handle h) { return h->opts.precision == SLR_PREC_FP64 ? h->op64.err : h->op32.err; }

slr_status clear_status(slr_handle h, cudaStream_t st) {
    CK(cudaMemsetAsync(h->op64.err, 0, sizeof(int32_t), st));
    if (h->op32.err && h->op32.err != h->op64.err) CK(cudaMemsetAsync(h->op32.err, 0, sizeof(int32_t), st));
    return SLR_OK;
}

slr_status read_status(slr_handle h, const int32_t* word, cudaStream_t st) {
    int32_t e = 0;
    CK(cudaMemcpyAsync(&e, word, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (e) {
        set_error(e == 2   ? "a bounded grid-barrier wait expired in the C solve"
                  : e == 3 ? "a bounded tensor-core completion wait expired in the low-rank products"
                           : "a bounded device wait expired in the band solve");
        return SLR_ERR_TIMEOUT;
    }
    (void)h;
    return SLR_OK;
}

// Section 5.1: m steps of Lanczos with full reorthogonalisation on H, Ritz pairs,
// U_k = V Y_k, theta.  Start vector v_1 = L^{-1} C z / ||.||, z from SplitMix64.
slr_status run_lanczos(slr_handle h, cudaStream_t st) {
    const int32_t s = h->hs.s;
    int32_t k = std::min(h->opts.k, s);
    if (k <= 0 || s == 0) {
        h->k = 0;
        h->theta = 0.0;
        h->nritz = 0;
        return SLR_OK;
    }
    const int32_t m = std::min(h->opts.lanczos_steps > 0 ? h->opts.lanczos_steps : 5 * k, s);
    DevOperator<double>& op = h->op64;
    double *V = nullptr, *w = nullptr, *hv = nullptr, *part = nullptr, *sc = nullptr, *Yd = nullptr, *Ud = nullptr;
    CS(dalloc(h, &V, (size_t)s * m));
    CS(dalloc(h, &w, (size_t)s));
    CS(dalloc(h, &hv, (size_t)m));
    CS(dalloc(h, &part, (size_t)m * kRedBlocks));
    CS(dalloc(h, &sc, 4));
    std::vector<double> z(s);
    for (int32_t i = 0; i < s; ++i) z[i] = splitmix_pm1(h->opts.seed, (uint64_t)i);
    CK(cudaMemcpyAsync(w, z.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
    CK(launch_csr_spmv(s, h->c_rp, h->c_ci, h->c_v, w, s, op.gp, s, 1, st));     // C z (DD order)
    CK(launch_c_forward<double>(op.cf, op.gp, s, V, 1, st));              // L^{-1} C z
    slr_status err = SLR_OK;
    CK(launch_dots(s, 1, V, s, V, s, part, sc, 1, st));
    double nrm = std::sqrt(read_scalar(sc, st, &err));
    CS(err);
    if (!(nrm > 0.0)) { set_error("Lanczos start vector is zero"); return SLR_ERR_BREAKDOWN; }
    CK(launch_axpby(s, 0.0, V, 1.0 / nrm, V, st));
    std::vector<double> alpha(m), beta(m);
    int32_t m_eff = m;
    double amax = 0.0;
    // time split (both reads synchronise the stream): H applies with the alpha dot,
    // reorthogonalisation with the beta norm, then the host eigensolve and U_k = V Y_k
    double ta = 0.0, tr = 0.0, tcur = now_s();
    for (int32_t j = 0; j < m; ++j) {
        double* vj = V + (int64_t)j * s;
        CS(h_apply(h, vj, w, st));
        if (j > 0) CK(launch_axpby(s, -beta[j - 1], V + (int64_t)(j - 1) * s, 1.0, w, st));
        CK(launch_dots(s, 1, vj, s, w, s, part, sc, 1, st));
        alpha[j] = read_scalar(sc, st, &err);
        CS(err);
        ta += now_s() - tcur;
        tcur = now_s();
        amax = std::max(amax, std::fabs(alpha[j]));
        CK(launch_axpby(s, -alpha[j], vj, 1.0, w, st));
        for (int pass = 0; pass < 2; ++pass) {                       // full reorthogonalisation
            CK(launch_gemv_t(s, j + 1, V, w, part, hv, st));
            CK(launch_gemv_n_sub(s, j + 1, V, hv, w, st));
        }
        CK(launch_dots(s, 1, w, s, w, s, part, sc, 1, st));
        beta[j] = std::sqrt(read_scalar(sc, st, &err));
        CS(err);
        tr += now_s() - tcur;
        tcur = now_s();
        if (j + 1 == m) break;
        if (beta[j] <= 1e-12 * amax) { m_eff = j + 1; break; }
        CK(launch_axpby(s, 1.0 / beta[j], w, 0.0, V + (int64_t)(j + 1) * s, st));
    }
    CS(read_status(h, op.err, st));                // the H applies ran without an expired wait
    const double te0 = now_s();
    std::vector<double> lam(m_eff), Y((size_t)m_eff * m_eff);
    host_tridiag_eig(m_eff, alpha.data(), beta.data(), lam.data(), Y.data());
    k = std::min(k, m_eff);
    if (h->opts.target_kappa >= 2) {
        // rank rule of Section 4 (Eq. condk): the condition number of S S~^{-1} stays
        // below K when lambda_{k+1} <= 1 - 1/K; keep the Ritz values above 1 - 1/K
        const double thr = 1.0 - 1.0 / (double)h->opts.target_kappa;
        int32_t cnt = 0;
        while (cnt < m_eff && lam[cnt] > thr) ++cnt;   // descending
        k = std::min(k, cnt);
    }
    h->ritz = lam;
    h->nritz = m_eff;
    h->m_steps = m_eff;
    // theta = lambda_{k+1} (Eq. 4.11) while it is below 1; an indefinite B can give H
    // eigenvalues >= 1, where it would flip the sign of the C^{-1} term: then theta = 0
    h->theta = (h->opts.theta_mode == SLR_THETA_LAMBDA_K1 && m_eff > k && lam[k] < 1.0) ? lam[k] : 0.0;
    h->lam.assign(lam.begin(), lam.begin() + k);
    CS(dalloc(h, &Yd, (size_t)m_eff * k));
    CK(cudaMemcpyAsync(Yd, Y.data(), sizeof(double) * m_eff * k, cudaMemcpyHostToDevice, st));
    CS(dalloc(h, &Ud, (size_t)s * k));
    CK(launch_gemm_nn(s, m_eff, k, V, Yd, Ud, st));
    CK(cudaStreamSynchronize(st));
    h->lanczos_seconds[0] = ta;
    h->lanczos_seconds[1] = tr;
    h->lanczos_seconds[2] = now_s() - te0;
    CS(set_operator_lowrank<double>(h, op, Ud, 0, k, h->lam, h->theta));
    h->k = k;
    dfree(h, Ud, (size_t)s * k);
    dfree(h, Yd, (size_t)m_eff * k);
    dfree(h, V, (size_t)s * m);
    dfree(h, w, (size_t)s);
    dfree(h, hv, (size_t)m);
    dfree(h, part, (size_t)m * kRedBlocks);
    dfree(h, sc, 4);
    return SLR_OK;
}

void drop_graphs(slr_handle h);

// Section 5.3: append eigenvector estimates of H found by Lanczos on the
// deflated operator P H P, P = I - U_k U_k^T (all FP64, as the setup Lanczos).
slr_status run_lanczos_deflated(slr_handle h, int32_t k_add, int32_t steps, cudaStream_t st, int32_t* added) {
    HostSetup& hs = h->hs;
    const int32_t s = hs.s, k = h->k;
    *added = 0;
    if (k_add == 0 || s == 0) return SLR_OK;
    const int32_t m = std::min(steps > 0 ? steps : 5 * k_add, s - k);
    if (m <= 0) return SLR_OK;
    DevOperator<double>& op = h->op64;
    // the mixed path keeps only the FP32 band factor after setup: reload the FP64 one for the run
    const bool reload = op.bfac == nullptr;
    if (reload && hs.bfac.empty()) {                // never launch the band solve without its factor
        set_error("slr_add_vectors: the FP64 band factor is not available on this handle");
        return SLR_ERR_UNSUPPORTED;
    }
    if (reload) {
        dfree(h, op.band, hs.band.size());
        CS(upload_band(h, &op.band));
        CS(upload(h, &op.bfac, hs.bfac));
        op.band_G = hs.band_G;
    }
    const int32_t mk = std::max(m, k);
    double *V = nullptr, *w = nullptr, *hv = nullptr, *part = nullptr, *sc = nullptr, *Yd = nullptr, *Un = nullptr;
    CS(dalloc(h, &V, (size_t)s * m));
    CS(dalloc(h, &w, (size_t)s));
    CS(dalloc(h, &hv, (size_t)mk));
    CS(dalloc(h, &part, (size_t)mk * kRedBlocks));
    CS(dalloc(h, &sc, 4));
    auto project = [&](double* x) -> slr_status {       // x -= U (U^T x), two passes
        for (int pass = 0; pass < 2 && k > 0; ++pass) {
            CK(launch_gemv_t(s, k, op.U, x, part, hv, st));
            CK(launch_gemv_n_sub(s, k, op.U, hv, x, st));
        }
        return SLR_OK;
    };
    h->improvements += 1;
    std::vector<double> z(s);
    for (int32_t i = 0; i < s; ++i) z[i] = splitmix_pm1(h->opts.seed + (uint64_t)h->improvements, (uint64_t)i);
    CK(cudaMemcpyAsync(w, z.data(), sizeof(double) * s, cudaMemcpyHostToDevice, st));
    CK(launch_csr_spmv(s, h->c_rp, h->c_ci, h->c_v, w, s, op.gp, s, 1, st));     // C z (DD order)
    CK(launch_c_forward<double>(op.cf, op.gp, s, V, 1, st));              // L^{-1} C z
    CS(project(V));
    slr_status err = SLR_OK;
    CK(launch_dots(s, 1, V, s, V, s, part, sc, 1, st));
    const double nrm = std::sqrt(read_scalar(sc, st, &err));
    CS(err);
    if (!(nrm > 0.0)) { set_error("deflated Lanczos start vector is zero"); return SLR_ERR_BREAKDOWN; }
    CK(launch_axpby(s, 0.0, V, 1.0 / nrm, V, st));
    std::vector<double> alpha(m), beta(m);
    int32_t m_eff = m;
    double amax = 0.0;
    for (int32_t j = 0; j < m; ++j) {
        double* vj = V + (int64_t)j * s;
        CS(h_apply(h, vj, w, st));
        CS(project(w));
        if (j > 0) CK(launch_axpby(s, -beta[j - 1], V + (int64_t)(j - 1) * s, 1.0, w, st));
        CK(launch_dots(s, 1, vj, s, w, s, part, sc, 1, st));
        alpha[j] = read_scalar(sc, st, &err);
        CS(err);
        amax = std::max(amax, std::fabs(alpha[j]));
        CK(launch_axpby(s, -alpha[j], vj, 1.0, w, st));
        for (int pass = 0; pass < 2; ++pass) {                       // full reorthogonalisation
            CK(launch_gemv_t(s, j + 1, V, w, part, hv, st));
            CK(launch_gemv_n_sub(s, j + 1, V, hv, w, st));
        }
        CK(launch_dots(s, 1, w, s, w, s, part, sc, 1, st));
        beta[j] = std::sqrt(read_scalar(sc, st, &err));
        CS(err);
        if (j + 1 == m) break;
        if (beta[j] <= 1e-12 * amax) { m_eff = j + 1; break; }
        CK(launch_axpby(s, 1.0 / beta[j], w, 0.0, V + (int64_t)(j + 1) * s, st));
    }
    CS(read_status(h, op.err, st));
    std::vector<double> lam2(m_eff), Y((size_t)m_eff * m_eff);
    host_tridiag_eig(m_eff, alpha.data(), beta.data(), lam2.data(), Y.data());
    const int32_t ja = std::min(k_add, m_eff), kn = k + ja;
    // U_new = [U_k | V Y_ja]
    CS(dalloc(h, &Yd, (size_t)m_eff * ja));
    CK(cudaMemcpyAsync(Yd, Y.data(), sizeof(double) * m_eff * ja, cudaMemcpyHostToDevice, st));
    CS(dalloc(h, &Un, (size_t)s * kn));
    if (k > 0) CK(cudaMemcpyAsync(Un, op.U, sizeof(double) * s * k, cudaMemcpyDeviceToDevice, st));
    CK(launch_gemm_nn(s, m_eff, ja, V, Yd, Un + (int64_t)s * k, st));
    CK(cudaStreamSynchronize(st));
    std::vector<double> lam_new(h->lam);
    lam_new.insert(lam_new.end(), lam2.begin(), lam2.begin() + ja);
    const double theta =
        (h->opts.theta_mode == SLR_THETA_LAMBDA_K1 && m_eff > ja && lam2[ja] < 1.0) ? lam2[ja] : 0.0;
    {
        std::unique_lock<std::shared_mutex> lk(g_capture_mu);
        drop_graphs(h);
    }
    CS(set_operator_lowrank<double>(h, h->op64, Un, k, kn, lam_new, theta));
    if (h->opts.precision == SLR_PREC_MIXED) CS(set_operator_lowrank<float>(h, h->op32, Un, k, kn, lam_new, theta));
    h->k = kn;
    h->lam = lam_new;
    h->theta = theta;
    h->ritz = lam_new;
    h->ritz.insert(h->ritz.end(), lam2.begin() + ja, lam2.end());
    h->nritz = (int32_t)h->ritz.size();
    h->m_steps = std::max(h->m_steps, h->nritz);
    dfree(h, Un, (size_t)s * kn);
    dfree(h, Yd, (size_t)m_eff * ja);
    dfree(h, V, (size_t)s * m);
    dfree(h, w, (size_t)s);
    dfree(h, hv, (size_t)mk);
    dfree(h, part, (size_t)mk * kRedBlocks);
    dfree(h, sc, 4);
    if (reload) dfree(h, op.bfac, hs.bfac.size());
    *added = ja;
    return SLR_OK;
}

void account(slr_handle h) {
    const HostSetup& hs = h->hs;
    const bool fp64 = h->opts.precision == SLR_PREC_FP64;
    const int64_t wf = fp64 ? 8 : 4, wv = fp64 ? 8 : 4;
    int64_t band = 0;
    for (const BandBlock& b : hs.band) band += (int64_t)b.c * b.w * (b.w + 1);
    const int64_t nnzE = (int64_t)hs.e_v.size();
    const int64_t cvals = (hs.cf.pan_off.empty() ? 0 : hs.cf.pan_off.back()) +
                          (hs.cf.dinv_off.empty() ? 0 : hs.cf.dinv_off.back());
    const int64_t nseg = hs.cf.seg_ptr.empty() ? 0 : hs.cf.seg_ptr.back();
    const int64_t nrow = (int64_t)hs.cf.rows.size();   // also the w values written and gathered
    const int64_t s = hs.s, k = h->k;
    h->bytes_per_apply = 4 * band * wf + 2 * nnzE * (wf + 4) + 2 * cvals * wf + nseg * (4 + wf) + nrow * (4 + wf) +
                         2 * s * k * wf + (2 * (int64_t)hs.n + 2 * (int64_t)hs.nI) * wv;
    h->flops_per_apply = 2 * (4 * band + 2 * nnzE + 2 * cvals + 2 * s * k);
    h->vector_bytes_per_column = nseg * wf + nrow * wf + (2 * (int64_t)hs.n + 2 * (int64_t)hs.nI) * wv;
}

// ------------------------------------------------------------------ autotuning
// Choices of the band solve (CTAs per subdomain, stream buffers) and of the C
// solve (per-level or persistent), timed on the handle's own apply operator and
// cached per device, precision and problem shape.
struct TuneKey {
    int32_t dev, prec, p, wmax, cmax, nI, s, ns, nlev, nrhs;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, prec, p, wmax, cmax, nI, s, ns, nlev, nrhs) <
               std::tie(o.dev, o.prec, o.p, o.wmax, o.cmax, o.nI, o.s, o.ns, o.nlev, o.nrhs);
    }
};
struct TuneChoice {
    int32_t G = 1, slots = 0, nt = 512;
    bool persistent = false;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

// Average time of `reps` calls of f on stream st after two untimed ones (us).
template <typename F>
slr_status time_us(F f, cudaStream_t st, int reps, double* us) {
    for (int i = 0; i < 2; ++i) CS(f());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, st));
    slr_status r = SLR_OK;
    for (int i = 0; i < reps && r == SLR_OK; ++i) r = f();
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *us = 1e3 * ms / reps;
    return r;
}

// Capture what f launches (on a capture stream) into an executable graph.
template <typename F>
slr_status capture_graph(slr_handle h, F f, cudaGraphExec_t* out) {
    (void)h;
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    slr_status r;
    {
        std::shared_lock<std::shared_mutex> lk(g_capture_mu);
        const int64_t l0 = thread_launches();
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            set_error(std::string("capture: ") + cudaGetErrorString(e));
            return SLR_ERR_CUDA;
        }
        r = f(cs);
        e = cudaStreamEndCapture(cs, &g);
        count_launches(-(thread_launches() - l0));   // captured, not run
        if (r == SLR_OK && e != cudaSuccess) {
            set_error(std::string("capture: ") + cudaGetErrorString(e));
            r = SLR_ERR_CUDA;
        }
    }
    if (r == SLR_OK) {
        const cudaError_t e = cudaGraphInstantiate(out, g, 0);
        if (e != cudaSuccess) {
            set_error(std::string("instantiate: ") + cudaGetErrorString(e));
            r = SLR_ERR_CUDA;
        }
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    return r;
}

// Section 5.2 on the device: the plane blocks of every B_i into h->bf_scr; a
// non-positive pivot returns SLR_ERR_NOT_SPD naming the subdomain.
slr_status device_band_factor(slr_handle h, cudaStream_t st) {
    HostSetup& hs = h->hs;
    const int32_t p = hs.p;
    std::vector<int64_t> soff(p + 1, 0);
    for (int32_t i = 0; i < p; ++i) {
        const BandBlock& b = hs.band[i];
        soff[i + 1] = soff[i] + (b.m ? (int64_t)(1 + 2 * b.c) * b.w * b.w + (int64_t)b.c * b.w : 0);
    }
    h->bf_scr_len = std::max<int64_t>(soff[p], 1);
    CS(dalloc(h, &h->bf_scr, (size_t)h->bf_scr_len));
    CS(upload(h, &h->bf_soff, soff));
    ScopedBuf<BandBlock> dband(h);
    ScopedBuf<int32_t> bad(h);
    CS(dband.alloc(hs.band.size()));
    CK(cudaMemcpyAsync(dband.p, hs.band.data(), sizeof(BandBlock) * hs.band.size(), cudaMemcpyHostToDevice, st));
    CS(bad.alloc(1));
    CK(cudaMemsetAsync(bad.p, 0xff, sizeof(int32_t), st));   // -1: no failure
    CK(launch_band_factor(dband.p, p, h->a_rp, h->a_ci, h->a_v, h->bf_scr, h->bf_soff, bad.p, hs.indefinite, st));
    int32_t hb = -1;
    CK(cudaMemcpyAsync(&hb, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hb >= 0) {
        if (hs.indefinite) {
            set_error("B_" + std::to_string(hb) + " has a zero pivot in its symmetric factorisation");
            return SLR_ERR_BREAKDOWN;
        }
        set_error("B_" + std::to_string(hb) + " is not positive definite (Cholesky pivot <= 0)");
        return SLR_ERR_NOT_SPD;
    }
    return SLR_OK;
}

// The operator's band factor, packed on the device for the current layout (op.band).
template <typename T>
slr_status device_band_pack(slr_handle h, DevOperator<T>& op, cudaStream_t st) {
    HostSetup& hs = h->hs;
    int32_t cmax = 0;
    for (const BandBlock& b : hs.band) cmax = std::max(cmax, b.c);
    CS(dalloc(h, &op.bfac, (size_t)hs.bfac_len));
    CK(cudaMemsetAsync(op.bfac, 0, sizeof(T) * hs.bfac_len, st));
    CK(launch_band_pack<T>(op.band, hs.p, cmax, hs.band_G, h->bf_scr, h->bf_soff, op.bfac, hs.indefinite, st));
    return SLR_OK;
}

// Repack the band factor for G CTAs per subdomain and reload it into the apply
// operator (from the device plane blocks when the B_i were factored there).
template <typename T>
slr_status repack_band(slr_handle h, DevOperator<T>& op, int32_t G) {
    HostSetup& hs = h->hs;
    const size_t old_band = hs.band.size();
    const int64_t old_fac = hs.bfac_len;
    if (h->bf_scr) host_band_layout(hs, G);
    else CS(host_band_factor(hs, G));
    CK(cudaStreamSynchronize(h->stream));
    dfree(h, op.band, old_band);
    dfree(h, op.bfac, (size_t)old_fac);
    CS(upload_band(h, &op.band));
    if (h->bf_scr) CS(device_band_pack<T>(h, op, h->stream));
    else CS(upload(h, &op.bfac, hs.bfac));
    CK(cudaStreamSynchronize(h->stream));
    op.band_G = hs.band_G;
    return SLR_OK;
}

template <typename T>
slr_status autotune(slr_handle h, DevOperator<T>& op, cudaStream_t st) {
    HostSetup& hs = h->hs;
    const auto t0 = std::chrono::steady_clock::now();
    int dev = 0, nsm = 152;
    CK(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int32_t cmax = 0;
    for (const BandBlock& b : hs.band) cmax = std::max(cmax, b.c);
    const TuneKey key{dev, h->opts.precision, hs.p, hs.wmax, cmax, hs.nI, hs.s, hs.cf.ns, hs.cf.nlev,
                      h->opts.nrhs_max};
    TuneChoice best;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    // the candidates are timed on blocks of nrhs_max right-hand sides (the workspaces'
    // width), the block the handle's solves will carry
    const int32_t r = std::max(1, h->opts.nrhs_max);
    if (!cached && hs.p > 0 && hs.wmax > 0) {
        CK(cudaMemsetAsync(op.eb, 0, sizeof(T) * std::max(hs.nI, 1) * r, st));
        CK(cudaMemsetAsync(op.gp, 0, sizeof(T) * std::max(hs.s, 1) * r, st));
        double best_us = 1e30;
        for (int32_t G : {1, 2, 4}) {
            if (!band_split_ok(hs.wmax, G) || (G > 1 && hs.wmax < 32 * G) || hs.p * G > 2 * nsm) continue;
            if (G != hs.band_G) CS(repack_band<T>(h, op, G));
            for (int32_t nt : {512, 256, 32})
                for (int32_t slots : {2, 3, 4}) {
                    // the warp kernel: planes of at most 64 rows in one slice, its own ring
                    if (nt == 32 && (G != 1 || hs.wmax > 64 || slots != 2)) continue;
                    op.band_nbuf = slots;
                    op.band_nt = nt;
                    double us = 0;
                    CS(time_us([&]() -> slr_status {
                        CK(launch_band_solve<T>(op, hs.p, hs.wmax, op.eb, hs.nI, op.tB, hs.nI, nullptr, 0, r, st));
                        return SLR_OK;
                    }, st, 5, &us));
                    if (us < best_us) {
                        best_us = us;
                        best.G = G;
                        best.slots = slots;
                        best.nt = nt;
                    }
                }
        }
        // the C solves run inside the PCG graph: time them as a replayed graph
        double c_us[2] = {0, 0};
        for (int v = 0; v < 2; ++v) {
            op.cf.per_level = (v == 0);
            cudaGraphExec_t ex = nullptr;
            CS(capture_graph(h, [&](cudaStream_t cs) -> slr_status {
                CK(launch_c_forward<T>(op.cf, op.gp, hs.s, op.wf, r, cs));
                CK(launch_c_backward<T>(op.cf, op.wf, op.xf, op.gp, hs.s, r, cs));
                return SLR_OK;
            }, &ex));
            const slr_status rs = time_us([&]() -> slr_status {
                CK(cudaGraphLaunch(ex, st));
                return SLR_OK;
            }, st, 5, &c_us[v]);
            cudaGraphExecDestroy(ex);
            CS(rs);
        }
        // the two paths often time within noise of each other: keep the per-level default
        // unless the persistent one is clearly (5%) faster, so the pick is stable from run to run
        best.persistent = c_us[1] < 0.95 * c_us[0];
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    if (best.G != hs.band_G) CS(repack_band<T>(h, op, best.G));
    op.band_nbuf = best.slots;
    op.band_nt = best.nt;
    hs.band_nt = best.nt;
    op.cf.per_level = !best.persistent;
    h->tuned = true;
    h->tune_seconds = cached ? 0.0 : std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return SLR_OK;
}

slr_status setup_impl(slr_handle h, int32_t n, const int32_t* rowptr, const int32_t* colind, const double* val,
                      int32_t nparts, const int32_t* part, cudaStream_t st) {
    HostSetup& hs = h->hs;
    const bool vb = h->opts.verbose != 0;
    hs.indefinite = h->opts.indefinite == 1;
    double t0 = now_s();
    CS(host_validate_csr(n, rowptr, colind, val, nparts, part));
    CS(host_dd_order(n, rowptr, colind, nparts, part, hs));
    CS(host_split_blocks(rowptr, colind, val, hs));
    double t1 = now_s();
    bool dev_band = false;
    // CTAs per subdomain in the band solve: a slice holds at most 256 rows of a
    // plane; with few subdomains two CTAs (a cluster) share each one so that
    // more SMs stream the factor
    {
        int32_t G = 1;
        int dev = 0, nsm = 152;
        const bool have_dev = cudaGetDevice(&dev) == cudaSuccess;
        if (have_dev) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        else cudaGetLastError();
        // the widest plane decides the minimum split
        int32_t wmx = 0;
        for (int32_t q = 0; q < nparts; ++q) {
            int32_t r0 = hs.int_off[q], m = hs.int_off[q + 1] - r0, w = 0;
            for (int32_t a = r0; a < r0 + m; ++a)
                for (int32_t t = hs.a_rp[a]; t < hs.a_rp[a + 1]; ++t) {
                    int32_t cc = hs.a_ci[t];
                    if (cc >= r0 && cc < r0 + m) w = std::max(w, std::abs(a - cc));
                }
            wmx = std::max(wmx, w);
        }
        while (!band_split_ok(wmx, G) && G < 4) G *= 2;
        if (!band_split_ok(wmx, G)) {
            set_error("a B_i has plane width " + std::to_string(wmx) + " beyond the band kernel's limit (1024)");
            return SLR_ERR_UNSUPPORTED;
        }
        const int32_t req = h->opts.band_split;        // 0 = automatic
        if (req == 1 || req == 2 || req == 4) {
            if (band_split_ok(wmx, req)) G = req;
        } else if (G == 1 && 2 * nparts <= nsm && wmx >= 64) {
            // a subdomain's planes are a dependent chain: with few subdomains two
            // CTAs (a cluster) per subdomain put twice the SMs on it (measured
            // faster in both precisions on 16^3 boxes; four CTAs need two waves)
            G = 2;
        }
        // Section 5.2: factor the B_i on the device when every plane fits its kernel (at
        // most 256 rows), else on the host
        dev_band = have_dev && h->opts.band_factor_host == 0 && wmx > 0 && wmx <= 256;
        if (dev_band) host_band_layout(hs, G);
        else CS(host_band_factor(hs, G));
        // more CTAs than SMs would run in two waves: 256-thread CTAs put two subdomains on an SM;
        // planes of at most 64 rows in one slice take a warp per subdomain
        const bool narrow = G == 1 && wmx <= 64;
        const int32_t nt_req = h->opts.band_threads == 32 && !narrow ? 0 : h->opts.band_threads;
        hs.band_nt = nt_req ? nt_req : narrow ? 32 : (nparts * G > nsm ? 256 : 512);
    }
    double t2 = now_s();
    CS(host_c_factor(hs, h->opts.c_leaf > 0 ? h->opts.c_leaf : 64, 32));
    host_c_top(hs.cf, h->opts.c_levels_only == 1 ? hs.cf.nlev : host_c_top_choose(hs.cf));
    double t3 = now_s();
    if (vb)
        fprintf(stderr, "[slr] n=%d nI=%d s=%d p=%d wmax=%d band=%zu cvals=%zu sn=%d lev=%d | analysis %.3fs B %.3fs C %.3fs\n",
                hs.n, hs.nI, hs.s, hs.p, hs.wmax, hs.bfac.size(), hs.cf.panel.size() + hs.cf.dinv.size(), hs.cf.ns,
                hs.cf.nlev, t1 - t0, t2 - t1, t3 - t2);
    CK(cudaGetDevice(&h->device));
    CS(noalloc_lookup(h));
    if (h->opts.zform) {
        CK(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    CS(upload(h, &h->perm, hs.perm));
    CS(upload(h, &h->a_rp, hs.a_rp));
    CS(upload(h, &h->a_ci, hs.a_ci));
    CS(upload(h, &h->a_v, hs.a_v));
    CS(upload(h, &h->c_rp, hs.c_rp));
    CS(upload(h, &h->c_ci, hs.c_ci));
    CS(upload(h, &h->c_v, hs.c_v));
    double tb = 0.0;   // device band factorization time (part of the B-factor figure)
    h->band_on_device = dev_band;
    if (dev_band) {
        const double tb0 = now_s();
        CS(device_band_factor(h, st));
        tb = now_s() - tb0;
    }
    CS(upload_operator<double>(h, h->op64, !dev_band));
    if (dev_band) CS(device_band_pack<double>(h, h->op64, st));
    const int32_t r = std::max(1, h->opts.nrhs_max);
    const size_t nr = (size_t)std::max(1, n) * r;
    CS(dalloc(h, &h->px, nr));
    CS(dalloc(h, &h->pr, nr));
    if (h->opts.precision == SLR_PREC_MIXED) {
        CS(dalloc(h, &h->pr32, nr));
        CS(dalloc(h, &h->pz32, nr));
    } else {
        CS(dalloc(h, &h->pz, nr));
    }
    CS(dalloc(h, &h->pp, nr));
    CS(dalloc(h, &h->pq, nr));
    CS(dalloc(h, &h->scal, (size_t)8 * r));
    CS(dalloc(h, &h->iflags, (size_t)4 * r + 4));
    CS(dalloc(h, &h->dpart, (size_t)2 * kRedBlocks * r));
    CK(cudaStreamSynchronize(st));
    double t4 = now_s();
    CS(run_lanczos(h, st));
    CK(cudaStreamSynchronize(st));
    double t5 = now_s();
    if (h->opts.precision == SLR_PREC_MIXED) {
        CS(upload_operator<float>(h, h->op32, !dev_band));
        if (dev_band) CS(device_band_pack<float>(h, h->op32, st));
        CS(set_operator_lowrank<float>(h, h->op32, h->op64.U, 0, h->k, h->lam, h->theta));
        // the FP64 band factor served the FP64 Lanczos only
        dfree(h, h->op64.bfac, (size_t)hs.bfac_len);
    }
    if (h->opts.autotune == 1) {
        if (h->opts.precision == SLR_PREC_FP64) CS(autotune<double>(h, h->op64, st));
        else CS(autotune<float>(h, h->op32, st));
    }
    if (dev_band && h->opts.band_mma != 0 && h->opts.precision == SLR_PREC_MIXED) {
        // the tensor-core band solve's factor, packed from the same plane blocks; its
        // table follows the launch order of the CUDA-core kernel's clusters
        DevOperator<float>& op = h->op32;
        int32_t cmax = 0;
        for (const BandBlock& b : hs.band) cmax = std::max(cmax, b.c);
        const std::vector<BandTcBlock> tcb = band_tc_layout(
            band_run_order(hs.band, h->opts.band_order ? h->opts.band_order : kBandOrderAuto), h->opts.band_mma,
            &op.band_tc_bytes);
        CS(upload(h, &op.band_tc, tcb));
        CS(dalloc(h, &op.band_tc_fac, (size_t)op.band_tc_bytes));
        CK(launch_band_tc_pack(h->opts.band_mma, op.band_tc, hs.p, cmax, h->bf_scr, h->bf_soff, op.band_tc_fac,
                               hs.indefinite, st));
        op.band_mma = h->opts.band_mma;
        op.band_tc_wmax = hs.wmax;
    }
    if (dev_band) {
        // a mixed-precision handle keeps an FP64 copy of the band factor on the host
        // for slr_add_vectors (packed for the final layout); the plane blocks go
        if (h->opts.precision == SLR_PREC_MIXED) {
            double* tmp = nullptr;
            CS(dalloc(h, &tmp, (size_t)hs.bfac_len));
            CK(cudaMemsetAsync(tmp, 0, sizeof(double) * hs.bfac_len, st));
            int32_t cmax = 0;
            for (const BandBlock& b : hs.band) cmax = std::max(cmax, b.c);
            CK(launch_band_pack<double>(h->op32.band, hs.p, cmax, hs.band_G, h->bf_scr, h->bf_soff, tmp,
                                        hs.indefinite, st));
            hs.bfac.assign((size_t)hs.bfac_len, 0.0);
            CK(cudaMemcpyAsync(hs.bfac.data(), tmp, sizeof(double) * hs.bfac_len, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            dfree(h, tmp, (size_t)hs.bfac_len);
        }
        CK(cudaStreamSynchronize(st));
        dfree(h, h->bf_scr, (size_t)h->bf_scr_len);
        dfree(h, h->bf_soff, (size_t)hs.p + 1);
    }
    CK(cudaStreamSynchronize(st));
    double t6 = now_s();
    h->setup_seconds[0] = t1 - t0;
    h->setup_seconds[1] = t2 - t1 + tb;
    h->setup_seconds[2] = t3 - t2;
    h->setup_seconds[3] = (t4 - t3 - tb) + (t6 - t5);
    h->setup_seconds[4] = t5 - t4;
    account(h);
    if (vb)
        fprintf(stderr, "[slr] upload %.3fs lanczos %.3fs (m=%d k=%d theta=%.6g) device %.1f MB\n", t4 - t3 + t6 - t5,
                t5 - t4, h->m_steps, h->k, h->theta, h->device_bytes / 1e6);
    // host copies of the big factors are no longer needed, except the FP64 band
    // factor of a mixed-precision handle: slr_add_vectors runs its FP64 Lanczos on it
    if (h->opts.precision == SLR_PREC_FP64) std::vector<double>().swap(hs.bfac);
    std::vector<double>().swap(hs.cf.panel);
    std::vector<double>().swap(hs.cf.dinv);
    std::vector<double>().swap(hs.cf.tsk);
    std::vector<double>().swap(hs.cf.tb);
    h->op64.ready = true;
    h->op32.ready = h->opts.precision == SLR_PREC_MIXED;
    return SLR_OK;
}

slr_status check_handle(slr_handle h) {
    if (!h || !h->op64.ready) { set_error("invalid handle"); return SLR_ERR_INVALID_ARG; }
    return SLR_OK;
}


// One CG iteration is split in two parts (Section 6, preconditioned CG):
//   update (every iteration after the first): z = M^{-1} r, rho' = r.z, beta, p = z + beta p
//   test:   q = A p, alpha = rho / p.q, x += alpha p, r -= alpha q, r.r, convergence
// The flexible beta (rho' - r.z_old) / rho takes r.z_old from the test part, which
// forms it with the new r and the z still in place before the next apply replaces
// it (no copy of z is kept).  With the single-precision preconditioner the CG
// vectors stay FP64, the apply reads r rounded to FP32 (written by the r update)
// and its z stays in FP32: widening z to FP64 is exact, so every product with it
// equals the one with the converted vector.
slr_status pcg_apply(slr_handle h, int32_t nrhs, cudaStream_t st) {
    const int64_t nn = h->hs.n;
    if (h->opts.precision == SLR_PREC_FP64) return run_apply<double>(h, h->op64, h->pr, nn, h->pz, nn, nrhs, st);
    return run_apply<float>(h, h->op32, h->pr32, nn, h->pz32, nn, nrhs, st);
}

slr_status pcg_update_part(slr_handle h, int32_t nrhs, cudaStream_t st) {
    const int64_t nn = h->hs.n;
    CS(pcg_apply(h, nrhs, st));
    if (h->pz32) {
        CK(launch_pcg_dot<float>(nn, nrhs, h->pr, h->pz32, h->dpart, h->scal + 6, 8, st));   // rho_new
        CK(launch_pcg_beta(nrhs, h->scal, h->iflags, h->opts.flexible_cg, st));
        CK(launch_pcg_update_pz<float>(nn, nrhs, h->pp, h->pz32, h->scal, h->iflags, st));
    } else {
        CK(launch_pcg_dot<double>(nn, nrhs, h->pr, h->pz, h->dpart, h->scal + 6, 8, st));
        CK(launch_pcg_beta(nrhs, h->scal, h->iflags, h->opts.flexible_cg, st));
        CK(launch_pcg_update_pz<double>(nn, nrhs, h->pp, h->pz, h->scal, h->iflags, st));
    }
    return SLR_OK;
}

slr_status pcg_test_part(slr_handle h, int32_t nrhs, cudaStream_t st) {
    const int64_t nn = h->hs.n;
    const bool fl = h->opts.flexible_cg != 0;
    CK(launch_pcg_spmv_dot(nn, nrhs, h->a_rp, h->a_ci, h->a_v, h->pp, h->pq, h->dpart, h->scal, st));  // q, p.q
    CK(launch_pcg_alpha(nrhs, h->scal, h->iflags, st));
    if (h->pz32)       // x, r, fl32(r), r.r and r.z_old
        CK(launch_pcg_xr_dots<float>(nn, nrhs, h->px, h->pr, h->pp, h->pq, h->pr32, fl ? h->pz32 : nullptr,
                                     h->scal, h->iflags, h->dpart, st));
    else
        CK(launch_pcg_xr_dots<double>(nn, nrhs, h->px, h->pr, h->pp, h->pq, nullptr, fl ? h->pz : nullptr,
                                      h->scal, h->iflags, h->dpart, st));
    return SLR_OK;
}

// Host-driven loop: one stream synchronisation per iteration (kept for comparison).
slr_status pcg_host_loop(slr_handle h, int32_t nrhs, double tol, int32_t maxit, cudaStream_t st) {
    int32_t active = 1;
    for (int32_t it = 1; it <= maxit; ++it) {
        if (it > 1) CS(pcg_update_part(h, nrhs, st));
        CS(pcg_test_part(h, nrhs, st));
        CK(launch_pcg_check(nrhs, h->scal, h->iflags, it, tol, st));
        CK(cudaMemcpyAsync(&active, h->iflags + 4 * nrhs, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (active == 0) break;
    }
    return SLR_OK;
}

// The whole CG loop as one CUDA graph: WHILE(active and it < maxit) { IF(it > 0) update; test }.
// The test part's last kernel sets both conditions on the device.
slr_status pcg_graph(slr_handle h, int32_t nrhs, slr_handle_s::PcgGraph** out) {
    for (auto& gr : h->pcg_graphs)
        if (gr.nrhs == nrhs) { *out = &gr; return SLR_OK; }
    if (!h->ctl) CS(dalloc(h, &h->ctl, 2));
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { if (s) cudaStreamDestroy(s); }
    } sg{cs};
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    struct GraphGuard {
        cudaGraph_t g;
        ~GraphGuard() { if (g) cudaGraphDestroy(g); }
    } gg{graph};
    cudaGraphConditionalHandle hw, hi;
    CK(cudaGraphConditionalHandleCreate(&hw, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    CK(cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    CK(cudaGraphAddNode(&inode, body, nullptr, nullptr, 0, &ip));
    cudaGraph_t ibody = ip.conditional.phGraph_out[0];
    slr_handle_s::PcgGraph gr;
    gr.nrhs = nrhs;
    std::shared_lock<std::shared_mutex> capture_lock(g_capture_mu);
    const int64_t l0 = thread_launches();
    // A capture that fails part-way leaves nodes in a conditional body of
    // `graph`, and destroying such a graph has crashed inside the driver: on
    // that error path the graph is left allocated (one graph per failure).
    auto capture_failed = [&](slr_status st, cudaError_t ce) {
        count_launches(-(thread_launches() - l0));
        gg.g = nullptr;
        cudaGetLastError();                       // the failure is reported by the status
        if (st == SLR_OK) {
            set_error(std::string("pcg graph capture: ") + cudaGetErrorString(ce));
            st = SLR_ERR_CUDA;
        }
        return st;
    };
    CK(cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    slr_status s1 = pcg_update_part(h, nrhs, cs);
    cudaGraph_t tmp = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &tmp);
    if (s1 != SLR_OK || ce != cudaSuccess) return capture_failed(s1, ce);
    const int64_t l1 = thread_launches();
    CK(cudaStreamBeginCaptureToGraph(cs, body, &inode, nullptr, 1, cudaStreamCaptureModeRelaxed));
    s1 = pcg_test_part(h, nrhs, cs);
    if (s1 == SLR_OK) {
        cudaError_t e2 = launch_pcg_check_graph(nrhs, h->scal, h->iflags, h->ctl, hw, hi, cs);
        if (e2 != cudaSuccess) {
            set_error(std::string("pcg check launch: ") + cudaGetErrorString(e2));
            s1 = SLR_ERR_CUDA;
        }
    }
    ce = cudaStreamEndCapture(cs, &tmp);
    if (s1 != SLR_OK || ce != cudaSuccess) return capture_failed(s1, ce);
    capture_lock.unlock();
    const int64_t l2 = thread_launches();
    gr.kB = l1 - l0;
    gr.kA = l2 - l1;
    count_launches(-(l2 - l0));               // captured, not run
    CK(cudaGraphInstantiate(&gr.exec, graph, 0));
    h->pcg_graphs.push_back(gr);
    *out = &h->pcg_graphs.back();
    return SLR_OK;
}

void drop_graphs(slr_handle h) {
    for (auto& gr : h->pcg_graphs)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    h->pcg_graphs.clear();
}

// Section 6 accelerator for the indefinite problems: flexible GMRES(m) on one
// DD-order column b (device, length n) into x (device), x_0 = 0.  Device work:
// applies of M^{-1} (kept as Z), products with A, two classical Gram-Schmidt passes
// and the norm per step (one host read per step); host: the Hessenberg column's
// Givens rotations and the triangular solve at each restart.
slr_status gmres_column(slr_handle h, const double* b, double* x, double tol, int32_t maxit, int32_t m,
                        cudaStream_t st, int32_t* its_out, double* rel_out) {
    const int32_t n = h->hs.n;
    const int64_t nn = n;
    ScopedBuf<double> bV(h), bZ(h), bw(h), bh(h), bp(h), bs(h);
    CS(bV.alloc((size_t)nn * (m + 1)));
    CS(bZ.alloc((size_t)nn * m));
    CS(bw.alloc((size_t)nn));
    CS(bh.alloc((size_t)2 * (m + 1) + 2));
    CS(bp.alloc((size_t)(m + 1) * kRedBlocks));
    CS(bs.alloc(2));
    double *V = bV.p, *Z = bZ.p, *w = bw.p, *hcol = bh.p, *part = bp.p, *sc = bs.p;
    slr_status err = SLR_OK;
    auto norm2 = [&](const double* v) -> double {   // ||v||, synchronising
        if (launch_dots(nn, 1, v, nn, v, nn, part, sc, 1, st) != cudaSuccess) err = SLR_ERR_CUDA;
        return std::sqrt(std::max(read_scalar(sc, st, &err), 0.0));
    };
    // r = b - A x into w (x = 0: r = b)
    auto residual = [&](bool zero_x) -> cudaError_t {
        if (zero_x) return cudaMemcpyAsync(w, b, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st);
        cudaError_t e = launch_csr_spmv(n, h->a_rp, h->a_ci, h->a_v, x, nn, w, nn, 1, st);
        if (e != cudaSuccess) return e;
        return launch_axpby(nn, 1.0, b, -1.0, w, st);
    };
    CK(cudaMemsetAsync(x, 0, sizeof(double) * nn, st));
    const double bnorm = norm2(b);
    if (err != SLR_OK) return err;
    int32_t its = 0;
    bool first = true;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hv(2 * (m + 1) + 2), y(m);
    while (bnorm > 0.0) {
        CK(residual(first));
        first = false;
        const double beta = norm2(w);
        if (err != SLR_OK) break;
        if (beta <= tol * bnorm || its >= maxit) break;
        CK(launch_axpby(nn, 1.0 / beta, w, 0.0, V, st));            // v_0 = r / beta
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int32_t jd = 0;
        for (int32_t j = 0; j < m; ++j) {
            double* vj = V + (int64_t)j * nn;
            double* zj = Z + (int64_t)j * nn;
            CS(apply_any(h, vj, nn, zj, nn, 1, st));                // z_j = M^{-1} v_j
            CK(launch_csr_spmv(n, h->a_rp, h->a_ci, h->a_v, zj, nn, w, nn, 1, st));   // w = A z_j
            ++its;
            // two classical Gram-Schmidt passes: h = V^T w, w -= V h (twice), then ||w||
            CK(launch_gemv_t(n, j + 1, V, w, part, hcol, st));
            CK(launch_gemv_n_sub(n, j + 1, V, hcol, w, st));
            CK(launch_gemv_t(n, j + 1, V, w, part, hcol + (m + 1), st));
            CK(launch_gemv_n_sub(n, j + 1, V, hcol + (m + 1), w, st));
            CK(launch_dots(nn, 1, w, nn, w, nn, part, hcol + 2 * (m + 1), 1, st));
            CK(cudaMemcpyAsync(hv.data(), hcol, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            double* Hj = H.data() + (size_t)j * (m + 1);            // column j, rows 0 .. j+1
            for (int32_t i = 0; i <= j; ++i) Hj[i] = hv[i] + hv[(m + 1) + i];
            const double hn = std::sqrt(std::max(hv[2 * (m + 1)], 0.0));
            Hj[j + 1] = hn;
            if (hn > 0.0) CK(launch_axpby(nn, 1.0 / hn, w, 0.0, V + (int64_t)(j + 1) * nn, st));
            for (int32_t i = 0; i < j; ++i) {                         // earlier rotations
                const double t = cs[i] * Hj[i] + sn[i] * Hj[i + 1];
                Hj[i + 1] = -sn[i] * Hj[i] + cs[i] * Hj[i + 1];
                Hj[i] = t;
            }
            const double d = std::hypot(Hj[j], Hj[j + 1]);          // the rotation that zeroes H[j+1, j]
            cs[j] = d > 0.0 ? Hj[j] / d : 1.0;
            sn[j] = d > 0.0 ? Hj[j + 1] / d : 0.0;
            Hj[j] = d;
            Hj[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jd = j + 1;
            if (std::fabs(g[j + 1]) <= tol * bnorm || its >= maxit || hn == 0.0) break;
        }
        // y = R^{-1} g (R upper triangular, jd x jd), then x += Z y (as x -= Z (-y))
        for (int32_t i = jd - 1; i >= 0; --i) {
            double s = g[i];
            for (int32_t q = i + 1; q < jd; ++q) s -= H[(size_t)q * (m + 1) + i] * y[q];
            const double rii = H[(size_t)i * (m + 1) + i];
            y[i] = rii != 0.0 ? s / rii : 0.0;
        }
        for (int32_t i = 0; i < jd; ++i) y[i] = -y[i];
        CK(cudaMemcpyAsync(hcol, y.data(), sizeof(double) * jd, cudaMemcpyHostToDevice, st));
        CK(launch_gemv_n_sub(n, jd, Z, hcol, x, st));
    }
    double rel = 0.0;
    if (err == SLR_OK && bnorm > 0.0) {
        CK(residual(false));
        rel = norm2(w) / bnorm;
    }
    *its_out = its;
    *rel_out = rel;
    return err;
}

}  // namespace

extern "C" {

slr_status slr_setup(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* val, int32_t nparts,
                     const int32_t* part, const slr_opts* opts, void* stream, slr_handle* out) {
    if (!out) { set_error("out is NULL"); return SLR_ERR_INVALID_ARG; }
    *out = nullptr;
    slr_handle h = new (std::nothrow) slr_handle_s();
    if (!h) { set_error("host allocation failed"); return SLR_ERR_OOM; }
    if (opts) h->opts = *opts; else slr_default_opts(&h->opts);
    const slr_opts& o = h->opts;
    if (o.k < 0 || o.lanczos_steps < 0 || o.nrhs_max < 0 || o.nrhs_max > 64 ||
        (o.precision != SLR_PREC_FP64 && o.precision != SLR_PREC_MIXED) ||
        (o.theta_mode != SLR_THETA_LAMBDA_K1 && o.theta_mode != SLR_THETA_ZERO) ||
        (o.band_split != 0 && o.band_split != 1 && o.band_split != 2 && o.band_split != 4) ||
        o.host_loop < 0 || o.host_loop > 1 || o.band_slots < 0 || o.band_slots == 1 || o.band_slots > 8 ||
        o.c_persistent < 0 || o.c_persistent > 1 || o.autotune < 0 || o.autotune > 1 ||
        o.target_kappa < 0 || o.target_kappa == 1 ||
        (o.band_threads != 0 && o.band_threads != 32 && o.band_threads != 256 && o.band_threads != 512) ||
        o.c_levels_only < 0 || o.c_levels_only > 1 || o.band_factor_host < 0 || o.band_factor_host > 1 ||
        o.indefinite < 0 || o.indefinite > 1 || o.band_order < 0 || o.band_order > 3 ||
        o.u_dtype < SLR_U_FP32 || o.u_dtype > SLR_U_BF16 ||
        (o.u_dtype != SLR_U_FP32 && o.precision != SLR_PREC_MIXED) || o.spin_limit < 0 ||
        o.band_mma < 0 || o.band_mma > SLR_U_BF16 || (o.band_mma != 0 && o.precision != SLR_PREC_MIXED) ||
        o.zform < 0 || o.zform > 1 ||
        std::any_of(o.reserved, o.reserved + 6, [](int32_t v) { return v != 0; })) {
        set_error("invalid options");
        delete h;
        return SLR_ERR_INVALID_ARG;
    }
    if (h->opts.nrhs_max == 0) h->opts.nrhs_max = 1;
    slr_status s;
    try {
        h->stream = (cudaStream_t)stream;
        s = setup_impl(h, n, rowptr, colind, val, nparts, part, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        s = SLR_ERR_OOM;
    }
    if (s != SLR_OK) {
        slr_destroy(h);
        return s;
    }
    *out = h;
    return SLR_OK;
}

slr_status slr_apply(slr_handle h, const double* r, double* z, int32_t nrhs, int32_t ld, void* stream) {
    CS(check_handle(h));
    if (nrhs < 1 || nrhs > h->opts.nrhs_max || ld < h->hs.n || !r || !z) {
        set_error("slr_apply: bad nrhs, ld or pointer");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    CS(clear_status(h, (cudaStream_t)stream));
    return apply_any(h, r, ld, z, ld, nrhs, (cudaStream_t)stream);
}

slr_status slr_bsolve(slr_handle h, const double* f, double* t, int32_t nrhs, int32_t ld, void* stream) {
    CS(check_handle(h));
    const int32_t nI = h->hs.nI;
    if (nrhs < 1 || nrhs > h->opts.nrhs_max || ld < nI || (!f && nI) || (!t && nI)) {
        set_error("slr_bsolve: bad arguments");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    CS(clear_status(h, st));
    if (h->opts.precision == SLR_PREC_FP64) {
        CK(launch_band_solve<double>(h->op64, h->hs.p, h->hs.wmax, f, ld, t, ld, nullptr, 0, nrhs, st));
        return SLR_OK;
    }
    DevOperator<float>& op = h->op32;
    CK(launch_convert<double, float>(nI, nrhs, f, ld, op.wr, nI, st));
    CK(launch_band_solve<float>(op, h->hs.p, h->hs.wmax, op.wr, nI, op.wz, nI, nullptr, 0, nrhs, st));
    CK(launch_convert<float, double>(nI, nrhs, op.wz, nI, t, ld, st));
    return SLR_OK;
}

static slr_status interface_solve(slr_handle h, const double* g, double* y, int32_t nrhs, int32_t ld, bool lowrank,
                                  cudaStream_t st) {
    CS(check_handle(h));
    const int32_t s = h->hs.s;
    if (nrhs < 1 || nrhs > h->opts.nrhs_max || ld < s || (s && (!g || !y))) {
        set_error("interface solve: bad arguments");
        return SLR_ERR_INVALID_ARG;
    }
    if (s == 0) return SLR_OK;
    DeviceGuard gd(h->device);
    CS(clear_status(h, st));
    if (h->opts.precision == SLR_PREC_FP64) {
        DevOperator<double>& op = h->op64;
        CK(launch_c_forward<double>(op.cf, g, ld, op.wf, nrhs, st));
        if (lowrank) CK(launch_lowrank<double>(op, s, h->k, op.wf, nrhs, st));
        CK(launch_c_backward<double>(op.cf, op.wf, op.xf, y, ld, nrhs, st));
        return SLR_OK;
    }
    DevOperator<float>& op = h->op32;
    CK(launch_convert<double, float>(s, nrhs, g, ld, op.gp, s, st));
    CK(launch_c_forward<float>(op.cf, op.gp, s, op.wf, nrhs, st));
    if (lowrank) CK(launch_lowrank<float>(op, s, h->k, op.wf, nrhs, st));
    CK(launch_c_backward<float>(op.cf, op.wf, op.xf, op.gp, s, nrhs, st));
    CK(launch_convert<float, double>(s, nrhs, op.gp, s, y, ld, st));
    return SLR_OK;
}

slr_status slr_csolve(slr_handle h, const double* g, double* y, int32_t nrhs, int32_t ld, void* stream) {
    return interface_solve(h, g, y, nrhs, ld, false, (cudaStream_t)stream);
}

slr_status slr_stilde_solve(slr_handle h, const double* g, double* y, int32_t nrhs, int32_t ld, void* stream) {
    return interface_solve(h, g, y, nrhs, ld, true, (cudaStream_t)stream);
}

slr_status slr_pcg_solve(slr_handle h, const double* b, double* x, int32_t nrhs, int32_t ld, double tol,
                         int32_t maxit, void* stream, int32_t* iters_out, double* relres_out) {
    CS(check_handle(h));
    const int32_t n = h->hs.n;
    if (nrhs < 1 || nrhs > h->opts.nrhs_max || ld < n || !b || !x || maxit < 0 || !(tol >= 0.0)) {
        set_error("slr_pcg_solve: bad arguments");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nn = n;
    // start: r = P b (DD order), x = 0, b.b, flags, z = M^{-1} r, rho = r.z, p = z
    h->slots_live = false;
    CS(clear_status(h, st));
    CK(launch_permute(n, nrhs, h->perm, b, ld, h->pr, nn, true, st));
    CK(cudaMemsetAsync(h->px, 0, sizeof(double) * nn * nrhs, st));
    CK(launch_dots(nn, nrhs, h->pr, nn, h->pr, nn, h->dpart, h->scal + 4, 8, st));
    CK(launch_pcg_init(nrhs, h->scal, h->iflags, st));
    if (h->pz32) {
        CK(launch_convert<double, float>(nn, nrhs, h->pr, nn, h->pr32, nn, st));
        CS(pcg_apply(h, nrhs, st));
        CK(launch_pcg_dot<float>(nn, nrhs, h->pr, h->pz32, h->dpart, h->scal + 0, 8, st));
        CK(launch_convert<float, double>(nn, nrhs, h->pz32, nn, h->pp, nn, st));                 // p = z
    } else {
        CS(pcg_apply(h, nrhs, st));
        CK(launch_pcg_dot<double>(nn, nrhs, h->pr, h->pz, h->dpart, h->scal + 0, 8, st));
        CK(cudaMemcpyAsync(h->pp, h->pz, sizeof(double) * nn * nrhs, cudaMemcpyDeviceToDevice, st));
    }
    if (maxit > 0) {
        slr_handle_s::PcgGraph* gr = nullptr;
        // the graph is captured on first use for this right-hand-side count; if
        // the capture fails (another thread may have made a call that waits for
        // the whole device meanwhile) this solve runs the same kernels from the
        // host loop, and the next solve captures again
        if (h->opts.host_loop == 1 || pcg_graph(h, nrhs, &gr) != SLR_OK) {
            CS(pcg_host_loop(h, nrhs, tol, maxit, st));
        } else {
            const double ctl[2] = {tol * tol, (double)maxit};
            CK(cudaMemcpyAsync(h->ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, st));
            CK(cudaGraphLaunch(gr->exec, st));
            int32_t its = 0;
            CK(cudaMemcpyAsync(&its, h->iflags + 4 * nrhs + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            // kernels the graph ran: the test part every iteration, the update part from the second on
            count_launches(its * gr->kA + std::max(0, its - 1) * gr->kB);
        }
    }
    CK(launch_permute(n, nrhs, h->perm, h->px, nn, x, ld, false, st));                 // x = P^T x_dd
    std::vector<double> sc(8 * nrhs);
    std::vector<int32_t> fl(4 * nrhs + 4);
    CK(cudaMemcpyAsync(sc.data(), h->scal, sizeof(double) * 8 * nrhs, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(fl.data(), h->iflags, sizeof(int32_t) * fl.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    slr_status ret = SLR_OK;
    CS(read_status(h, status_word(h), st));
    for (int j = 0; j < nrhs; ++j) {
        if (iters_out) iters_out[j] = fl[4 * j + 1];
        double bb = sc[8 * j + 4];
        if (relres_out) relres_out[j] = bb > 0 ? std::sqrt(std::max(sc[8 * j + 3], 0.0) / bb) : 0.0;
        if (fl[4 * j + 2] == 2) ret = SLR_ERR_BREAKDOWN;
        else if (fl[4 * j + 2] == 0 && ret == SLR_OK) ret = SLR_ERR_NOT_CONVERGED;
    }
    if (ret == SLR_ERR_BREAKDOWN) set_error("PCG breakdown: p^T A p <= 0");
    if (ret == SLR_ERR_NOT_CONVERGED) set_error("PCG reached maxit");
    return ret;
}

slr_status slr_gmres_solve(slr_handle h, const double* b, double* x, int32_t nrhs, int32_t ld, double tol,
                           int32_t maxit, int32_t restart, void* stream, int32_t* iters_out, double* relres_out) {
    CS(check_handle(h));
    const int32_t n = h->hs.n;
    if (nrhs < 1 || nrhs > h->opts.nrhs_max || ld < n || !b || !x || maxit < 0 || !(tol >= 0.0) || restart < 1 ||
        restart > 1000) {
        set_error("slr_gmres_solve: bad arguments");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nn = n;
    h->slots_live = false;
    CS(clear_status(h, st));
    CK(launch_permute(n, nrhs, h->perm, b, ld, h->pr, nn, true, st));   // b in DD order
    slr_status ret = SLR_OK;
    for (int32_t j = 0; j < nrhs; ++j) {
        int32_t its = 0;
        double rel = 0.0;
        CS(gmres_column(h, h->pr + j * nn, h->px + j * nn, tol, maxit, restart, st, &its, &rel));
        if (iters_out) iters_out[j] = its;
        if (relres_out) relres_out[j] = rel;
        if (!(rel <= tol * (1.0 + 1e-6)) && ret == SLR_OK) ret = SLR_ERR_NOT_CONVERGED;
    }
    CK(launch_permute(n, nrhs, h->perm, h->px, nn, x, ld, false, st));  // x = P^T x_dd
    CS(read_status(h, status_word(h), st));
    if (ret == SLR_ERR_NOT_CONVERGED) set_error("GMRES reached maxit");
    return ret;
}

slr_status slr_cg_slot_start(slr_handle h, int32_t slot, const double* b, double tol, int32_t maxit, void* stream) {
    CS(check_handle(h));
    const int32_t n = h->hs.n;
    if (slot < 0 || slot >= h->opts.nrhs_max || !b || maxit < 0 || !(tol >= 0.0)) {
        set_error("slr_cg_slot_start: bad slot, pointer, tol or maxit");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!h->slot_ctl) CS(dalloc(h, &h->slot_ctl, (size_t)2 * h->opts.nrhs_max));
    if (!h->slots_live) {       // the workspaces last served slr_pcg_solve / slr_gmres_solve: every slot idle
        CK(cudaMemsetAsync(h->iflags, 0, sizeof(int32_t) * (4 * (size_t)h->opts.nrhs_max + 4), st));
        h->slots_live = true;
    }
    const int64_t nn = n, off = (int64_t)slot * nn;
    CK(launch_permute(n, 1, h->perm, b, nn, h->pr + off, nn, true, st));          // r = P b
    CK(cudaMemsetAsync(h->px + off, 0, sizeof(double) * nn, st));                 // x = 0
    CK(cudaMemsetAsync(h->pp + off, 0, sizeof(double) * nn, st));                 // p = 0
    if (h->pz32) {
        CK(cudaMemsetAsync(h->pz32 + off, 0, sizeof(float) * nn, st));            // z = 0
        CK(launch_convert<double, float>(nn, 1, h->pr + off, nn, h->pr32 + off, nn, st));   // fl32(r)
    } else {
        CK(cudaMemsetAsync(h->pz + off, 0, sizeof(double) * nn, st));             // z = 0
    }
    CK(cudaMemsetAsync(h->scal + 8 * slot + 7, 0, sizeof(double), st));           // r.z_old = 0 (z_old = 0)
    CK(launch_dots(nn, 1, h->pr + off, nn, h->pr + off, nn, h->dpart, h->scal + 8 * slot + 4, 8, st));   // b.b
    CK(launch_cg_slot_init(slot, tol, maxit, h->scal, h->iflags, h->slot_ctl, st));
    return SLR_OK;
}

slr_status slr_cg_advance(slr_handle h, int32_t iters, int32_t width, void* stream, int32_t* active_out,
                          int32_t* iters_out, double* relres_out, int32_t* status_out) {
    CS(check_handle(h));
    if (iters < 0 || width < 1 || width > h->opts.nrhs_max || !h->slots_live) {
        set_error("slr_cg_advance: bad iters or width, or no slot was started");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    CS(clear_status(h, st));
    for (int32_t it = 0; it < iters; ++it) {
        CS(pcg_update_part(h, width, st));
        CS(pcg_test_part(h, width, st));
        CK(launch_cg_slot_check(width, 4 * h->opts.nrhs_max, h->scal, h->iflags, h->slot_ctl, st));
    }
    std::vector<double> sc(8 * (size_t)width);
    std::vector<int32_t> fl(4 * (size_t)width);
    CK(cudaMemcpyAsync(sc.data(), h->scal, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(fl.data(), h->iflags, sizeof(int32_t) * fl.size(), cudaMemcpyDeviceToHost, st));
    CS(read_status(h, status_word(h), st));
    for (int32_t j = 0; j < width; ++j) {
        if (active_out) active_out[j] = fl[4 * j];
        if (iters_out) iters_out[j] = fl[4 * j + 1];
        if (status_out) status_out[j] = fl[4 * j + 2];
        const double bb = sc[8 * j + 4];
        if (relres_out) relres_out[j] = bb > 0 ? std::sqrt(std::max(sc[8 * j + 3], 0.0) / bb) : 0.0;
    }
    return SLR_OK;
}

slr_status slr_cg_slot_result(slr_handle h, int32_t slot, double* x, void* stream) {
    CS(check_handle(h));
    if (slot < 0 || slot >= h->opts.nrhs_max || !x) {
        set_error("slr_cg_slot_result: bad slot or pointer");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    const int64_t nn = h->hs.n;
    CK(launch_permute(h->hs.n, 1, h->perm, h->px + (int64_t)slot * nn, nn, x, nn, false, (cudaStream_t)stream));
    return SLR_OK;
}

slr_status slr_set_lowrank(slr_handle h, int32_t k, const double* Z, const double* lam, double theta, void* stream) {
    CS(check_handle(h));
    const int32_t s = h->hs.s;
    if (k < 0 || k > s || (k > 0 && (!Z || !lam)) || !(theta < 1.0 && (h->hs.indefinite || theta >= 0.0))) {
        set_error("slr_set_lowrank: bad arguments");
        return SLR_ERR_INVALID_ARG;
    }
    for (int32_t i = 0; i < k; ++i)
        if (h->hs.indefinite ? !(std::fabs(1.0 - lam[i]) > 0.0) : !(lam[i] < 1.0)) {
            set_error("slr_set_lowrank: lambda must be < 1 (indefinite A: different from 1)");
            return SLR_ERR_INVALID_ARG;
        }
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->stream = st;
    double *Zd = nullptr, *CZ = nullptr, *U = nullptr;
    if (k > 0) {
        CS(dalloc(h, &Zd, (size_t)s * k));
        CS(dalloc(h, &CZ, (size_t)s * k));
        CS(dalloc(h, &U, (size_t)s * k));
        CK(cudaMemcpyAsync(Zd, Z, sizeof(double) * s * k, cudaMemcpyHostToDevice, st));
        CK(launch_csr_spmv(s, h->c_rp, h->c_ci, h->c_v, Zd, s, CZ, s, k, st));       // C Z
        // U = L^{-1} C Z, at most nrhs_max columns at a time (the forward solve's
        // panel-product workspace holds nrhs_max columns)
        const int32_t r = std::max(1, h->opts.nrhs_max);
        for (int32_t c0 = 0; c0 < k; c0 += r) {
            const int32_t nc = std::min(r, k - c0);
            CK(launch_c_forward<double>(h->op64.cf, CZ + (int64_t)c0 * s, s, U + (int64_t)c0 * s, nc, st));
        }
        CK(cudaStreamSynchronize(st));
    }
    std::vector<double> lv(lam, lam + k);
    const int32_t k_old = h->k;
    {
        std::unique_lock<std::shared_mutex> lk(g_capture_mu);
        drop_graphs(h);
    }
    CS(set_operator_lowrank<double>(h, h->op64, U, k_old, k, lv, theta));
    if (h->opts.precision == SLR_PREC_MIXED) CS(set_operator_lowrank<float>(h, h->op32, U, k_old, k, lv, theta));
    h->k = k;
    h->lam = lv;
    h->theta = theta;
    if (k > 0) {
        dfree(h, Zd, (size_t)s * k);
        dfree(h, CZ, (size_t)s * k);
        dfree(h, U, (size_t)s * k);
    }
    account(h);
    return SLR_OK;
}

slr_status slr_add_vectors(slr_handle h, int32_t k_add, int32_t lanczos_steps, void* stream, int32_t* added_out) {
    CS(check_handle(h));
    if (k_add < 0 || lanczos_steps < 0) {
        set_error("slr_add_vectors: k_add and lanczos_steps must be >= 0");
        return SLR_ERR_INVALID_ARG;
    }
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    h->stream = st;
    int32_t added = 0;
    CS(clear_status(h, st));
    slr_status r = run_lanczos_deflated(h, k_add, lanczos_steps, st, &added);
    if (added_out) *added_out = added;
    if (r == SLR_OK) account(h);
    return r;
}

slr_status slr_get_lowrank(slr_handle h, double* Z, double* lam, double* theta_out, void* stream) {
    CS(check_handle(h));
    DeviceGuard g(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t s = h->hs.s, k = h->k;
    if (Z && k > 0) {
        double *X1 = nullptr, *Y1 = nullptr;
        CS(dalloc(h, &X1, (size_t)s * k));
        CS(dalloc(h, &Y1, (size_t)s * k));
        // Z = L^{-T} U (DD order), at most nrhs_max columns at a time (the top zone's
        // partial-sum workspace holds nrhs_max columns)
        const int32_t r = std::max(1, h->opts.nrhs_max);
        for (int32_t c0 = 0; c0 < k; c0 += r)
            CK(launch_c_backward<double>(h->op64.cf, h->op64.U + (int64_t)c0 * s, X1 + (int64_t)c0 * s,
                                         Y1 + (int64_t)c0 * s, s, std::min(r, k - c0), st));
        CK(cudaMemcpyAsync(Z, Y1, sizeof(double) * s * k, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        dfree(h, X1, (size_t)s * k);
        dfree(h, Y1, (size_t)s * k);
    }
    if (lam) {
        for (int32_t i = 0; i < k; ++i) lam[i] = h->lam[i];
        lam[k] = (int32_t)h->ritz.size() > k ? h->ritz[k] : 0.0;
    }
    if (theta_out) *theta_out = h->theta;
    return SLR_OK;
}

slr_status slr_get_ritz(slr_handle h, double* lam, int32_t* count) {
    CS(check_handle(h));
    if (lam) for (size_t i = 0; i < h->ritz.size(); ++i) lam[i] = h->ritz[i];
    if (count) *count = (int32_t)h->ritz.size();
    return SLR_OK;
}

slr_status slr_get_perm(slr_handle h, int32_t* perm) {
    CS(check_handle(h));
    if (!perm) { set_error("perm is NULL"); return SLR_ERR_INVALID_ARG; }
    std::memcpy(perm, h->hs.perm.data(), sizeof(int32_t) * h->hs.n);
    return SLR_OK;
}

slr_status slr_get_info(slr_handle h, slr_info* info) {
    CS(check_handle(h));
    if (!info) { set_error("info is NULL"); return SLR_ERR_INVALID_ARG; }
    std::memset(info, 0, sizeof(*info));
    const HostSetup& hs = h->hs;
    info->n = hs.n;
    info->n_interior = hs.nI;
    info->s = hs.s;
    info->nparts = hs.p;
    info->k = h->k;
    info->lanczos_steps = h->m_steps;
    info->nnz_A = (int64_t)hs.a_v.size();
    info->nnz_E = (int64_t)hs.e_v.size();
    info->nnz_C = (int64_t)hs.c_v.size();
    int64_t band = 0;
    for (const BandBlock& b : hs.band) band += (int64_t)b.c * b.w * (b.w + 1);
    info->band_entries = band;
    info->c_diag_entries = hs.cf.dinv_off.empty() ? 0 : hs.cf.dinv_off.back();
    info->c_panel_entries = hs.cf.pan_off.empty() ? 0 : hs.cf.pan_off.back();
    info->c_supernodes = hs.cf.ns;
    info->c_levels = hs.cf.nlev;
    info->bytes_per_apply = h->bytes_per_apply;
    info->vector_bytes_per_column = h->vector_bytes_per_column;
    info->flops_per_apply = h->flops_per_apply;
    info->device_bytes = h->device_bytes;
    info->theta = h->theta;
    for (int i = 0; i < 5; ++i) info->setup_seconds[i] = h->setup_seconds[i];
    info->precision = h->opts.precision;
    info->theta_mode = h->opts.theta_mode;
    info->band_split = hs.band_G;
    const bool f64 = h->opts.precision == SLR_PREC_FP64;
    info->band_slots = f64 ? h->op64.band_nbuf : h->op32.band_nbuf;
    info->c_persistent = (f64 ? h->op64.cf.per_level : h->op32.cf.per_level) ? 0 : 1;
    info->tuned = h->tuned ? 1 : 0;
    info->tune_seconds = h->tune_seconds;
    info->band_threads = f64 ? h->op64.band_nt : h->op32.band_nt;
    info->c_top_levels = hs.cf.nlev - hs.cf.top_lev;
    info->c_top_positions = hs.cf.nT;
    info->c_top_entries = hs.cf.tsk_off.empty() ? 0 : hs.cf.tsk_off.back();
    info->band_on_device = h->band_on_device ? 1 : 0;
    for (int i = 0; i < 3; ++i) info->lanczos_seconds[i] = h->lanczos_seconds[i];
    info->band_mma = f64 ? 0 : h->op32.band_mma;
    info->u_dtype = f64 ? 0 : h->op32.u_dtype;
    return SLR_OK;
}

slr_status slr_device_status(slr_handle h, void* stream) {
    CS(check_handle(h));
    DeviceGuard g(h->device);
    return read_status(h, status_word(h), (cudaStream_t)stream);
}

void slr_inject_alloc_failure(int64_t nth) { g_fail_alloc.store(nth > 0 ? nth : 0); }

void slr_destroy(slr_handle h) {
    if (!h) return;
    int old = -1;
    cudaGetDevice(&old);
    if (old != h->device) cudaSetDevice(h->device);
    {
        std::unique_lock<std::shared_mutex> lk(g_capture_mu);
        drop_graphs(h);
        if (h->aux) {
            cudaStreamSynchronize(h->aux);
            cudaStreamDestroy(h->aux);
        }
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->ev_join) cudaEventDestroy(h->ev_join);
        for (void* p : h->allocs) cudaFree(p);
    }
    if (old >= 0 && old != h->device) cudaSetDevice(old);
    delete h;
}

}  // extern "C"
