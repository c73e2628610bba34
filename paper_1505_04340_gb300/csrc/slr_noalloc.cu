// slr_apply_noalloc: the preconditioner apply with its scratch vectors in a
// fixed, library-owned device array instead of the handle's workspaces.
//
// slr_setup allocates everything a handle needs, once.  The per-call scratch
// of slr_apply lives in that handle.  Some callers cannot let any device
// memory be allocated on their behalf after start-up (for example a host
// process that hands all device memory to its own fixed arena, or code that
// must not grow its footprint while it serves requests), yet want the apply
// without depending on the handle's workspace sizing.  This entry point
// allocates nothing: it carves its scratch from one static __device__ array
// of kNoAllocBytes, which every GPU that loads the library holds until exit.
// slr_setup looks up the array's device address (noalloc_lookup) and keeps it
// in the handle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <type_traits>

#include "slr_device.h"

using namespace slr;

namespace {

constexpr size_t kNoAllocBytes = 32ull << 20;   // 32 MiB per device

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

}  // namespace

// Device address of the array in the current device's context, stored in the
// handle by slr_setup (with the handle's device current, outside any stream
// capture).  In host code the array's name is only a host-side stand-in; its
// device address must come from cudaGetSymbolAddress.  The handle's other
// device memory lives in the same context, so the address stays valid for as
// long as the handle does.
slr_status slr::noalloc_lookup(slr_handle h) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        set_error(std::string("cudaGetSymbolAddress of the allocation-free scratch array failed: ") +
                  cudaGetErrorString(e));
        return SLR_ERR_CUDA;
    }
    h->noalloc_base = p;
    return SLR_OK;
}

namespace {

// Hands out 256-byte aligned slices of the array; `need` counts the bytes.
struct Carver {
    unsigned char* base;
    size_t used = 0;
    template <typename T>
    T* take(size_t count) {
        used = (used + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
        used += count * sizeof(T);
        return p;
    }
};

// Points every per-call workspace of a copy of the operator into the array.
template <typename T>
size_t carve(slr_handle h, DevOperator<T>& op, int32_t nrhs, unsigned char* base) {
    const int64_t n = h->hs.n, nI = std::max<int64_t>(h->hs.nI, 1), s = std::max<int64_t>(h->hs.s, 1);
    const int64_t k = std::max<int32_t>(h->k, 1);
    Carver c{base};
    op.tB = c.take<T>(nI * nrhs);
    op.eb = c.take<T>(nI * nrhs);
    op.gp = c.take<T>(s * nrhs);
    op.wf = c.take<T>(s * nrhs);
    op.xf = c.take<T>(s * nrhs);
    op.cf.wbuf = c.take<T>(std::max<int64_t>(op.cf.nrow, 1) * nrhs);
    op.cf.tws = c.take<T>(s * nrhs);
    op.cf.gfs = c.take<T>(s * nrhs);
    op.cf.ws_cols = nrhs;
    if (op.cf.nT > 0) {   // the top zone's workspaces; its counters are cleared before each apply
        op.cf.tT = c.take<T>((int64_t)op.cf.nT * nrhs);
        op.cf.tf_part = c.take<T>((int64_t)op.cf.tf_parts * nrhs);
        op.cf.tb_part = c.take<T>((int64_t)op.cf.tb_parts * nrhs);
        op.cf.tf_cnt = c.take<int32_t>(op.cf.n_tf_rb);
        op.cf.tb_cnt = c.take<int32_t>(op.cf.n_tb_cb);
    }
    op.cf.bar = c.take<unsigned>(1);          // the persistent C solves' grid barrier counter
    op.vk = c.take<T>(k * nrhs);
    op.part = c.take<T>(lowrank_part_elems((int32_t)s, (int32_t)k, nrhs));
    if constexpr (!std::is_same<T, double>::value) {
        op.wr = c.take<T>(n * nrhs);
        op.wz = c.take<T>(n * nrhs);
    }
    return c.used;
}

#define NA_CK(...)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (__VA_ARGS__);                                                    \
        if (e_ != cudaSuccess) {                                                           \
            set_error(std::string("slr_apply_noalloc: ") + cudaGetErrorString(e_));        \
            return SLR_ERR_CUDA;                                                           \
        }                                                                                  \
    } while (0)

// z = M^{-1} r with the operator's workspaces in the array (same kernels as slr_apply)
template <typename T>
slr_status apply_with(slr_handle h, DevOperator<T>& op, const T* r, int64_t ldr, T* z, int64_t ldz, int32_t nrhs,
                      cudaStream_t st) {
    const HostSetup& hs = h->hs;
    const int32_t nI = hs.nI, s = hs.s;
    NA_CK(launch_band_solve<T>(op, hs.p, hs.wmax, r, ldr, op.tB, nI, nullptr, 0, nrhs, st));
    NA_CK(launch_gather_et<T>(op, s, r + nI, ldr, op.tB, nI, op.gp, s, nrhs, st));
    if (op.cf.nT > 0) {   // the array's bytes there may hold another call's data
        NA_CK(cudaMemsetAsync(op.cf.tf_cnt, 0, sizeof(int32_t) * op.cf.n_tf_rb, st));
        NA_CK(cudaMemsetAsync(op.cf.tb_cnt, 0, sizeof(int32_t) * op.cf.n_tb_cb, st));
    }
    NA_CK(launch_c_forward<T>(op.cf, op.gp, s, op.wf, nrhs, st));
    NA_CK(launch_lowrank<T>(op, s, h->k, op.wf, nrhs, st));
    NA_CK(launch_c_backward<T>(op.cf, op.wf, op.xf, z + nI, ldz, nrhs, st));
    NA_CK(launch_spmv_e<T>(op, nI, z + nI, ldz, op.eb, nI, nrhs, st));
    NA_CK(launch_band_solve<T>(op, hs.p, hs.wmax, op.eb, nI, z, ldz, op.tB, nI, nrhs, st));
    return SLR_OK;
}

template <typename T>
slr_status run_noalloc(slr_handle h, DevOperator<T> op, const double* r, double* z, int32_t nrhs, int32_t ld,
                       cudaStream_t s) {
    const size_t need = carve(h, op, nrhs, nullptr);       // size check before any device work
    if (need > kNoAllocBytes) {
        set_error("slr_apply_noalloc: needs " + std::to_string(need) + " bytes of scratch for nrhs=" +
                  std::to_string(nrhs) + ", more than its fixed " + std::to_string(kNoAllocBytes) + " bytes");
        return SLR_ERR_UNSUPPORTED;
    }
    unsigned char* base = static_cast<unsigned char*>(h->noalloc_base);
    if (!base) {
        set_error("slr_apply_noalloc: the handle holds no address of the scratch array");
        return SLR_ERR_CUDA;
    }
    carve(h, op, nrhs, base);
    NA_CK(cudaMemsetAsync(op.err, 0, sizeof(int32_t), s));   // the call's status word (slr_device_status)
    if constexpr (std::is_same<T, double>::value) {
        return apply_with<double>(h, op, r, ld, z, ld, nrhs, s);
    } else {
        const int64_t n = h->hs.n;
        NA_CK(launch_convert<double, float>(n, nrhs, r, ld, op.wr, n, s));
        const slr_status st = apply_with<float>(h, op, op.wr, n, op.wz, n, nrhs, s);
        if (st != SLR_OK) return st;
        NA_CK(launch_convert<float, double>(n, nrhs, op.wz, n, z, ld, s));
        return SLR_OK;
    }
}

}  // namespace

extern "C" slr_status slr_apply_noalloc(slr_handle h, const double* r, double* z, int32_t nrhs, int32_t ld,
                                        void* stream) {
    if (!h || !h->op64.ready) {
        set_error("slr_apply_noalloc: invalid handle");
        return SLR_ERR_INVALID_ARG;
    }
    if (nrhs < 1 || nrhs > h->opts.nrhs_max || ld < h->hs.n || !r || !z) {
        set_error("slr_apply_noalloc: bad nrhs, ld or pointer");
        return SLR_ERR_INVALID_ARG;
    }
    int old = -1;
    cudaError_t e = cudaGetDevice(&old);
    if (e == cudaSuccess && old != h->device) e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("slr_apply_noalloc: cannot make the handle's device current: ") + cudaGetErrorString(e));
        return SLR_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    slr_status st = h->opts.precision == SLR_PREC_FP64 ? run_noalloc<double>(h, h->op64, r, z, nrhs, ld, s)
                                                       : run_noalloc<float>(h, h->op32, r, z, nrhs, ld, s);
    if (old >= 0 && old != h->device && cudaSetDevice(old) != cudaSuccess) {
        cudaGetLastError();
        if (st == SLR_OK) {
            set_error("slr_apply_noalloc: cannot restore the caller's current device");
            st = SLR_ERR_CUDA;
        }
    }
    return st;
}
