// The 256-thread variants of the band-solve kernel (two CTAs, two subdomains,
// per SM), for launches with more CTAs than SMs; compiled apart from the
// 512-thread ones so the two halves build in parallel.
#include "slr_band_kernel.cuh"

namespace slr {

template <typename T, int NR>
cudaError_t band_launch_half(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                             int64_t ldo, const T* base, int64_t ldb, cudaStream_t st) {
    return band_launch_g<T, NR, 256>(op, p, wmax, in, ldi, out, ldo, base, ldb, st);
}

#define SLR_HALF(T, NR)                                                                                            \
    template cudaError_t band_launch_half<T, NR>(const DevOperator<T>&, int32_t, int32_t, const T*, int64_t, T*, \
                                                 int64_t, const T*, int64_t, cudaStream_t);
SLR_HALF(float, 1)
SLR_HALF(float, 2)
SLR_HALF(float, 4)
SLR_HALF(float, 8)
SLR_HALF(double, 1)
SLR_HALF(double, 2)
SLR_HALF(double, 4)
#undef SLR_HALF

}  // namespace slr
