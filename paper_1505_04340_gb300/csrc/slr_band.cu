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
// rows are dealt to the G CTAs of a cluster (r mod G = rank).  Each CTA's slice
// of a block is tiled: row block rb (its slice rows 32 rb .. 32 rb + 31) keeps,
// for every column that meets it, one segment of 32 values (zero outside the
// triangle), row blocks one after the other, columns ascending.  A lane owns a
// row and a segment is one coalesced 32-wide load, so the inner loop is a
// shared load, a broadcast load and an FMA; the padding costs about 16 values
// per column (14% of a 225-wide block).
//
// Each CTA streams its slices through a ring of `nbuf` shared buffers of `slot`
// bytes (2 by default, filling the shared memory left over) with 1-D bulk
// asynchronous copies of whole segments completed on "full" mbarriers.  Every
// warp releases a buffer on its "empty" mbarrier when done with it; thread 0
// refills a buffer once all warps have released it, so copies run ahead of the
// slowest warp across planes and phases with no CTA-wide barrier per chunk.
// Each phase's input vector (t, or y/x) reaches every CTA of the cluster by
// st.async stores into distributed shared memory that complete bytes on the
// receiver's mbarrier, so a CTA waits only for the vector it reads and no
// cluster-wide barrier is taken per phase.  Every wait is a bounded spin that
// sets a device status word instead of hanging.  Warp w takes the columns
// c = w (mod warps) of every row block, so a warp's partial sums (added once
// per phase) do not depend on the chunking.
#include "slr_band_kernel.cuh"

namespace slr {

template <typename T>
cudaError_t launch_band_solve(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi, T* out,
                              int64_t ldo, const T* base, int64_t ldb, int32_t nrhs, cudaStream_t st) {
    if (p == 0 || wmax == 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        // blocks of right-hand sides on the tensor cores when the operator carries that factor
        if (op.band_tc && nrhs >= 8) return launch_band_solve_tc(op, p, in, ldi, out, ldo, base, ldb, nrhs, st);
    }
    // planes of at most 64 rows in one slice: a warp per subdomain (band_nt 32)
    if (op.band_nt == 32 && op.band_G == 1 && wmax <= 64)
        return launch_band_warp(op, p, in, ldi, out, ldo, base, ldb, nrhs, st);
    for (int32_t c = 0; c < nrhs;) {
        const int32_t left = nrhs - c;
        int nr = 1;
        int32_t nb, sl;
        const int nt = op.band_nt;
        // FP32 takes up to 8 columns per CTA (FP64's partial sums would not fit): each
        // group re-reads the factor, so wider groups save bytes on multi-RHS blocks
        if (sizeof(T) == 4 && left >= 8 && band_ring(wmax, 8, sizeof(T), 0, nt, &nb, &sl)) nr = 8;
        else if (left >= 4 && band_ring(wmax, 4, sizeof(T), 0, nt, &nb, &sl)) nr = 4;
        else if (left >= 2 && band_ring(wmax, 2, sizeof(T), 0, nt, &nb, &sl)) nr = 2;
        const T* bs = base ? base + c * ldb : nullptr;
        cudaError_t e = cudaSuccess;
        const T* ic = in + c * ldi;
        T* oc = out + c * ldo;
        if (nt == 256) {
            if constexpr (sizeof(T) == 4) {
                if (nr == 8) e = band_launch_half<T, 8>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
            }
            if (nr == 4) e = band_launch_half<T, 4>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
            else if (nr == 2) e = band_launch_half<T, 2>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
            else if (nr == 1) e = band_launch_half<T, 1>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
        } else {
            if constexpr (sizeof(T) == 4) {
                if (nr == 8) e = band_launch_g<T, 8, 512>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
            }
            if (nr == 4) e = band_launch_g<T, 4, 512>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
            else if (nr == 2) e = band_launch_g<T, 2, 512>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
            else if (nr == 1) e = band_launch_g<T, 1, 512>(op, p, wmax, ic, ldi, oc, ldo, bs, ldb, st);
        }
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
