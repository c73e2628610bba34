// Internal structures of the SLR library: host-side setup results and the
// device-resident handle.  Not part of the public ABI (see include/slr.h).
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/slr.h"

namespace slr {

// ---------------------------------------------------------------- host setup

// Band factor layout (Section 5.2).  B_i = L_i L_i^T is banded with
// half-bandwidth w; rows are grouped in planes of W = w rows.  For plane J:
// O_J = L[J, J-1] (upper triangular), D_J = L[J, J]^{-1} (lower, inverted on the
// host) and their transposes O_J^T (lower), D_J^T (upper): each of the four
// products of a pass is "output row = sum over columns".  The W rows of a plane
// form 32-row blocks; block k holds rows 32 k .. 32 k + 31.  The G CTAs of a
// cluster (slices) each own whole blocks, assigned so that the slices' shares
// of upper-block and lower-block work are even (band_assign_blocks); slice g's
// local row block rb is block rbmap[g][rb].  A slice of a block is tiled: for
// every (local row block, column) pair that meets the triangle, one segment of
// 32 values (zero outside the triangle and past W), row blocks one after the
// other, columns ascending.  Per plane and slice: [O_J | D_J | O_J^T | D_J^T] =
// [SU | SL | SL | SU] elements; a plane occupies G * 2 (SU + SL).  The last plane
// is padded with identity rows.  (Shared with slr_band.cu.)
struct BandBlock {
    int32_t m = 0;        // rows of B_i
    int32_t w = 0;        // plane width W
    int32_t c = 0;        // planes, c * W >= m
    int32_t row0 = 0;     // first row of B_i inside u (DD interior order)
    int64_t foff = 0;     // offset of plane 0 in the factor array (elements)
    int32_t SU = 0;       // elements of one upper slice block (32 per segment, widest slice)
    int32_t SL = 0;       // elements of one lower slice block (32 per segment, widest slice)
    uint8_t nrb[4] = {0, 0, 0, 0};   // row blocks of each slice (at most 8: 256 rows)
    uint8_t rbmap[4][8] = {};        // block of slice g's local row block rb
};

// Slice geometry (the host packer and the device kernel agree on it).
// Local row block rb of slice g starts at plane row band_R0; in an upper block
// it meets columns [band_cU0, W), in a lower block columns [0, band_cL1).
inline int band_R0(const BandBlock& b, int g, int rb) { return 32 * b.rbmap[g][rb]; }
inline int band_cU0(const BandBlock& b, int g, int rb) { return std::min(b.w, band_R0(b, g, rb)); }
inline int band_cL1(const BandBlock& b, int g, int rb) {
    return std::min(b.w, std::min(band_R0(b, g, rb) + 31, b.w - 1) + 1);
}
// True if G slices can hold a plane of W rows (at most 8 blocks of 32 rows each).
inline bool band_split_ok(int W, int G) { return (W + 31) / 32 <= 8 * G; }
// Deal the 32-row blocks of a plane of b.w rows to G slices (fills nrb, rbmap).
void band_assign_blocks(BandBlock& b, int G);

// Supernodal Cholesky factor of the interface matrix C (Eq. 3.1) in a
// nested-dissection order.  Supernode J owns factor positions [c0[J], c0[J+1]).
struct CFactorHost {
    int32_t s = 0, ns = 0;
    std::vector<int32_t> cperm;        // factor position -> DD interface index
    std::vector<int32_t> c0;           // [ns+1]
    std::vector<int32_t> parent;       // [ns], -1 at a root
    std::vector<int32_t> level;        // [ns], 0 at leaves
    std::vector<int64_t> r_off;        // [ns+1] offsets of R_J in rows
    std::vector<int32_t> rows;         // R_J: factor positions below the diagonal block
    std::vector<int64_t> pan_off;      // [ns+1] offsets of the row-major |R_J| x n_J panels
    std::vector<double> panel;         // L[R_J, J]
    std::vector<int64_t> dinv_off;     // [ns+1] offsets of the packed inverse blocks
    std::vector<double> dinv;          // L_JJ^{-1}: lower triangle, column-major, packed
    // Forward solve: after level l, w[r_off[K] + p] = L[R_K[p], K] x_K for its supernodes K;
    // position i then needs the sum of w over the panel rows that hold row i.
    std::vector<int64_t> seg_ptr;      // [s+1] panel rows of each position, CSR
    std::vector<int32_t> seg_row;      // global panel-row index r_off[K] + p
    int32_t nlev = 0;
    std::vector<int32_t> lev_task_ptr; // [nlev+1] column-block tasks per level
    std::vector<int32_t> tasks;        // 4 ints each: supernode, first column, count (<= 32), 0
    std::vector<int32_t> lev_ptask_ptr;// [nlev+1] panel-row tasks per level
    std::vector<int32_t> ptasks;       // 4 ints each: supernode, first panel row, count (<= 32), 0
    // Levels with many supernodes, each with at most kSmallN columns, kSmallR
    // panel rows and kSmallPanel panel entries, are solved by one fused kernel
    // (one CTA per supernode).
    std::vector<int32_t> lev_sn_ptr;   // [nlev+1] supernodes per level
    std::vector<int32_t> lev_sn;       // supernode ids, level by level
    std::vector<uint8_t> lev_small;    // [nlev]
};
constexpr int32_t kSmallN = 128;
constexpr int32_t kSmallR = 1024;
constexpr int32_t kSmallPanel = 16384;     // panel entries of one supernode
constexpr int32_t kSmallMinCount = 152;    // supernodes a level needs (one wave of SMs)

struct HostSetup {
    int32_t n = 0, nI = 0, s = 0, p = 0;
    std::vector<int32_t> perm, iperm, int_off, ifc_off;
    std::vector<int32_t> a_rp, a_ci;  std::vector<double> a_v;    // P A P^T, CSR
    std::vector<int32_t> e_rp, e_ci;  std::vector<double> e_v;    // E   (nI x s)
    std::vector<int32_t> et_rp, et_ci; std::vector<double> et_v;  // E^T (s x nI)
    std::vector<int32_t> c_rp, c_ci;  std::vector<double> c_v;    // C   (s x s)
    std::vector<BandBlock> band;
    std::vector<double> bfac;
    int32_t wmax = 0;
    int32_t band_G = 1;   // CTAs (slices) per subdomain in the band solve
    int32_t band_nt = 512;   // threads per band-solve CTA (256: two CTAs per SM)
    CFactorHost cf;
};

// Thread-local error text for slr_last_error_message().
void set_error(const std::string& msg);

// Host setup steps (slr_host.cpp).  Each returns SLR_OK or an error status.
slr_status host_dd_order(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts,
                         const int32_t* part, HostSetup& hs);
slr_status host_validate_csr(int32_t n, const int32_t* rowptr, const int32_t* colind,
                             const double* val, int32_t nparts, const int32_t* part);
slr_status host_split_blocks(const int32_t* rowptr, const int32_t* colind, const double* val,
                             HostSetup& hs);
slr_status host_band_factor(HostSetup& hs, int32_t G);
slr_status host_c_factor(HostSetup& hs, int32_t leaf, int32_t task_rows);
// Symmetric eigen-decomposition of the m x m tridiagonal T (Jacobi rotations):
// eigenvalues descending in lam[m], eigenvectors as columns of Y (column-major m x m).
void host_tridiag_eig(int32_t m, const double* alpha, const double* beta, double* lam, double* Y);
// SplitMix64 output i (0-based) of stream seed, as a double in [-1, 1).
double splitmix_pm1(uint64_t seed, uint64_t i);

}  // namespace slr
