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
    int32_t id = 0;       // the subdomain i (blocks may be launched in another order)
    uint8_t nrb[4] = {0, 0, 0, 0};   // row blocks of each slice (at most 8: 256 rows)
    uint8_t rbmap[4][8] = {};        // block of slice g's local row block rb
};

// The tensor-core band solve's view of a subdomain (slr_band_tc.cu): its factor is
// stored as 4096-byte sub-tiles (128 rows x one K-step) from byte foff on, per plane
// [O_J: nU | D_J: nL | O_J^T: nL | D_J^T: nU] sub-tiles.
struct BandTcBlock {
    int32_t m = 0, w = 0, c = 0, row0 = 0, id = 0;
    int32_t nU = 0, nL = 0;      // sub-tiles of an upper / a lower block
    int64_t foff = 0;            // bytes
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
// The blocks in the order their clusters are launched: 1 = subdomain order,
// 2 = heaviest first, 3 = heaviest and lightest alternating (work c W (W+1)).
std::vector<BandBlock> band_run_order(const std::vector<BandBlock>& band, int mode);
// The order opts.band_order = 0 selects: with two CTAs per SM the most and
// least loaded subdomains tend to share SMs (FP64 3-D 64^3: 326 us per B-solve
// instead of 370 in subdomain order; the HBM-bound FP32 solve does not change).
constexpr int kBandOrderAuto = 3;

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
    std::vector<double> panel;         // M_J = L[R_J, J] L_JJ^{-1} (unit block factor, see below)
    std::vector<int64_t> dinv_off;     // [ns+1] offsets of the packed inverse blocks
    std::vector<double> dinv;          // L_JJ^{-1}: lower triangle, column-major, packed
    // With Lhat = L D^{-1} (D = diag(L_JJ), unit diagonal blocks, off-diagonal
    // blocks M_J) the solves are L^{-1} = D^{-1} Lhat^{-1} and L^{-T} = Lhat^{-T} D^{-T}:
    // forward  t_J = g_J - sum_K M_K[rows in J] t_K,  x_J = L_JJ^{-1} t_J
    // backward x_J = L_JJ^{-T} y_J - M_J^T x_{R_J}
    // so each level is one dependent step in either direction.
    // Forward solve: after level l, w[r_off[K] + p] = M_K[p, :] t_K for its supernodes K;
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
    // Top zone: the supernodes of levels >= top_lev (closed under parents) are
    // solved with an explicit inverse of their diagonal block L_TT of L (a
    // partitioned inverse): forward x_T = L_TT^{-1} t_T with t_T = g_T - L_TS x_S,
    // backward y_T = L_TT^{-T} x_T, so the zone costs one step per direction
    // (plus the gather of t_T) instead of one per level.  Local index la of the
    // zone's positions follows the factor order; the zone of a supernode's
    // subtree then covers one contiguous range of local indices.
    int32_t top_lev = 0;               // = nlev when there is no zone
    int32_t nT = 0;                    // positions in the zone
    std::vector<int32_t> tpos;         // [nT] local index -> factor position
    std::vector<int64_t> tseg_ptr;     // [nT+1] gather lists of the zone's rows, restricted to
    std::vector<int32_t> tseg_row;     //   panel rows of supernodes outside the zone
    std::vector<int64_t> tsk_off;      // [nT+1] forward, row skyline: row la of L_TT^{-1} holds
    std::vector<int32_t> tsk_lo;       //   local columns tsk_lo[la] .. la, starting at tsk_off[la]
    std::vector<double> tsk;
    std::vector<int32_t> tf_rb;        // forward row blocks, 4 ints: first row, count (<= 32),
                                       //   chunks, partial-sum offset
    std::vector<int32_t> tf_tasks;     // 4 ints: row block, first column, end column, chunk
    std::vector<int64_t> tb_off;       // [ns+1] backward: block column of J (zone only), row-major
    std::vector<double> tb;            //   |path_J| x n_J, path_J = rows of J, then of its ancestors
    std::vector<int64_t> tp_off;       // [ns+1] factor positions of the path rows
    std::vector<int32_t> tp_pos;
    std::vector<int32_t> tb_cb;        // backward column blocks, 4 ints: J, first column, count, chunks
    std::vector<int32_t> tb_cb_part;   //   partial-sum offset of each column block
    std::vector<int32_t> tb_tasks;     // 4 ints: column block, first path row, end path row, chunk
    int32_t tf_parts = 0, tb_parts = 0;   // partial sums per right-hand side
};
constexpr int32_t kTopCW = 512;        // forward: columns per chunk of a 32-row block
constexpr int32_t kTopRCH = 256;       // backward: path rows per chunk of a 32-column block
constexpr double kTopEntries = 2.0;    // zone inverse at most this many times the factor's entries
constexpr double kTopFmas = 1.5e10;    // and at most this many host multiply-adds to build
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
    std::vector<int32_t> band_w;          // half-bandwidth of each B_i
    int64_t bfac_len = 0;                 // elements of the packed band factor (one precision)
    bool indefinite = false;              // A symmetric indefinite with an SPD interface C:
                                          // B_i = L S L^T, S the pivot signs, folded into the
                                          // forward blocks (O_J S_{J-1} and S_J D_J^{-1})
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
// Plane geometry and slice layout of every B_i for G CTAs per subdomain (band,
// band_w, wmax, band_G, bfac_len); host_band_factor then factors and packs on the host.
void host_band_layout(HostSetup& hs, int32_t G);
slr_status host_band_factor(HostSetup& hs, int32_t G);
slr_status host_c_factor(HostSetup& hs, int32_t leaf, int32_t task_rows);
// Lowest level of the top zone within the entry and multiply-add budgets (nlev: no zone).
int32_t host_c_top_choose(const CFactorHost& cf);
// Builds the top zone from level top_lev up (no zone when top_lev >= nlev or
// when the zone's subtrees are not contiguous in the factor order).
void host_c_top(CFactorHost& cf, int32_t top_lev);
// Symmetric eigen-decomposition of the m x m tridiagonal T (implicit QL):
// eigenvalues descending in lam[m], eigenvectors as columns of Y (column-major m x m).
void host_tridiag_eig(int32_t m, const double* alpha, const double* beta, double* lam, double* Y);
// SplitMix64 output i (0-based) of stream seed, as a double in [-1, 1).
double splitmix_pm1(uint64_t seed, uint64_t i);

}  // namespace slr
