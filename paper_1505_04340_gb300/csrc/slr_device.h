// Device-resident SLR handle and the launchers of the hot-path kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "slr_internal.h"

namespace slr {

// Supernodal factor of C on the device, values in precision T.
template <typename T>
struct DevCFactor {
    int32_t s = 0, ns = 0, nlev = 0;
    int32_t* cperm = nullptr;      // factor position -> DD interface index
    int32_t* ciperm = nullptr;     // DD interface index -> factor position
    int32_t* c0 = nullptr;         // [ns+1]
    int64_t* r_off = nullptr;      // [ns+1]
    int32_t* rows = nullptr;       // R_J
    int64_t* pan_off = nullptr;    // [ns+1]
    T* panel = nullptr;            // M_J = L[R_J, J] L_JJ^{-1}, row-major |R_J| x n_J
    int64_t* dinv_off = nullptr;   // [ns+1]
    T* dinv = nullptr;             // packed lower, column-major
    int64_t* seg_ptr = nullptr;    // [s+1]
    int32_t* seg_row = nullptr;    // panel rows holding each position
    int64_t nrow = 0;              // panel rows in total
    int32_t max_n = 0;             // widest supernode (shared memory of a forward task: t_J)
    T* wbuf = nullptr;             // [nrow x nrhs_max] panel products M_J t_J of the forward solve
    T* tws = nullptr;              // [s x nrhs_max] t_J gathered once per level (per-level forward tasks)
    T* gfs = nullptr;              // [s x nrhs_max] the forward's input g in factor order, a row per position
    std::vector<int32_t> lev_maxn; // widest supernode of each level (0 for the fused small levels)
    int4* tasks = nullptr;         // (supernode, first column, count <= 32, 0)
    int4* ptasks = nullptr;        // (supernode, first panel row, count <= 32, 0)
    std::vector<int32_t> lev_task_ptr;    // host copies, [nlev+1]
    std::vector<int32_t> lev_ptask_ptr;
    std::vector<int32_t> lev_sn_ptr;
    std::vector<uint8_t> lev_small;
    int32_t* lev_sn = nullptr;            // device: supernodes level by level
    // the persistent (one launch per direction) solves
    int32_t *d_lev_task_ptr = nullptr, *d_lev_ptask_ptr = nullptr, *d_lev_sn_ptr = nullptr;   // device copies
    uint8_t* d_lev_small = nullptr;
    int32_t nsteps_fwd = 0, nsteps_bwd = 0;   // dependent steps (grid barriers + 1)
    int32_t max_cta_tasks = 1;                // most CTA tasks of any step (caps the grid)
    unsigned* bar = nullptr;                  // grid barrier counter, zeroed before each launch
    int32_t* err = nullptr;                   // the operator's status word
    long long grid_spin = 1ll << 22;          // polls of a grid-barrier wait (opts.spin_limit)
    // top zone (levels >= top_lev): explicit inverse of L_TT, one step per direction
    int32_t top_lev = 0, nT = 0;
    int32_t *tpos = nullptr, *tseg_row = nullptr, *tsk_lo = nullptr, *tp_pos = nullptr, *tb_cb_part = nullptr;
    int64_t *tseg_ptr = nullptr, *tsk_off = nullptr, *tb_off = nullptr, *tp_off = nullptr;
    T *tsk = nullptr, *tb = nullptr;          // forward row skyline, backward block columns
    int4 *tf_rb = nullptr, *tf_tasks = nullptr, *tb_cb = nullptr, *tb_tasks = nullptr;
    int32_t n_tf_rb = 0, n_tf_tasks = 0, n_tb_cb = 0, n_tb_tasks = 0, tf_parts = 0, tb_parts = 0;
    T *tT = nullptr, *tf_part = nullptr, *tb_part = nullptr;   // workspaces of nrhs_max columns
    int32_t *tf_cnt = nullptr, *tb_cnt = nullptr;              // arrival counters, zero between solves
    int32_t ws_cols = 0;                      // right-hand sides the workspaces (wbuf and the zone's) hold
    bool per_level = true;                    // one launch per level step (else one cooperative launch)
    int32_t nsm = 152;                        // SMs of the device (CTA size of the per-level kernels)
    std::vector<int32_t> lev_stage;           // fused levels: shared stage buffer (elements) of a supernode's block
    int32_t stage_cap = 0;                    // the largest of them (persistent kernels)
};

// Everything one apply needs in precision T (double: FP64 path; float: mixed).
template <typename T>
struct DevOperator {
    BandBlock* band = nullptr;     // [p]
    T* bfac = nullptr;
    int32_t band_G = 1;            // CTAs per subdomain (thread-block cluster size)
    int32_t band_nbuf = 0;         // ring slots of the band solve (0: the default count)
    int32_t band_nt = 512;         // threads per band-solve CTA: 512 (one per SM) or 256 (two per SM)
    int32_t* err = nullptr;        // device status word: 1 = a bounded wait expired
    int32_t *e_rp = nullptr, *e_ci = nullptr;  T* e_v = nullptr;     // E   (nI x s)
    int32_t *et_rp = nullptr, *et_ci = nullptr; T* et_v = nullptr;   // E^T (s x nI)
    DevCFactor<T> cf;
    T* U = nullptr;                // s x k column-major, factor order
    T* Zdd = nullptr;              // Z_k = L^{-T} U_k, s x k column-major, DD interface order (Z-form only)
    T* dvec = nullptr;             // [k] (1-lambda_i)^{-1} - (1-theta)^{-1}, from FP64
    T cinv = 1;                    // (1-theta)^{-1}
    // workspaces, nrhs_max columns each, leading dimension = rows
    T *wr = nullptr, *wz = nullptr;          // n: converted input / output (mixed only)
    T *tB = nullptr, *eb = nullptr;          // nI
    T *gp = nullptr, *wf = nullptr, *xf = nullptr;   // s
    T *vk = nullptr, *part = nullptr;        // k x r, partial sums (lowrank_part_elems)
    // tensor-core low-rank products (FP32 apply, opts.u_dtype TF32 or BF16): U in the
    // operand type, row-major (pass 2) and, for BF16, column-major (pass 1)
    int32_t u_dtype = 0;
    void *U_tc_rm = nullptr, *U_tc_cm = nullptr;
    // tensor-core band solve for blocks of >= 8 right-hand sides (FP32 apply,
    // opts.band_mma TF32 or BF16): sub-tile table in launch order and the packed factor
    int32_t band_mma = 0;
    BandTcBlock* band_tc = nullptr;
    unsigned char* band_tc_fac = nullptr;
    int64_t band_tc_bytes = 0;
    int32_t band_tc_wmax = 0;
    bool ready = false;
};

}  // namespace slr

struct slr_handle_s {
    int device = 0;
    slr_opts opts;
    cudaStream_t stream = nullptr;   // stream of the setup or set_lowrank call in progress
    slr::HostSetup hs;               // sizes, permutation, CSR blocks (host copies)
    int32_t k = 0, m_steps = 0, nritz = 0;
    int32_t improvements = 0;        // slr_add_vectors calls so far (their start-vector streams)
    double theta = 0.0;
    std::vector<double> ritz;        // all Ritz values, descending
    std::vector<double> lam;         // lambda_1..lambda_k
    slr::DevOperator<double> op64;
    slr::DevOperator<float> op32;
    // FP64 extras: C in DD interface order (for the start vector and set_lowrank)
    int32_t *c_rp = nullptr, *c_ci = nullptr; double* c_v = nullptr;
    // PCG state (DD order, n x nrhs_max) and scalars
    int32_t *perm = nullptr, *a_rp = nullptr, *a_ci = nullptr; double* a_v = nullptr;
    double *px = nullptr, *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr;
    // single-precision preconditioner: r rounded to FP32 (the apply's input, written by
    // the r update) and the apply's output z, kept in FP32 (pz is then not allocated)
    float *pr32 = nullptr, *pz32 = nullptr;
    double *scal = nullptr;          // per-column scalars, see slr_api.cu
    double *dpart = nullptr;         // reduction partials
    int32_t *iflags = nullptr;       // per-column status words
    double* ctl = nullptr;           // PCG graph controls: tol^2, maxit
    double* slot_ctl = nullptr;      // slot CG: tol^2 and maxit of each slot (2 x nrhs_max)
    bool slots_live = false;         // the CG workspaces hold slot state (cleared by pcg / gmres)
    struct PcgGraph {
        int32_t nrhs = 0;
        cudaGraphExec_t exec = nullptr;
        int64_t kA = 0, kB = 0;      // kernels per iteration: test part, update part
    };
    std::vector<PcgGraph> pcg_graphs;   // one per right-hand-side count, built on first use
    std::vector<void*> allocs;       // every device allocation, freed by slr_destroy
    int64_t device_bytes = 0;
    double setup_seconds[5] = {0, 0, 0, 0, 0};
    int64_t bytes_per_apply = 0, flops_per_apply = 0, vector_bytes_per_column = 0;
    bool tuned = false;
    double tune_seconds = 0.0;
    // band factorization on the device: per-subdomain plane blocks D_J and O_J
    // (kept through setup so that a repack for another split needs no refactoring)
    double* bf_scr = nullptr;
    int64_t bf_scr_len = 0;
    int64_t* bf_soff = nullptr;
    bool band_on_device = false;     // the B_i were factored on the device
    double lanczos_seconds[3] = {0, 0, 0};   // setup Lanczos: H applies, reorthogonalisation, eigensolve + U_k
    void* noalloc_base = nullptr;    // device address of slr_apply_noalloc's scratch array (slr_noalloc.cu)
    // Z-form apply: Z_k^T g' runs on aux beside the C solves (fork and join events)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace slr {

// Looks up the device address of slr_apply_noalloc's scratch array in the
// current context and stores it in h->noalloc_base (slr_noalloc.cu).
slr_status noalloc_lookup(slr_handle h);

// Kernel launches of the library: a process-wide count, and the calling
// thread's own count (a graph capture takes back what its thread captured).
void count_launches(int64_t n);
int64_t thread_launches();

constexpr int kRedBlocks = 256;     // fixed grid of the deterministic reductions

// ---- K1: batched banded B_i solves (out = B^{-1} in, or out = base - B^{-1} in)
template <typename T>
cudaError_t launch_band_solve(const DevOperator<T>& op, int32_t p, int32_t wmax, const T* in, int64_t ldi,
                              T* out, int64_t ldo, const T* base, int64_t ldb, int32_t nrhs,
                              cudaStream_t st);
// shared memory one band-solve CTA needs for plane width wmax and nr columns per pass
// ---- K1 on the tensor cores (slr_band_tc.cu): the sub-tile layout of the band
// factor (per subdomain, in the given launch order; *bytes: factor size), its
// pack kernel from the device plane blocks, and the solve of 8-64 columns at a time
std::vector<BandTcBlock> band_tc_layout(const std::vector<BandBlock>& run_order, int32_t mma_dtype, int64_t* bytes);
cudaError_t launch_band_tc_pack(int32_t mma_dtype, const BandTcBlock* band, int32_t p, int32_t cmax,
                                const double* scr, const int64_t* soff, unsigned char* fac, bool indef,
                                cudaStream_t st);
// K1 with one warp per subdomain, for planes of at most 64 rows packed as one slice (slr_band_warp.cu)
template <typename T>
cudaError_t launch_band_warp(const DevOperator<T>& op, int32_t p, const T* in, int64_t ldi, T* out, int64_t ldo,
                             const T* base, int64_t ldb, int32_t nrhs, cudaStream_t st);
cudaError_t launch_band_solve_tc(const DevOperator<float>& op, int32_t p, const float* in, int64_t ldi, float* out,
                                 int64_t ldo, const float* base, int64_t ldb, int32_t nrhs, cudaStream_t st);
// ---- K2: gp = g - E^T t (g == NULL: gp = E^T t) ;  eb = E y
template <typename T>
cudaError_t launch_gather_et(const DevOperator<T>& op, int32_t s, const T* g, int64_t ldg, const T* t,
                             int64_t ldt, T* gp, int64_t ldgp, int32_t nrhs, cudaStream_t st);
template <typename T>
cudaError_t launch_spmv_e(const DevOperator<T>& op, int32_t nI, const T* y, int64_t ldy, T* out,
                          int64_t ldo, int32_t nrhs, cudaStream_t st);
// ---- band factorization on the device (slr_band_factor.cu): the plane blocks of
// every B_i into scr (per subdomain at soff[i]: S (W^2), then D_J for every plane,
// then O_J, then the pivot signs (c W)); *bad receives a subdomain whose pivot is
// not positive, or zero when indef (it must hold -1)
cudaError_t launch_band_factor(const BandBlock* band, int32_t p, const int32_t* a_rp, const int32_t* a_ci,
                               const double* a_v, double* scr, const int64_t* soff, int32_t* bad, bool indef,
                               cudaStream_t st);
// packs them into the tiled slice layout of `band` (split G) in precision T, the
// pivot signs folded into the forward blocks when indef; bfac must be zeroed first
// (slices shorter than the widest keep zeros)
template <typename T>
cudaError_t launch_band_pack(const BandBlock* band, int32_t p, int32_t cmax, int32_t G, const double* scr,
                             const int64_t* soff, T* bfac, bool indef, cudaStream_t st);
// ---- K3: C solves.  fwd: xf = L^{-1} P g (g in DD order, xf in factor order)
//              bwd: xf = L^{-T} yf (factor order), optional scatter to DD order y_dd
// xf, yf: s x nrhs (leading dimension s); yf is read only and must not overlap xf.
// The forward solve also writes cf.wbuf and both use the top zone's workspaces,
// which hold cf.ws_cols (= nrhs_max) columns: a wider call returns
// cudaErrorInvalidValue without launching anything.
template <typename T>
cudaError_t launch_c_forward(const DevCFactor<T>& cf, const T* g_dd, int64_t ldg, T* xf, int32_t nrhs,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_c_backward(const DevCFactor<T>& cf, const T* yf, T* xf, T* y_dd, int64_t ldy,
                              int32_t nrhs, cudaStream_t st);
// ---- K4: w' = cinv w + U (d o (U^T w)) in factor order (in place on w)
template <typename T>
cudaError_t launch_lowrank(const DevOperator<T>& op, int32_t s, int32_t k, T* w, int32_t nrhs,
                           cudaStream_t st);
// its two passes on a basis Ub (s x k column-major) and a block w (leading dimension
// ldw): op.vk = d o (Ub^T w), then w = cinv w + Ub op.vk (the Z-form of Proposition 4.3
// runs them on Z_k, the first beside the C solves)
template <typename T>
cudaError_t launch_lowrank_v(const DevOperator<T>& op, int32_t s, int32_t k, const T* Ub, const T* w, int64_t ldw,
                             int32_t nrhs, cudaStream_t st);
template <typename T>
cudaError_t launch_lowrank_update(const DevOperator<T>& op, int32_t s, int32_t k, const T* Ub, T* w, int64_t ldw,
                                  int32_t nrhs, cudaStream_t st);
// elements of op.part that launch_lowrank needs for rank k and nrhs columns
int64_t lowrank_part_elems(int32_t s, int32_t k, int32_t nrhs);
// the tensor-core variant (slr_lowrank_tc.cu): usable for u_dtype TF32/BF16, 8..64
// right-hand sides and k <= 128; the pack kernel fills U_tc_rm (and U_tc_cm for
// BF16) from the FP64 U (s x k column-major)
bool lowrank_tc_usable(const DevOperator<float>& op, int32_t k, int32_t nrhs);
cudaError_t launch_lowrank_tc(const DevOperator<float>& op, int32_t s, int32_t k, float* w, int32_t nrhs,
                              cudaStream_t st);
size_t lowrank_tc_elem(int32_t u_dtype);
cudaError_t launch_lowrank_tc_pack(int32_t u_dtype, int32_t s, int32_t k, const double* U, void* Urm, void* Ucm,
                                   cudaStream_t st);
// ---- helpers
template <typename TS, typename TD>
cudaError_t launch_convert(int64_t rows, int32_t cols, const TS* src, int64_t lds, TD* dst, int64_t ldd,
                           cudaStream_t st);
cudaError_t launch_permute(int32_t n, int32_t nrhs, const int32_t* idx, const double* src, int64_t lds,
                           double* dst, int64_t ldd, bool gather, cudaStream_t st);
cudaError_t launch_csr_spmv(int32_t n, const int32_t* rp, const int32_t* ci, const double* v,
                            const double* x, int64_t ldx, double* y, int64_t ldy, int32_t nrhs,
                            cudaStream_t st);
// dots: out[j] = sum_i a[i + j lda] b[i + j ldb], deterministic two-stage reduction
cudaError_t launch_dots(int64_t n, int32_t cols, const double* a, int64_t lda, const double* b,
                        int64_t ldb, double* part, double* out, int32_t out_stride, cudaStream_t st);
// Lanczos helpers: h = V[:, :j]^T w ; w -= V[:, :j] h  (V column-major, ld = s)
cudaError_t launch_gemv_t(int32_t s, int32_t j, const double* V, const double* w, double* part,
                          double* h, cudaStream_t st);
cudaError_t launch_gemv_n_sub(int32_t s, int32_t j, const double* V, const double* h, double* w,
                              cudaStream_t st);
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);
// U (s x k) = V (s x m) Y (m x k), column-major
cudaError_t launch_gemm_nn(int32_t s, int32_t m, int32_t k, const double* V, const double* Y, double* U,
                           cudaStream_t st);

// ---- PCG (DD order), per-column scalars; see slr_api.cu for the scalar layout
cudaError_t launch_pcg_alpha(int32_t nrhs, double* scal, int32_t* flags, cudaStream_t st);
cudaError_t launch_pcg_update_xr(int32_t n, int32_t nrhs, double* x, double* r, const double* p,
                                 const double* q, const double* scal, const int32_t* flags,
                                 cudaStream_t st);
cudaError_t launch_pcg_check(int32_t nrhs, double* scal, int32_t* flags, int32_t it, double tol,
                             cudaStream_t st);
cudaError_t launch_pcg_beta(int32_t nrhs, double* scal, int32_t* flags, int32_t flexible,
                            cudaStream_t st);
cudaError_t launch_pcg_init(int32_t nrhs, const double* scal, int32_t* flags, cudaStream_t st);
cudaError_t launch_pcg_check_graph(int32_t nrhs, const double* scal, int32_t* flags, const double* ctl,
                                   cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hi,
                                   cudaStream_t st);
cudaError_t launch_pcg_update_p(int32_t n, int32_t nrhs, double* p, const double* z, const double* scal,
                                const int32_t* flags, cudaStream_t st);
// Fused CG vector kernels (slr_pcg.cu), column j of each vector at offset j n; the
// dots use one fixed two-stage reduction whatever kernel forms them.
// out[j stride] = a_j . b_j, b in FP64 or FP32 (widened before the product)
template <typename TB>
cudaError_t launch_pcg_dot(int64_t n, int32_t cols, const double* a, const TB* b, double* part, double* out,
                           int32_t out_stride, cudaStream_t st);
// q = A p (CSR) and scal[8 j + 1] = p_j . q_j
cudaError_t launch_pcg_spmv_dot(int64_t n, int32_t nrhs, const int32_t* rp, const int32_t* ci, const double* v,
                                const double* p, double* q, double* part, double* scal, cudaStream_t st);
// active columns: x += alpha p, r -= alpha q, r32 = fl32(r) (r32 may be null); every column:
// scal[8 j + 3] = r.r and, z not null, scal[8 j + 7] = r.z; part holds 2 nrhs kRedBlocks values
template <typename TZ>
cudaError_t launch_pcg_xr_dots(int64_t n, int32_t nrhs, double* x, double* r, const double* p, const double* q,
                               float* r32, const TZ* z, double* scal, const int32_t* flags, double* part,
                               cudaStream_t st);
// active columns: p = z + beta p
template <typename TZ>
cudaError_t launch_pcg_update_pz(int64_t n, int32_t nrhs, double* p, const TZ* z, const double* scal,
                                 const int32_t* flags, cudaStream_t st);
// slot CG (continuous batching, slr_cg_*): start slot j; per-slot test after an iteration
cudaError_t launch_cg_slot_init(int32_t j, double tol, int32_t maxit, double* scal, int32_t* flags, double* ctl,
                               cudaStream_t st);
cudaError_t launch_cg_slot_check(int32_t width, int32_t count_at, const double* scal, int32_t* flags,
                                 const double* ctl, cudaStream_t st);

}  // namespace slr
