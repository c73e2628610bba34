/*
 * slr.h - C ABI of the GB300 (sm_103a) Schur-complement Low-Rank (SLR)
 * preconditioner and SLR-preconditioned CG.
 *
 * Method: R. Li, Y. Xi, Y. Saad, "Schur complement based domain
 * decomposition preconditioners with low-rank corrections", arXiv 1505.04340.
 *
 *   A x = b, A sparse symmetric positive definite (Section 1, Eq. 1.1), or
 *   symmetric indefinite with an SPD interface matrix C (an option; solved by
 *   slr_gmres_solve).
 *   A vertex-based partition (Section 2.1) splits the unknowns into interiors
 *   u_1..u_p and interfaces y; in that order P A P^T = [[B, E], [E^T, C]]
 *   with B = diag(B_i) (Eqs. 2.2-2.3).  C = L L^T, H = L^{-1} E^T B^{-1} E L^{-T}
 *   (Eqs. 3.1-3.2), the k largest eigenpairs (U_k, Lambda_k) of H come from
 *   Lanczos (Section 5.1), and the preconditioner is
 *     M = [[I, 0], [E^T B^{-1}, I]] [[B, E], [0, S~]]                  (Eq. 4.1)
 *     S~^{-1} = L^{-T} ( I/(1-theta) + U_k [(I-Lambda_k)^{-1} - I/(1-theta)] U_k^T ) L^{-1}
 *   (Eq. 4.7 with Lambda~ of Eq. 4.11; theta = lambda_{k+1} or 0 (Eq. 4.10)).
 *
 * Conventions used by every entry point:
 *  - "DD order" is the order of Eq. 2.2: interiors of part 0, ..., part p-1,
 *    then interfaces of part 0, ..., part p-1, then the separator vertices
 *    (part = -1, if any); inside each group nodes keep ascending original
 *    index.  A node of a part is an interface node iff A couples it to a node
 *    of another part (a coupling to a separator vertex keeps it interior);
 *    separator vertices are always interface nodes.
 *  - Multi-column vectors are column-major with leading dimension ld >= rows;
 *    *_dev pointers are caller-owned device memory (e.g. torch tensors) on
 *    the device that was current at slr_setup, *_host pointers are host memory.
 *  - stream is a cudaStream_t (NULL = legacy default stream).  Device work is
 *    enqueued on it; entry points that return host results synchronise it.
 *  - Every call returns an slr_status; nothing throws or aborts.  On failure
 *    slr_last_error_message() describes the cause (thread-local).
 *  - The handle owns all device memory it allocates (factors, U, workspaces);
 *    the caller's host arrays are copied and may be freed after the call.
 */
#ifndef SLR_H
#define SLR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slr_handle_s* slr_handle;

typedef enum {
    SLR_OK = 0,
    SLR_ERR_INVALID_ARG = 1,   /* bad size, pointer, CSR structure or option     */
    SLR_ERR_NOT_SPD = 2,       /* a Cholesky pivot of some B_i or of C was <= 0  */
    SLR_ERR_OOM = 3,           /* device or host allocation failed               */
    SLR_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed    */
    SLR_ERR_NOT_CONVERGED = 5, /* PCG hit maxit; iterations/relres are filled    */
    SLR_ERR_BREAKDOWN = 6,     /* PCG saw p^T A p <= 0 or rho <= 0               */
    SLR_ERR_TIMEOUT = 7,       /* a bounded device-side wait expired             */
    SLR_ERR_UNSUPPORTED = 8    /* a size beyond what the kernels are built for   */
} slr_status;

enum { SLR_THETA_LAMBDA_K1 = 0, SLR_THETA_ZERO = 1 };   /* Eq. 4.11 / Eq. 4.10      */
enum { SLR_PREC_FP64 = 0, SLR_PREC_MIXED = 1 };         /* apply in FP64 / in FP32  */
enum { SLR_U_FP32 = 0, SLR_U_TF32 = 1, SLR_U_BF16 = 2 }; /* low-rank products (u_dtype) */

typedef struct {
    int32_t k;              /* rank of the correction (Section 4); clamped to s           */
    int32_t lanczos_steps;  /* m Lanczos steps; 0 => 5k (Section 6)                       */
    int32_t theta_mode;     /* SLR_THETA_LAMBDA_K1 (default) or SLR_THETA_ZERO            */
    int32_t precision;      /* SLR_PREC_FP64: factors, E, U and apply in FP64.
                               SLR_PREC_MIXED: apply with FP32 factors/E/U and FP32
                               arithmetic; PCG, Lanczos and the (1-lambda)^{-1} scaling
                               stay FP64                                               */
    int32_t nrhs_max;       /* widest right-hand-side block later calls may pass; 0 => 1 */
    int32_t flexible_cg;    /* 1: Polak-Ribiere beta in PCG (for the FP32 apply)          */
    uint64_t seed;          /* SplitMix64 stream of the Lanczos start vector z: v_1 is
                               L^{-1} C z normalised, z_i = 2 u_i - 1 in DD interface
                               order, u_i = (x_i >> 11) 2^-53, x_i output i of the stream */
    int32_t c_leaf;         /* nested-dissection leaf size for C's ordering; 0 => 64     */
    int32_t verbose;        /* 1: setup prints timings to stderr                          */

    /* ---- method options */
    int32_t target_kappa;   /* a target condition number K >= 2 for S S~^{-1} (0 = off): the
                               rank becomes the number of Ritz values above 1 - 1/K, at most
                               k (Section 4, Eq. condk: lambda_{k+1} <= 1 - 1/K keeps the
                               condition number of S S~^{-1} below K); slr_get_info reports
                               the rank used                                             */
    int32_t indefinite;     /* 1: A is symmetric indefinite with an SPD interface matrix C
                               (Section 1; the shifted problems of Section 6): each B_i is
                               factored as L S L^T with S the pivot signs (no pivoting; a
                               zero pivot returns SLR_ERR_BREAKDOWN), H may have eigenvalues
                               >= 1, and the accelerator is slr_gmres_solve.  0 = SPD     */
    int32_t u_dtype;        /* arithmetic of the low-rank products U_k^T W and U_k (d o V)
                               (Eq. 4.7) on right-hand-side blocks of the mixed path:
                               SLR_U_FP32 (default; FP32 CUDA cores), SLR_U_TF32 or
                               SLR_U_BF16 (tensor cores: U and W rounded to TF32 / BF16,
                               products accumulated in FP32; used for blocks of 8 or more
                               right-hand sides, narrower blocks take the FP32 kernel).
                               Must be SLR_U_FP32 with SLR_PREC_FP64                       */

    /* ---- execution choices: each gives the same preconditioner up to rounding; the
       band_* fields, c_persistent, host_loop and autotune give bitwise the same result */
    int32_t band_split;     /* CTAs (a thread-block cluster) per subdomain in the band solve:
                               1, 2 or 4; 0 = automatic                                  */
    int32_t band_slots;     /* shared-memory buffers the band solve streams its factor
                               through: 2..8; 0 = automatic                              */
    int32_t band_threads;   /* threads per band-solve CTA: 512 (one CTA per SM), 256 (two
                               per SM, for more CTAs than SMs) or 32 (one warp per
                               subdomain, for planes of at most 64 rows in one slice;
                               other planes take the automatic choice); 0 = automatic
                               (32 where it applies)                                     */
    int32_t band_order;     /* the order in which the band solve's subdomain clusters are
                               launched (it sets which subdomains share SMs): 1 = subdomain
                               order, 2 = most work first, 3 = most and least work
                               alternating; 0 = automatic (3)                            */
    int32_t band_factor_host; /* where the B_i are factored (Section 5.2): 0 = on the device
                               when every plane is at most 256 rows wide, else on the host;
                               1 = on the host                                           */
    int32_t c_persistent;   /* 1: solve with C's factor in one cooperative launch per
                               direction (grid barriers between level steps) instead of one
                               launch per step                                           */
    int32_t c_levels_only;  /* 1: solve every level of C's factor level by level; 0 = the top
                               levels, as many as fit a fill and setup budget, are solved
                               with an explicit inverse of their block of the factor (one
                               step per direction instead of one per level)              */
    int32_t host_loop;      /* 1: drive the CG loop from the host (one synchronisation per
                               iteration) instead of one CUDA graph per solve            */
    int32_t autotune;       /* 1: setup times the band solve for each split (1, 2, 4 CTAs),
                               CTA size (512 or 256 threads) and buffer count (2, 3, 4) that
                               fit, and both C-solve paths, on this operator, and keeps the
                               fastest; the choice is cached per device, precision and
                               problem shape for the process's life                      */
    int32_t zform;          /* 1: apply S~^{-1} in the form of Proposition 4.3 (Eq. 4.15),
                               (1-theta)^{-1} C^{-1} g + Z_k (d o Z_k^T g) with Z_k = L^{-T} U_k
                               formed at setup: the product Z_k^T g runs beside the two
                               solves with C's factor instead of between them.  The same
                               operator as the default U-form (Eq. 4.7) up to rounding.
                               0 (default): the U-form                                 */
    int32_t band_mma;       /* 0 (default): the band solve runs on the CUDA cores.
                               SLR_U_TF32 or SLR_U_BF16 (mixed path only): blocks of 8 or
                               more right-hand sides are solved with the band factor and
                               the plane vectors rounded to TF32 / BF16 and every block
                               product on the tensor cores, accumulated in FP32; needs the
                               B_i factored on the device (planes of at most 256 rows),
                               else it is not used (slr_info.band_mma says which ran)   */
    int32_t spin_limit;     /* polls of a bounded device wait between steps of the
                               cooperative C solve (c_persistent) before it gives up and
                               reports SLR_ERR_TIMEOUT; 0 = the default (2^22 polls, about a
                               quarter second)                                           */
    int32_t reserved[6];    /* must be 0                                                  */
} slr_opts;

typedef struct {
    int64_t n, n_interior, s, nparts, k, lanczos_steps;   /* sizes; k after clamping      */
    int64_t nnz_A, nnz_E, nnz_C;                          /* nnz(E) counts E only, not E^T */
    int64_t band_entries;        /* stored B-factor entries, sum c_i w_i (w_i + 1)         */
    int64_t c_diag_entries;      /* stored entries of the inverted supernode diagonal blocks */
    int64_t c_panel_entries;     /* stored entries of the supernode off-diagonal panels      */
    int64_t c_supernodes, c_levels;
    int64_t bytes_per_apply;     /* algorithmic bytes one apply of one RHS column reads/writes */
    int64_t flops_per_apply;     /* multiply-adds x 2 of one apply per RHS column          */
    int64_t device_bytes;        /* device memory the handle holds                          */
    double theta;                /* theta used in S~^{-1}                                  */
    double setup_seconds[5];     /* analysis, B factor, C factor, upload, Lanczos          */
    int32_t precision, theta_mode;
    int32_t band_split;          /* CTAs per subdomain in the band solve                    */
    int32_t band_slots;          /* band-solve stream buffers (0: the default)              */
    int32_t c_persistent;        /* 1: C solves in one cooperative launch per direction     */
    int32_t tuned;               /* 1: the three above were chosen by timing (autotune)    */
    double tune_seconds;         /* time the tuning took (0 when taken from the cache)      */
    int32_t band_threads;        /* threads per band-solve CTA (256: two subdomains per SM;
                                    32: a warp per subdomain)                               */
    int32_t c_top_levels;        /* levels of C's factor solved with the explicit inverse   */
    int32_t c_top_positions;     /* interface positions in those levels                     */
    int64_t c_top_entries;       /* stored entries of that inverse (each layout)            */
    int32_t band_on_device;      /* 1: the B_i were factored on the device               */
    double lanczos_seconds[3];   /* setup Lanczos (Section 5.1) split: H applies with the alpha
                                    dot, full reorthogonalisation with the beta norm, the
                                    tridiagonal eigensolve on the host and U_k = V Y_k      */
    int32_t band_mma;            /* the band solve's tensor-core factor in use: 0 (none),
                                    SLR_U_TF32 or SLR_U_BF16 (opts.band_mma)               */
    int32_t u_dtype;             /* the low-rank products' arithmetic (opts.u_dtype)        */
    int64_t vector_bytes_per_column; /* the part of bytes_per_apply that every further column of
                                    a block repeats (vectors, the w values written and
                                    gathered); the factors, U_k and the index arrays are read
                                    once per block: a block of r columns moves
                                    bytes_per_apply + (r - 1) vector_bytes_per_column        */
} slr_info;

/* Fill *opts with defaults: k = 16, m = 5k, theta = lambda_{k+1}, FP64, 1 RHS, seed 1. */
void slr_default_opts(slr_opts* opts);

/* Build the SLR preconditioner of A (Sections 2-5).
 * n, rowptr[n+1], colind[nnz], val[nnz]: host CSR of the FULL symmetric matrix
 *   (both triangles, sorted or unsorted columns, no duplicates), 0-based, n < 2^31.
 * nparts, part[n]: host partition, part[i] in [0, nparts) (vertex-based, Section 2.1),
 * or -1 for a vertex-separator node (a partition with vertex separators, which
 * Section 2.1 notes the method also covers): separator nodes are interface
 * nodes listed after y_p, and a part's node coupled only to its own part and to
 * separators is interior.
 * opts: NULL => defaults.  stream: where the setup's device work runs.
 * *out: new handle on success, NULL on failure.  Errors: INVALID_ARG (sizes,
 * structure, part out of range), NOT_SPD (a pivot <= 0 in B_i or C), OOM, CUDA. */
slr_status slr_setup(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* val,
                     int32_t nparts, const int32_t* part, const slr_opts* opts, void* stream,
                     slr_handle* out);

/* z = M^{-1} r (Eq. 4.1 with the block LU of Eq. 2.4), both in DD order:
 *   t = B^{-1} f;  g' = g - E^T t;  y = S~^{-1} g';  u = t - B^{-1} E y;  z = [u; y].
 * r_dev, z_dev: n x nrhs FP64, leading dimension ld >= n, must not overlap.
 * 1 <= nrhs <= opts.nrhs_max.  Asynchronous on stream. */
slr_status slr_apply(slr_handle h, const double* r_dev, double* z_dev, int32_t nrhs, int32_t ld,
                     void* stream);

/* Solve A x = b with SLR-preconditioned CG (Section 6): x_0 = 0, stop column j
 * when ||r_j|| <= tol ||b_j|| (recurrence residual) or after maxit iterations.
 * The iteration loop runs as one CUDA graph with a device-side WHILE node (built
 * and cached per nrhs on first use, so the first call of each nrhs captures it;
 * make that call outside any stream capture of your own).
 * b_dev, x_dev: n x nrhs FP64 in ORIGINAL order, leading dimension ld.  Columns
 * are independent CG runs advanced together.  iters_out[nrhs], relres_out[nrhs]:
 * host arrays (may be NULL).  Synchronises stream.  Returns NOT_CONVERGED if a
 * column reached maxit, BREAKDOWN if p^T A p <= 0 for a column. */
slr_status slr_pcg_solve(slr_handle h, const double* b_dev, double* x_dev, int32_t nrhs, int32_t ld,
                         double tol, int32_t maxit, void* stream, int32_t* iters_out,
                         double* relres_out);

/* Solve A x = b with SLR-preconditioned GMRES(restart) (Section 6: GMRES(40) for
 * the symmetric indefinite problems, slr_opts.indefinite = 1; it works for SPD A
 * too).  Flexible right preconditioning: z_j = M^{-1} v_j are kept and
 * x = x_0 + Z_j y, so an FP32 apply (varying by rounding) does not spoil the
 * minimal-residual property.  Arnoldi orthogonalises by two classical
 * Gram-Schmidt passes; the Hessenberg least-squares problem is solved on the
 * host by Givens rotations.  x_0 = 0; a column stops when the residual estimate
 * satisfies ||r|| <= tol ||b|| or after maxit products with A; relres_out[j] is
 * the true ||b - A x|| / ||b|| at exit.  Columns run one after another.
 * b_dev, x_dev: n x nrhs FP64 in ORIGINAL order, leading dimension ld; nrhs <=
 * nrhs_max; 1 <= restart <= 1000.  iters_out[nrhs], relres_out[nrhs]: host arrays
 * (may be NULL).  Allocates its Krylov basis (2 restart + 1 vectors of n) per call.
 * Synchronises stream.  Returns NOT_CONVERGED if a column reached maxit. */
slr_status slr_gmres_solve(slr_handle h, const double* b_dev, double* x_dev, int32_t nrhs, int32_t ld,
                           double tol, int32_t maxit, int32_t restart, void* stream, int32_t* iters_out,
                           double* relres_out);

/* Continuous batching at iteration granularity: the handle's nrhs_max CG columns
 * serve as "slots", each an independent run of the CG of Section 6 (x_0 = 0,
 * stop when ||r|| <= tol ||b|| or after maxit iterations), which can be started
 * while other slots are mid-solve.  A slot runs exactly the arithmetic of a
 * column of slr_pcg_solve, so its answer does not depend on which other slots
 * ran beside it.  The slots share the handle's CG workspaces with slr_pcg_solve
 * and slr_gmres_solve: a call of either discards every slot's state.
 *
 * slr_cg_slot_start: load b_dev (n FP64, original order) into slot `slot`
 *   (0 <= slot < nrhs_max) with its own tol and maxit; asynchronous on stream.
 * slr_cg_advance: run `iters` CG iterations over slots 0 .. width-1 (finished or
 *   unused slots cost an apply column but change nothing), then report per slot
 *   active_out (1: still iterating), iters_out (its iterations so far),
 *   relres_out (||r|| / ||b||, recurrence residual) and status_out (1: met its
 *   tolerance, 2: breakdown p^T A p <= 0, 0: still running or stopped at maxit);
 *   any output may be NULL; synchronises stream.
 * slr_cg_slot_result: x of the slot (n FP64, original order) into x_dev;
 *   asynchronous on stream.
 * Errors: INVALID_ARG (bad slot, width, pointer, tol or maxit; advance before any
 * start), TIMEOUT (a bounded device wait expired), CUDA. */
slr_status slr_cg_slot_start(slr_handle h, int32_t slot, const double* b_dev, double tol, int32_t maxit,
                             void* stream);
slr_status slr_cg_advance(slr_handle h, int32_t iters, int32_t width, void* stream, int32_t* active_out,
                          int32_t* iters_out, double* relres_out, int32_t* status_out);
slr_status slr_cg_slot_result(slr_handle h, int32_t slot, double* x_dev, void* stream);

/* t = B^{-1} f for the interior block (Section 5.2), DD interior order,
 * f_dev/t_dev: n_interior x nrhs FP64, leading dimension ld.  May alias. */
slr_status slr_bsolve(slr_handle h, const double* f_dev, double* t_dev, int32_t nrhs, int32_t ld,
                      void* stream);

/* y = C^{-1} g = L^{-T} L^{-1} g for the interface block (Section 5.2),
 * DD interface order, s x nrhs FP64, leading dimension ld.  May alias. */
slr_status slr_csolve(slr_handle h, const double* g_dev, double* y_dev, int32_t nrhs, int32_t ld,
                      void* stream);

/* y = S~^{-1} g (Eq. 4.7), DD interface order, s x nrhs FP64, leading dim ld. */
slr_status slr_stilde_solve(slr_handle h, const double* g_dev, double* y_dev, int32_t nrhs,
                            int32_t ld, void* stream);

/* Replace the low-rank part by caller-given eigenpairs (Section 5.3: an SLR
 * preconditioner is improved by changing its vectors, not its factors).
 * Z_host: s x k column-major, DD interface order, C-orthonormal columns
 * Z_k = L^{-T} U_k of Proposition 4.3 (independent of how C is ordered);
 * lam_host[k]: lambda_1..lambda_k, each in [0, 1); theta in [0, 1).
 * 0 <= k <= s.  The handle stores U_k = L^{-1} C Z_k in its own ordering.
 * Synchronises stream. */
slr_status slr_set_lowrank(slr_handle h, int32_t k, const double* Z_host, const double* lam_host,
                           double theta, void* stream);

/* Improve the preconditioner by adding vectors (Section 5.3: its low-rank
 * part grows without discarding the vectors it has).  Runs FP64 Lanczos with
 * full reorthogonalisation on the deflated operator (I - U_k U_k^T) H (I - U_k U_k^T),
 * lanczos_steps steps (0: 5 k_add, at most s - k), started from L^{-1} C z with z
 * from SplitMix64 stream seed + (number of earlier calls) + 1, projected out of
 * span(U_k); appends its leading min(k_add, steps) Ritz pairs to (Lambda_k, U_k);
 * with theta = lambda_{k+1} (Eq. 4.11) theta becomes the next Ritz value of that
 * run.  *added_out (may be NULL): vectors added.  The handle's CUDA graphs are
 * rebuilt on the next solve.  Synchronises stream.  Errors: INVALID_ARG
 * (k_add < 0), OOM, CUDA. */
slr_status slr_add_vectors(slr_handle h, int32_t k_add, int32_t lanczos_steps, void* stream, int32_t* added_out);

/* Export the low-rank part: Z_host (s x k column-major, DD interface order,
 * may be NULL), lam_host[k+1] (Ritz values lambda_1..lambda_{k+1} from Lanczos,
 * the last 0 when unavailable; may be NULL), *theta_out (may be NULL). */
slr_status slr_get_lowrank(slr_handle h, double* Z_host, double* lam_host, double* theta_out,
                           void* stream);

/* All Ritz values of the setup Lanczos run, descending (after slr_add_vectors:
 * lambda_1..lambda_k, then the last deflated run's remaining Ritz values);
 * lam_host has room for info.lanczos_steps values; *count_out gets how many. */
slr_status slr_get_ritz(slr_handle h, double* lam_host, int32_t* count_out);

/* perm_host[n]: DD position -> original index (new -> old), Eq. 2.2. */
slr_status slr_get_perm(slr_handle h, int32_t* perm_host);

slr_status slr_get_info(slr_handle h, slr_info* info);

/* Host-only analysis (no GPU needed): interface detection and the DD order
 * of Eq. 2.2.  perm_out[n] (new -> old), int_off[nparts+1] and
 * ifc_off[nparts+1] (offsets of u_i in u and of y_i in y), *s_out = interface
 * size.  Any output pointer may be NULL. */
slr_status slr_dd_order(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts,
                        const int32_t* part, int32_t* perm_out, int32_t* int_off, int32_t* ifc_off,
                        int32_t* s_out);

/* z = M^{-1} r exactly as slr_apply, for callers that cannot let device memory
 * be allocated while they run: a process whose device memory is handed to an
 * allocator it does not control (a fixed arena set up at start-up), or a server
 * that must not grow its device footprint while it answers requests.  It
 * allocates nothing: its per-call scratch (band-solve intermediates, interface
 * vectors, panel products, reduction partials) is carved from one file-scope
 * __device__ array of 32 MiB that every GPU loading this library holds until
 * exit, instead of the handle's workspaces.  The paper has no counterpart; this
 * is a deployment variant of the apply of Eq. 4.1.
 * Same arguments, layout and ownership as slr_apply.  Errors: INVALID_ARG as
 * slr_apply; UNSUPPORTED (nothing launched) when the scratch for this handle
 * and nrhs exceeds 32 MiB.  slr_setup looks up the array's device address
 * (cudaGetSymbolAddress, with the handle's device current) and keeps it in the
 * handle, so this call looks nothing up; a cudaDeviceReset ends the handle and
 * the address with it.  Every call shares the one array and no part of it needs
 * to start at zero (each call writes what it reads, and clears its arrival
 * counters); calls that overlap on the GPU, from any thread, stream or handle,
 * race on it. */
slr_status slr_apply_noalloc(slr_handle h, const double* r_dev, double* z_dev, int32_t nrhs, int32_t ld,
                             void* stream);

/* The device status word of the handle's operator after the calls enqueued on
 * stream so far: SLR_OK, or SLR_ERR_TIMEOUT when a bounded device wait expired
 * (a band-solve copy that did not land within its bound, or a grid-barrier wait
 * of the cooperative C solve beyond opts.spin_limit polls); the outputs of the
 * call that saw it are then invalid.  Every call that runs the operator
 * (slr_apply, slr_apply_noalloc, slr_bsolve, slr_csolve, slr_stilde_solve,
 * slr_pcg_solve, slr_gmres_solve) clears the word on its stream before its
 * kernels; slr_pcg_solve, slr_gmres_solve, slr_setup and slr_add_vectors read
 * it themselves and return SLR_ERR_TIMEOUT.  Synchronises stream.  Bookkeeping
 * of the device kernels' bounded waits; the paper has no counterpart. */
slr_status slr_device_status(slr_handle h, void* stream);

/* Fault injection for tests of the error paths (the paper has no counterpart):
 * the nth device allocation this library makes from now on, counting every
 * handle in the process, fails as if the device were out of memory (the call
 * making it returns SLR_ERR_OOM and releases what it holds); nth <= 0 turns
 * the injection off.  One failure per call of this function. */
void slr_inject_alloc_failure(int64_t nth);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles, all devices).  Lets a caller count the launches of a region. */
int64_t slr_kernel_launches(void);

void slr_destroy(slr_handle h);
const char* slr_status_str(slr_status s);
const char* slr_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* SLR_H */
