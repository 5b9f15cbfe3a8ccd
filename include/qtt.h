/*
 * qtt.h -- C ABI of the GB300 library for the QTT (quantics tensor-train) fractional-step
 * method for incompressible flow around a cylinder on a curvilinear O-grid
 * (arXiv:2507.05222).
 *
 * Objects
 *   qtt_ctx  -- one CUDA device, one stream, one device memory pool.  All calls on a
 *               context are enqueued on its stream, in order; none blocks the host unless
 *               its description says so.  A context must be used by one host thread at a time.
 *   qtt_mps  -- a TT-vector (matrix product state, eq:simpleMPS): n cores A[k] of shape
 *               (r_{k-1}, d, r_k), r_0 = r_n = 1, stored row-major with the left bond slowest.
 *               Core 1 carries the most significant bit (App. D).
 *   qtt_mpo  -- a TT-matrix (eq:simpleMatrix): n cores M[k] of shape (w_{k-1}, d, d, w_k),
 *               index order (left bond, output bit, input bit, right bond).
 *   qtt_case -- grid, analytic metric terms, curvilinear FD operators and boundary vectors of
 *               one cylinder case, plus the flow state (u, v, p) (Sec. III, App. A, App. E).
 *
 * Ownership
 *   Every qtt_mps / qtt_mpo / qtt_case returned through an out-pointer is owned by the caller
 *   and released with the matching *_free.  Inputs are never modified unless the parameter is
 *   named *_inout.  Device memory comes from the context's pool, which draws large blocks from
 *   the allocator given to qtt_ctx_create (or cudaMalloc when none is given).
 *
 * Gauge
 *   Every MPS produced by the library is right-canonical (cores 2..n right-orthonormal, the
 *   norm in core 1; Sec. II).  Results are compared through reconstructed values, overlaps
 *   and norms, never raw cores.
 *
 * Errors
 *   Every int-returning call returns QTT_OK (0) or a negative QTT_ERR_* code; qtt_last_error()
 *   gives a message for the calling thread.  Argument errors are detected on the host before
 *   anything is enqueued.  Device-side outcomes (CG iterations, residuals, non-finite values)
 *   land in the *_info structs and are valid after qtt_ctx_sync().  No C++ exception crosses
 *   this interface.
 */
#ifndef QTT_H
#define QTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QTT_OK 0
#define QTT_ERR_ARG (-1)          /* invalid argument (shape, size, null pointer, range) */
#define QTT_ERR_ALLOC (-2)        /* device allocation failed */
#define QTT_ERR_CUDA (-3)         /* a CUDA runtime call or kernel launch failed */
#define QTT_ERR_NOT_CONVERGED (-4)/* a solver stopped at its sweep limit above tolerance */
#define QTT_ERR_TIMEOUT (-5)      /* a bounded device wait ran out */
#define QTT_ERR_NONFINITE (-6)    /* a NaN or Inf appeared in a result */
#define QTT_ERR_UNSUPPORTED (-7)  /* size outside what the kernels support (e.g. bond > 128) */

#define QTT_HOST 0                /* pointer is host memory */
#define QTT_DEVICE 1              /* pointer is device memory of the context's device */

#define QTT_ORDER_SEQUENTIAL 0    /* eta bits of i first, then xi bits of j (Sec. III.B.1) */
#define QTT_ORDER_INTERLEAVED 1   /* eta and xi bits alternate, level by level */

typedef struct qtt_ctx qtt_ctx;
typedef struct qtt_mps qtt_mps;
typedef struct qtt_mpo qtt_mpo;
typedef struct qtt_case qtt_case;

/* Device allocator hooks: alloc(bytes, user) returns a device pointer or NULL; free(ptr, user). */
typedef void* (*qtt_alloc_fn)(size_t bytes, void* user);
typedef void (*qtt_free_fn)(void* ptr, void* user);

/* Contraction precision (the precision study of Sec. IV.C's cost breakdown: the contractions
 * are the dominant cost).  QTT_PREC_FP64: every product is FP64 (FP64 pipe, or the exact
 * seven-digit split on the tensor cores).  The reduced modes run every core contraction that
 * reaches the batched GEMM (M, N, K >= 16) as a digit-split bf16 tensor-core product keeping
 * the leading digits of each operand (8-bit balanced digits, rounded to nearest relative to
 * the row's or column's largest entry) with exact integer accumulation: QTT_PREC_FP32 3 digits
 * (24 bits, relative error ~2^-24 of |A||B|), QTT_PREC_TF32 2 digits (16 bits, ~2^-16; finer
 * than TF32's 11), QTT_PREC_BF16 1 digit (8 bits, ~2^-8).  FP64 is kept for the small direct
 * contractions, the QR and eigen decompositions of the rounding (and their refinement
 * products), the local CG solves, and in the step for the divergence and the Poisson solve. */
#define QTT_PREC_FP64 0
#define QTT_PREC_FP32 1
#define QTT_PREC_TF32 2
#define QTT_PREC_BF16 3

/* Rounding of mpo_apply_round (and of the step's four products, qtt_case_params.apply).
 * QTT_APPLY_GRAM: right-to-left TT-SVD through left Gram environments of M x; only (d chi)-sized
 * eigenproblems appear, but the Gram matrices square the singular values, so directions below
 * ~sqrt(eps) sigma_1 of a cut are not resolved (on smooth fields, whose cut spectra reach
 * 1e-10 sigma_1 at chi, the result differs from the TT-SVD by ~1e-8).  QTT_APPLY_SKETCH: the left
 * part of M x is orthogonalised through a random sketch of its right part (bond 2 chi + 32) and
 * one Householder QR per site, and every cut's matrix is then explicit, its eigenpairs refined
 * in factored form: equal to the TT-SVD up to the sketch's range error (which falls with the
 * cut spectra's tail beyond 2 chi + 32: ~1e-13 on smooth fields, large on flat spectra such as
 * random tensor trains, where the Gram rounding is accurate).  Needs d chi <= 256. */
#define QTT_APPLY_GRAM 0
#define QTT_APPLY_SKETCH 1

/* Truncation rule of every rounding (Sec. II: keep the first chi singular values, or those
 * above a threshold): keep k = min(chi_max, structural rank, #{sigma_i > rel_tol sigma_1});
 * rel_tol = 0 keeps the structural count (fixed bond profile min(2^k, 2^(n-k), chi_max)).
 * prec: QTT_PREC_* of the contractions of the call (0: FP64).  apply: QTT_APPLY_* (read by
 * mpo_apply_round with rel_tol = 0; must be 0 or 1 everywhere). */
typedef struct {
  int chi_max;
  double rel_tol;
  int prec;
  int apply;
} qtt_trunc;

typedef struct {
  int max_bond;            /* largest bond of the result */
  double norm;             /* ||result||_2 */
  double discarded_norm;   /* sqrt(sum over cuts of the discarded sigma^2): the TT-SVD error bound
                              (Sec. II, rounding), equal to ||exact - result|| for a canonical
                              sweep.  From Gram eigenvalues (QTT_APPLY_GRAM and the other
                              Gram roundings) it resolves only values above ~1e-8 ||exact||
                              (they square the singular values); the sketched rounding of
                              mpo_apply_round sums Rayleigh quotients formed from explicit cut
                              matrices, resolved down to the FP64 floor.  -1 for
                              mps_hadamard_round, whose result is a variational fit. */
} qtt_round_info;

/* Options of the single-site ALS solver (Sec. II.A.4).  The paper leaves the stop open; the
 * solver evaluates the true relative residual ||A x - b|| / ||b|| after every full sweep (left
 * to right, then right to left) and stops
 *   - when it is <= rel_tol                                   (QTT_SOLVE_CONVERGED),
 *   - when a sweep after the first reduced it by less than the fraction stall
 *                                                             (QTT_SOLVE_STALLED: at a fixed
 *     bond the sweeps approach a stationary point on the rank-chi manifold whose residual the
 *     truncation bounds from below; stall <= 0 disables this test; the first sweep is exempt
 *     because sweeps minimise the energy, and from a poor start the residual may first rise),
 *   - after max_sweeps sweeps                                 (QTT_SOLVE_MAX_SWEEPS).
 * Each local CG solve of a sweep stops when ||r_loc|| <= cg_tol * res * ||b_loc||, res being the
 * true relative residual before the sweep, or after cg_max_iter iterations.
 * The residual is the un-truncated TT A x (+) (-b) evaluated entry by entry on the device
 * (2^n values, n <= 30), so it carries only the rounding of each entry. */
typedef struct {
  int max_sweeps;
  double rel_tol;
  int cg_max_iter;
  double cg_tol;
  double stall;
} qtt_solve_opts;

#define QTT_SOLVE_CONVERGED 0
#define QTT_SOLVE_STALLED 1
#define QTT_SOLVE_MAX_SWEEPS 2
#define QTT_SOLVE_NONFINITE 3     /* the residual became NaN or Inf */
#define QTT_SOLVE_TIMEOUT 4       /* a bounded grid barrier of a local CG solve ran out */

typedef struct {
  int sweeps;              /* full sweeps done */
  int cg_iters;            /* CG iterations spent (all sites, all sweeps) */
  double rel_residual;     /* ||A x - b|| / ||b|| of the returned x */
  int status;              /* QTT_SOLVE_* */
} qtt_solve_info;

/* ------------------------------------------------------------------------------ context */

/* Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t, may be NULL
 * for the legacy default stream).  alloc/free may be NULL (cudaMalloc/cudaFree are used). */
int qtt_ctx_create(qtt_ctx** out, int device, void* cuda_stream, qtt_alloc_fn alloc,
                   qtt_free_fn free_fn, void* user);
void qtt_ctx_destroy(qtt_ctx* ctx);
/* Block the host until all work enqueued on the context's stream has finished. */
int qtt_ctx_sync(qtt_ctx* ctx);
/* Message of the last error on the calling thread ("" if none). */
const char* qtt_last_error(void);
/* cudaProfilerStart (start != 0) or cudaProfilerStop: brackets the launches an external
 * profiler started with profiling off captures. */
int qtt_profiler_range(int start);
/* Number of kernels this context has launched so far (all entry points). */
int64_t qtt_ctx_kernel_launches(qtt_ctx* ctx);
/* Bytes currently held by the device pools of the context and its worker streams (in use,
 * cached, and the scratch arenas of captured step graphs). */
size_t qtt_ctx_pool_bytes(qtt_ctx* ctx);
/* Per-kernel-class timing.  Synchronises the stream, then writes, for classes 0 FP64 GEMM,
 * 1 Householder QR, 2 Jacobi eigensolver, 3 CG update, 4 other, and the phases of
 * fractional_step 5 MPO-MPS products, 6 right-hand-side fits with the momentum solves (they
 * overlap on worker streams), 7 unused, 8 Poisson solve, 9 projection fits, the summed CUDA-event time (ms), the algorithmic flops and the
 * launch count recorded since the previous call (each array of 10, any may be NULL), resets
 * them, and turns event recording on (on != 0) or off.  Events are recorded on the context
 * stream around each launch (or phase) of a timed class. */
int qtt_ctx_profile(qtt_ctx* ctx, int on, double* ms_out, double* flops_out, int64_t* launches_out);
/* The kernel-class times of the last qtt_ctx_profile read-out split by step phase:
 * ms_out[6 * 5] (row i = phase i of the fractional step -- MPO-MPS products, right-hand sides
 * with momentum, unused, Poisson, projection -- row 5 = outside any phase; column k = kernel
 * class k), and launches_out[6] (kernel launches enqueued in each row).  Either may be NULL. */
int qtt_ctx_profile_phases(qtt_ctx* ctx, double* ms_out, int64_t* launches_out);
/* Limit (seconds, > 0) of every bounded device wait of this context: the grid barriers of the
 * cooperative CG solves (default 2 s).  A wait that runs out makes its kernel leave at once;
 * the solve then ends with QTT_SOLVE_TIMEOUT and the call returns QTT_ERR_TIMEOUT, with the
 * context still usable.  Takes effect for work enqueued afterwards (a captured step keeps the
 * limit it was captured with: set it before the first fractional_step or after
 * qtt_case_use_graph).  Tests shorten it to exercise the timeout path without any fault. */
int qtt_ctx_set_wait_limit(qtt_ctx* ctx, double seconds);
/* How ALS local systems are solved (Sec. II.A.4).  Mode 2 runs each local CG solve as one
 * cooperative kernel on the FP64 pipe (one CTA per SM, grid barriers between its stages) where
 * the bonds allow it (bonds <= 128, operator bonds <= 16, d <= 4).  Mode 3 does the same but,
 * on the context's own stream with left bond <= 64 and the tensor-core product mode
 * (qtt_ctx_set_gemm_mode 0), runs both contractions as exact digit-split products on the
 * tensor cores.  Mode 0 (default) takes mode 3 at sites whose bonds multiply to at least 4096
 * and mode 2 elsewhere.  Mode 1 launches one kernel per contraction and per CG update.  All give
 * the same iterates up to rounding order.  Returns QTT_ERR_ARG for another mode. */
int qtt_ctx_set_cg_mode(qtt_ctx* ctx, int mode);

/* ------------------------------------------------------------------------ MPS and MPO */

/* New MPS with n cores of physical size d and bonds[0..n] (bonds[0] = bonds[n] = 1), its
 * cores copied from `cores` (all cores concatenated, each row-major; kind QTT_HOST or
 * QTT_DEVICE).  `cores` may be NULL: the cores are then zero. */
int qtt_mps_create(qtt_ctx* ctx, int n, int d, const int* bonds, const double* cores, int kind,
                   qtt_mps** out);
int qtt_mps_free(qtt_mps* x);
int qtt_mps_n(const qtt_mps* x);
int qtt_mps_d(const qtt_mps* x);
/* Copy the n+1 bonds into bonds_out. */
int qtt_mps_bonds(const qtt_mps* x, int* bonds_out);
/* Total number of stored values (NVPS_TT, Sec. IV). */
int64_t qtt_mps_size(const qtt_mps* x);
/* Copy all cores (concatenated) to `dst` (kind QTT_HOST or QTT_DEVICE); synchronous for host. */
int qtt_mps_get_cores(const qtt_mps* x, double* dst, int kind);
/* Device pointer of the concatenated cores (valid while x lives). */
const double* qtt_mps_device_ptr(const qtt_mps* x);
int qtt_mps_copy(const qtt_mps* x, qtt_mps** out);

int qtt_mpo_create(qtt_ctx* ctx, int n, int d, const int* bonds, const double* cores, int kind,
                   qtt_mpo** out);
int qtt_mpo_free(qtt_mpo* m);
int qtt_mpo_bonds(const qtt_mpo* m, int* bonds_out);
int qtt_mpo_get_cores(const qtt_mpo* m, double* dst, int kind);

/* ------------------------------------------------------------------ TT operations (Sec. II) */

/* TT-SVD of a dense vector of d^n values (Fig. 1), swept right to left, truncated by `tr`.
 * `dense` (kind QTT_HOST or QTT_DEVICE) is indexed with core 1 as the most significant digit
 * (for 2-D fields use qtt_field_to_vector first). */
int qtt_encode(qtt_ctx* ctx, const double* dense, int kind, int n, int d, qtt_trunc tr,
               qtt_mps** out, qtt_round_info* info);
/* Dense reconstruction (d^n values) into `dense` (kind QTT_HOST or QTT_DEVICE).  Tests only;
 * n <= 26. */
int qtt_decode(qtt_ctx* ctx, const qtt_mps* x, double* dense, int kind);
/* Reorder a 2^n_eta x 2^n_xi row-major field into the QTT vector index of `ordering`
 * (Sec. III.B.1) or back (inverse = 1).  Device or host buffers of 2^(n_eta+n_xi) doubles. */
int qtt_field_to_vector(qtt_ctx* ctx, const double* src, double* dst, int kind, int n_eta,
                        int n_xi, int ordering, int inverse);

/* TT-rounding of x (Sec. II.A): exact TT-SVD semantics, right-to-left. */
int qtt_round(qtt_ctx* ctx, const qtt_mps* x, qtt_trunc tr, qtt_mps** out, qtt_round_info* info);
/* z = round(alpha x + beta y): direct sum of the cores (Sec. II.A.1) then TT-rounding. */
int mps_axpby_round(qtt_ctx* ctx, double alpha, const qtt_mps* x, double beta, const qtt_mps* y,
                    qtt_trunc tr, qtt_mps** out, qtt_round_info* info);
/* y = round(M x): core-wise contraction over the physical index (Sec. II.A.2) then
 * TT-rounding without forming the bond chi*w product: by Gram environments or by the sketched
 * orthogonalisation (tr.apply, QTT_APPLY_*).  rel_tol > 0 forms the product and rounds it by
 * QR and SVD where the bonds allow it. */
int mpo_apply_round(qtt_ctx* ctx, const qtt_mpo* M, const qtt_mps* x, qtt_trunc tr,
                    qtt_mps** out, qtt_round_info* info);
/* c ~ a (.) b (Sec. II.A.3) at the bond profile of `tr`, by the variational fit of Table I:
 * start from `init` (right-canonical, may be NULL: a right-to-left zip-up of a (.) b is used),
 * then `sweeps` fit sweeps. */
int mps_hadamard_round(qtt_ctx* ctx, const qtt_mps* a, const qtt_mps* b, qtt_trunc tr,
                       const qtt_mps* init, int sweeps, qtt_mps** out, qtt_round_info* info);
/* <a, b> without any device memory allocation (the paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need an overlap -- code
 * running inside another allocator's callback, loops that cannot afford a cudaMalloc that may
 * synchronise the device, or processes whose device memory is fully reserved by another pool).
 *   n, d       number of cores and physical size (1 <= n <= 64, 1 <= d <= 4)
 *   a_bonds, b_bonds   host arrays of n+1 bonds, each in [1, 128], first and last equal to 1
 *   a_cores, b_cores   device arrays: all cores concatenated, each (r_{k-1}, d, r_k) row-major,
 *                      no padding between cores (caller-owned, read only)
 *   out_dev    device pointer receiving the overlap (one double, caller-owned)
 *   cuda_stream  stream (cudaStream_t) the work is enqueued on; the call returns without
 *                waiting for it
 * Intermediates live in one fixed 768 KiB array of device memory compiled into the library,
 * held by every device that loads the library until the process exits.  Bonds above 128 or
 * d > 4 return QTT_ERR_UNSUPPORTED.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress); make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents: calls that overlap on the GPU (other
 * streams or host threads) race and must be serialised by the caller.  No context is used and
 * nothing is allocated: not by cudaMalloc, not by the context pool, not by any library. */
int mps_dot_noalloc(int n, int d, const int* a_bonds, const double* a_cores, const int* b_bonds,
                    const double* b_cores, double* out_dev, void* cuda_stream);
/* Symmetric eigendecomposition of a small dense matrix (n <= 256), the building block of every
 * Gram-based rounding: FP32 Jacobi sweeps refined to FP64 accuracy.  S (n x n row-major,
 * symmetric), w (n, descending) and V (n x n row-major, eigenvectors as columns) are host
 * buffers owned by the caller; synchronous. */
int qtt_sym_eig(qtt_ctx* ctx, int n, const double* S, double* w, double* V);
/* Householder QR of a small dense matrix, the gauge move of every fit and ALS sweep (the QR
 * of a core's unfolding, Sec. II.A.4): A (m x n) = Q (m x kk) R (kk x n), kk = min(m, n),
 * R upper triangular with R_jj = -sign(alpha_j) ||x_j|| (the LAPACK convention).  trans = 0:
 * A is row-major m x n and Q is returned row-major m x kk; trans = 1: the buffer holds A^T
 * (row-major n x m) and Q^T (kk x m) is returned.  path 0 picks the kernel (cluster QR over up
 * to 16 CTAs for m >= n >= 16, else one CTA), 1 forces one CTA, 2 forces the cluster kernel
 * (QTT_ERR_UNSUPPORTED if the shape does not allow it).  Host buffers; R may be NULL;
 * synchronous. */
int qtt_qr(qtt_ctx* ctx, int m, int n, int trans, const double* A, double* Q, double* R, int path);
/* C = A B for row-major host matrices A (m x k), B (k x n), C (m x n); synchronous.  The product
 * behind every core contraction of the sweeps (Sec. II.A).  path 0 uses the context's mode (see
 * qtt_ctx_set_gemm_mode), 1 forces the FP64 pipe, 2 and 3 force the tensor-core product: every row
 * of A and column of B is split into seven 8-bit digits scaled by a power of two, digit products
 * are summed exactly in FP32 on the bf16 tensor cores and combined in FP64 (Ozaki scheme; error
 * ~2^-53 max_k|A_ik| sum_k|B_kj|) -- with warp-level mma.sync (2) or with tcgen05.mma on
 * TMA-staged tiles and tensor-memory accumulators (3); both give bit-identical results. */
int qtt_dgemm(qtt_ctx* ctx, int m, int n, int k, const double* A, const double* B, double* C, int path);
/* Matrix products of the whole library: mode 0 (default) sends products of at least 2^23
 * multiply-adds to the tensor cores (digit-split FP64, the digit products by tcgen05.mma on
 * TMA-staged tiles), mode 1 keeps every product on the FP64 pipe, modes 2 and 3 are mode 0 with
 * the digit products forced onto warp-level mma.sync (2) or tcgen05 (3); 0, 2 and 3 give
 * bit-identical results.
 * Takes effect for work enqueued afterwards (a captured step keeps its kernels). */
int qtt_ctx_set_gemm_mode(qtt_ctx* ctx, int mode);
/* Self-check of the QR's Householder scalars: the maximum relative errors of its Newton-Raphson
 * reciprocal (err2[0]) and reciprocal square root (err2[1]) against CUDA's correctly rounded
 * 1/x and 1/sqrt(x) over the n positive host values x.  Synchronous. */
int qtt_check_recip(qtt_ctx* ctx, int n, const double* x, double* err2);
/* GEMM autotuner (the contractions that reach the batched GEMM: core products of the
 * environments, the fits and the local solves outside the cooperative CG kernels).  on = 1:
 * every GEMM shape met for the first time (gemm mode, batch, M, N, K, strides, beta != 0) is
 * timed under each candidate engine -- the FP64-pipe kernel at tile sizes 64, 32 and 16, with
 * the cost model's split-K and unsplit, and the digit-split tensor-core product where the
 * shape allows it (gemm mode != 1, M, N, K >= 16) -- on a stream of the tuner's own over
 * scratch operands, and the fastest is kept; this also happens while a step graph is being
 * captured, the captured step then using the picks.  Shapes already in the table use their
 * pick whether tuning is on or off (on = 0); on = -1 clears the table and turns tuning off.
 * Results of a tuned product differ from the cost model's only in rounding order. */
int qtt_ctx_set_autotune(qtt_ctx* ctx, int on);
/* Contraction precision (QTT_PREC_*) of the fractional steps and solves run on this context
 * (the operations taking a qtt_trunc use its prec field instead).  Read when a step graph is
 * captured: set it before a case's first step, or call qtt_case_set_state again after. */
int qtt_ctx_set_precision(qtt_ctx* ctx, int prec);
/* The tuner's table: *count = number of tuned shapes; up to max_rows rows of 9 int64 are
 * written to rows: batch, M, N, K, engine (0 FP64 tiles, 1 digit-split tensor-core product,
 * -1 not tunable), tile, k splits, time of the pick (ns), time of the cost model's choice (ns). */
int qtt_ctx_autotune_table(qtt_ctx* ctx, int max_rows, int64_t* rows, int* count);
/* <a, b> into *out_host (synchronous). */
int mps_dot(qtt_ctx* ctx, const qtt_mps* a, const qtt_mps* b, double* out_host);

/* Solve A x = b for SPD A by single-site ALS (Sec. II.A.4, Sec. III.C) under the stop rule of
 * qtt_solve_opts: x_inout is the warm start and receives the solution (its bond profile is
 * kept).  Blocks the host until the solve has finished.  Returns QTT_OK when the residual met
 * opts->rel_tol, QTT_ERR_NOT_CONVERGED when the solve stalled or ran out of sweeps (x_inout then
 * holds the last iterate), QTT_ERR_TIMEOUT when a grid barrier ran out, QTT_ERR_NONFINITE when
 * the residual became NaN or Inf; info (may be NULL) is filled in every one of these cases.
 * n <= 30 (the residual is evaluated on 2^n entries). */
int poisson_solve(qtt_ctx* ctx, const qtt_mpo* A, const qtt_mps* b, qtt_mps* x_inout,
                  const qtt_solve_opts* opts, qtt_solve_info* info);

/* -------------------------------------------------------- cylinder case (Sec. III, IV) */

typedef struct {
  int n_eta, n_xi;         /* 2^n_eta radial x 2^n_xi angular interior nodes */
  int ordering;            /* QTT_ORDER_* */
  double D;                /* cylinder diameter (1) */
  double R;                /* outer / inner diameter ratio D_outer / D (App. E) */
  double Re, dt;           /* Reynolds number, fixed time step (Sec. III.C) */
  double rot;              /* wall rotation rate: u_G = rot sin(theta), v_G = -rot cos(theta) */
  double u_inf;            /* far-field velocity (u_inf, 0) */
  int chi;                 /* bond cap of u, v, p and of every rounding in the step */
  int fit_sweeps;          /* sweeps of each variational fit in the step */
  qtt_solve_opts mom, poi; /* ALS options of the momentum and Poisson solves */
  int poisson_warm;        /* warm start of the Poisson solve: 0 the previous pressure p^m; 1 the
                              extrapolation 2 p^m - p^(m-1), fitted at the pressure's bonds from
                              p^m with fit_sweeps sweeps (the first step after set_state, which
                              has no p^(m-1), starts from p^m and runs outside the step graph) */
  int apply;               /* QTT_APPLY_* of the step's four MPO-MPS products */
} qtt_case_params;

typedef struct {
  qtt_solve_info u, v, p;  /* the two momentum solves and the Poisson solve of the step */
  int finite;              /* 1 if the new u and v have finite norms */
  double cd, cl;           /* drag and lift coefficients after the step (eq:liftdrag) */
} qtt_step_info;

/* Build grid, analytic metric terms, operators (rounded at 1e-14) and boundary vectors
 * (Sec. III.B.3, App. A, App. E).  Blocks the host (operator ranks are data dependent). */
int qtt_case_create(qtt_ctx* ctx, const qtt_case_params* p, qtt_case** out);
int qtt_case_free(qtt_case* c);
/* Set the flow state (copies; p may be NULL: a zero pressure padded with tiny seeded noise
 * from `p_pad`, which must then have the bond profile of chi). */
int qtt_case_set_state(qtt_case* c, const qtt_mps* u, const qtt_mps* v, const qtt_mps* p);
/* Copies of the current state. */
int qtt_case_get_state(qtt_case* c, qtt_mps** u, qtt_mps** v, qtt_mps** p);
/* Operator access for tests: which = 0 Dx, 1 Dz, 2 Dx^p, 3 Dz^p, 4 H, 5 A_p, 6 P_x, 7 P_z.
 * Returns a copy. */
int qtt_case_get_operator(qtt_case* c, int which, qtt_mpo** out);
/* Boundary vectors for tests: which = 0 bcx_u, 1 bcz_u, 2 bcx_v, 3 bcz_v, 4 |J| bcLap_u,
 * 5 |J| bcLap_v, 6 bc_div (weighted), 7 |J|.  *out = NULL when the vector is identically zero. */
int qtt_case_get_vector(qtt_case* c, int which, qtt_mps** out);
/* Advance nsteps fractional steps (Sec. III.C) and block the host until they have finished.
 * per_step (may be NULL) receives nsteps records.  Forces are evaluated when with_forces != 0
 * and per_step is given.  Returns QTT_ERR_TIMEOUT if a local CG barrier ran out, QTT_ERR_NONFINITE
 * if a residual or a new velocity norm was NaN or Inf, QTT_ERR_NOT_CONVERGED if a solve used all
 * of its sweeps without meeting its tolerance (a stall at the bond's floor is not an error),
 * checked over all steps whether or not per_step is given. */
int fractional_step(qtt_ctx* ctx, qtt_case* c, int nsteps, int with_forces,
                    qtt_step_info* per_step);
/* Advance several independent cases (Sec. III.C each; the rotating-wall cases of Sec. IV.B
 * differ only in their parameters) by nsteps fractional steps each, and block the host until
 * all have finished.  Each case's step is its captured CUDA graph (captured here when missing),
 * replayed on a stream of its own, so that the cases' kernels share the GPU concurrently; every
 * graph owns its scratch memory and split-K counters, and results are bit-identical to stepping
 * each case alone with fractional_step.  cases: ncases distinct cases of ctx, all in graph
 * replay mode (qtt_case_use_graph); they may differ in grid, chi, Re, dt, rotation and solver
 * options.  per_step (may be NULL): ncases * nsteps records, case-major (case i, step s at
 * i * nsteps + s).  status (may be NULL): ncases return codes, each as fractional_step would
 * return it for that case.  Returns the most severe of them (QTT_ERR_TIMEOUT over
 * QTT_ERR_NONFINITE over the others); the argument checks fail with QTT_ERR_ARG before any work. */
int fractional_step_batch(qtt_ctx* ctx, int ncases, qtt_case* const* cases, int nsteps, int with_forces,
                          qtt_step_info* per_step, int* status);
/* -------------------------------------------------------- learned warm start (growth direction)
 * A convolutional network on a coarse (eta, xi) grid that predicts the next step's pressure
 * change from the fields a step starts from; its prediction, prolonged to the fine grid and
 * compressed to a low-rank MPS, warm-starts the Poisson solve in place of the previous
 * pressure (which stays the fallback).  Stands in for the preconditioner of the Poisson sweeps
 * that the paper leaves unspecified (Sec. IV.C, App. G); the converged residual is required
 * either way, so the step's answer does not depend on it.
 * Network: `depth` 3 x 3 convolutions c_in -> width -> ... -> width -> 1 with bias and ReLU after
 * every layer but the last; zero padding in eta (first axis), periodic in xi (second axis);
 * NCHW FP32 tensors.  Parameters: one FP32 vector, layer by layer, weights (c_out, c_in, 3, 3)
 * row-major then bias (c_out); the caller draws the initial values.  Training: mean squared
 * error, Adam (beta1 0.9, beta2 0.999, eps 1e-8).  Inputs are mapped (x - shift_c) scale_c per
 * channel and the network predicts y / out_scale (qtt_nn_set_scaling; identity by default). */
typedef struct qtt_nn qtt_nn;
/* Number of parameters of the network (-1 for invalid sizes). */
int64_t qtt_nn_param_count(int c_in, int width, int depth);
/* 1 <= c_in <= 64, 1 <= width <= 256, 1 <= depth <= 16; params: host, qtt_nn_param_count values. */
int qtt_nn_create(qtt_ctx* ctx, int c_in, int width, int depth, const float* params, qtt_nn** out);
int qtt_nn_free(qtt_nn* nn);
/* Current parameters / gradient of the last training step (host, param_count values). */
int qtt_nn_get_params(const qtt_nn* nn, float* dst);
int qtt_nn_get_grad(const qtt_nn* nn, float* dst);
/* Per-channel input affine (c_in values each, host) and output scale (finite, non-zero). */
int qtt_nn_set_scaling(qtt_nn* nn, const float* in_shift, const float* in_scale, float out_scale);
/* y (B x H x W) = network(x (B x c_in x H x W)) x out_scale; kinds QTT_HOST or QTT_DEVICE;
 * synchronous. */
int qtt_nn_predict(qtt_nn* nn, int B, int H, int W, const float* x, int xkind, float* y, int ykind);
/* One Adam step of learning rate lr on the mean squared error between network(x) and
 * y / out_scale (x: B x c_in x H x W, y: B x H x W, both of pointer kind `kind`); *loss (may be
 * NULL) receives the loss before the step.  QTT_ERR_NONFINITE if the loss is not finite. */
int qtt_nn_train_step(qtt_nn* nn, int B, int H, int W, const float* x, const float* y, int kind, float lr,
                      float* loss);
/* Grid transfers between a fine (Hc 2^levels) x (Wc 2^levels) FP64 field and its coarse
 * Hc x Wc FP32 image (both row-major, eta the first axis): restriction averages each
 * 2^levels x 2^levels block; prolongation applies `levels` cell-centred bilinear doublings
 * (fine cell 2I takes 3/4 of coarse cell I and 1/4 of I - 1, cell 2I + 1 3/4 of I and 1/4 of
 * I + 1, clamped at the ends of eta, periodic in xi).  0 <= levels <= 12; synchronous. */
int qtt_grid_restrict(qtt_ctx* ctx, int Hc, int Wc, int levels, const double* fine, int fkind, float* coarse,
                      int ckind);
int qtt_grid_prolong(qtt_ctx* ctx, int Hc, int Wc, int levels, const float* coarse, int ckind, double* fine,
                     int fkind);
/* Mean and root mean square of n FP32 values (fixed summation order); synchronous. */
int qtt_field_moments(qtt_ctx* ctx, int64_t n, const float* x, int kind, double* mean, double* rms);

/* Replay mode of fractional_step.  enable != 0 (the default): the first call captures one
 * step as a CUDA graph on an internal stream (ordered after the context stream by events)
 * and every step replays it; the graph is dropped when the state is set again.  enable = 0:
 * every step is launched kernel by kernel (same kernels, same results). */
int qtt_case_use_graph(qtt_case* c, int enable);
/* Wall time (ms) of the phases of the last step, in order: MPO-MPS products, right-hand
 * sides with the momentum solves, Poisson solve, projection.  Synchronous. */
int qtt_case_phase_ms(qtt_case* c, double* ms4);
/* Drag and lift of the current state (App. F; synchronous). */
int qtt_case_forces(qtt_ctx* ctx, qtt_case* c, double* cd, double* cl);
/* Strouhal number from upward zero crossings of C_L(t) (eq:st); host-only arithmetic on a
 * scalar time series. */
int qtt_strouhal(const double* t, const double* cl, int n, double* st);

#ifdef __cplusplus
}
#endif
#endif
