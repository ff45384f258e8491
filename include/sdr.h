/*
 * sdr.h -- C ABI of the GB300 GMRES-SDR solver.
 *
 * GMRES-SDR (GMRES with sketching and deflated restarting; Burke, Guettel,
 * Soodhalter) solves A x = b and sequences of slowly changing systems
 * A^(i) x^(i) = b^(i) (Introduction, eq. (sequence_of_linear_systems)).  Each
 * restart cycle is Algorithm 1: a truncated Arnoldi process, a sparse
 * subspace embedding S applied to the new basis vectors, a sketched least
 * squares problem solved through an updated QR factorisation, residual
 * control with a safety factor (Section 3.4), and a sketched harmonic-Ritz
 * update of the recycle space U (Section 3.5).  Section 3.6 defines how U, SU
 * and SAU are carried from one system to the next.
 *
 * Conventions for every entry point:
 *  - Device pointers are CUDA device addresses on the handle's device; host
 *    pointers are ordinary process memory.  Each argument below says which.
 *  - The caller owns A, b and x.  The handle owns all workspace (the Krylov
 *    basis V, SV, SAV, U, SU, SAU, the QR factors and the small dense
 *    buffers); it is allocated once in sdr_create for n <= n_max.
 *  - All work is issued on the stream given to sdr_create.  sdr_solve and
 *    sdr_recycle return after that stream has finished the call's work.
 *  - Nothing throws across the ABI.  Every call returns an sdr_status; after
 *    any status other than SDR_ERR_CUDA the handle stays usable.
 *  - Matrices are square CSR with int32 row pointers and column indices,
 *    0-based; a row's columns need not be sorted.  Values are float64.
 *  - Vectors are contiguous float64 arrays of length n.
 *  - Multi-column arrays are column-major with leading dimension n (tall
 *    N x k arrays) or s (sketches, s x k).
 */
#ifndef SDR_H
#define SDR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SDR_ABI_VERSION 3

typedef struct sdr_handle sdr_handle; /* opaque */

typedef enum {
  SDR_OK = 0,
  SDR_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
  SDR_ERR_CUDA = 2,          /* a CUDA call failed; the handle must be destroyed */
  SDR_ERR_OOM = 3,           /* device allocation failed in sdr_create */
  SDR_ERR_NOT_CONVERGED = 4, /* max_cycles reached; x holds the last iterate */
  SDR_ERR_BREAKDOWN = 5,     /* H(j+1,j) = 0 or a non-finite value with res >= tol */
  SDR_ERR_RANK = 6,          /* sdr_recycle / sdr_recycle_import: the installed SAU is
                                numerically rank-deficient; the space was dropped */
  SDR_ERR_NOT_IMPLEMENTED = 7
} sdr_status;

/* Solver parameters (Algorithm 1 inputs m, t, k, S and safety; the stopping
 * rule of Section 3.4).
 *   m          Krylov columns per cycle (V has m+1 columns), 1 <= m <= 128.
 *   k          recycle dimension; up to k+1 columns are kept when the k-th and
 *              (k+1)-th harmonic Ritz values form a conjugate pair. 0 <= k <= 31.
 *   t          truncation window of the Arnoldi process, 1 <= t <= 4.
 *   s, zeta    sketch rows and nonzeros per sketch column; needs
 *              m + k + 2 <= s <= 768 and 1 <= zeta <= min(s, 32).
 *   seed       seed of the hash that defines S (fixed for the handle's life,
 *              so that SU and SAU remain valid from one system to the next).
 *   rel_tol    stop when ||b - A x|| < rel_tol * ||b||.
 *   safety0    initial safety factor (>= 1; the paper's default is 1.4).
 *   max_cycles restart cycles per sdr_solve call (>= 1).
 *   persist_safety 0: safety restarts from safety0 every cycle;
 *                  1: it carries over within one sdr_solve call.
 *   precision  SDR_PREC_F64: everything in float64.
 *              SDR_PREC_F32_REFINED: the basis V, U, the SpMV, the window
 *              dots, the Arnoldi update and the sketched vectors are float32
 *              (float32 accumulation; the sketch sums stay exact), the small
 *              sketched QR / least squares and the harmonic-Ritz eigenproblem
 *              stay float64, and sdr_solve wraps the float32 solver in a
 *              float64 iterative refinement: r = b - A x in float64, solve
 *              A d = r in float32 to inner_rel_tol, x += d, until
 *              ||b - A x|| < rel_tol ||b|| (max_cycles bounds the inner
 *              cycles of each refinement step; at most 40 steps).
 *   inner_rel_tol  refined form: relative tolerance of each inner solve
 *              (0 selects 1e-4).
 *   stale_check  0: off.  1: for a handle whose SAU may be stale (the inexact
 *              variant of Section 3.6, sdr_recycle mode 1): when a restart
 *              cycle of sdr_solve ends unconverged with its last true
 *              residual res > 4 * sres (its sketched residual), SAU of the
 *              new recycle space is recomputed as S A U (k products with A)
 *              before the next cycle.  With an exact SAU the true residual
 *              lies in the embedded subspace, so res <= sres / (1 - eps) <=
 *              4 sres for any embedding with eps <= 3/4 (Section 3, Eq.
 *              (sketch)); a larger ratio can only come from a stale SAU.
 *              Counted in sdr_stats.sau_refreshes.  Ignored by
 *              sdr_solve_batch and by SDR_PREC_F32_REFINED handles.
 *   sketch_kind  0: the sparse-sign embedding (s rows, zeta nonzeros +-1/sqrt(zeta)
 *              per column, rows and signs from a counter-based hash of seed).
 *              1: the subsampled randomised DCT of the paper's experiments
 *              (Section 6): S = sqrt(n/s) P F E, E a diagonal of random signs,
 *              F the orthonormal DCT-II, P a selection of s distinct
 *              frequencies.  Its draws (E and P) are inputs, set by
 *              sdr_set_sketch_draws for one system size n before any solve
 *              (zeta and seed are then unused).  Applied by direct summation
 *              with a cosine table: s n multiply-adds per sketch in FP64,
 *              against the sparse sign's zeta n additions; n_max < 2^29.
 *   test_flags bit 0: take the truncated-SVD path of the harmonic-Ritz step
 *              even when the full-rank certificate holds (for tests);
 *              bit 1: launch every kernel directly instead of replaying each
 *              restart cycle from a captured CUDA graph.  With graphs (the
 *              default) sdr_solve first copies A, b and x into buffers the
 *              handle owns, so that one graph per cycle state serves every
 *              later solve of the same size;
 *              bit 2: compute the recycle product U_new = [U V] P of a float64
 *              handle on the 32-bit integer pipe instead of the tensor cores
 *              (both are exact: the results are bit-identical).
 */
#define SDR_PREC_F64 0
#define SDR_PREC_F32_REFINED 1
typedef struct {
  int32_t m, k, t, s, zeta;
  uint64_t seed;
  double rel_tol;
  double safety0;
  int32_t max_cycles;
  int32_t persist_safety;
  int32_t precision;
  int32_t test_flags;
  double inner_rel_tol;
  int32_t stale_check;
  int32_t sketch_kind;
  int32_t reserved[2]; /* must be zero */
} sdr_params;

/* Square CSR matrix; all pointers are device pointers owned by the caller. */
typedef struct {
  int64_t n, nnz;
  const int32_t* rowptr; /* n + 1 entries */
  const int32_t* col;    /* nnz entries */
  const double* val;     /* nnz entries */
  const float* val32;    /* nnz entries, float32 copy of val: needed by sdr_solve and
                            sdr_recycle of an SDR_PREC_F32_REFINED handle, else NULL */
} sdr_csr;

/* Statistics of the last sdr_solve (host struct filled by the library). */
typedef struct {
  int32_t cycles;          /* restart cycles run */
  int32_t converged;       /* 1 if ||b - A x|| < tol at return */
  int32_t matvecs;         /* products with A, including true-residual checks */
  int32_t sketches;        /* applications of S to a length-n vector */
  int32_t true_res_evals;  /* true-residual checks (Algorithm 1, residual control) */
  int32_t arnoldi_steps;   /* truncated Arnoldi steps over all cycles */
  int32_t recycle_dim;     /* columns of U after the solve */
  int32_t full_svd_cycles; /* cycles that needed the truncated-SVD path */
  int32_t kernel_launches; /* kernels of this library launched by the call */
  int32_t refinements;     /* SDR_PREC_F32_REFINED: float64 refinement steps (0 otherwise) */
  int32_t sau_refreshes;   /* stale_check: SAU recomputations the rule triggered */
  int32_t refresh_matvecs; /* products with A those recomputations took (in matvecs) */
  double final_res;        /* last true residual norm */
  double tol;              /* rel_tol * ||b|| */
  double final_rel_res;    /* final_res / ||b|| */
  double bnorm;
} sdr_stats;

/* Per-cycle log entry (host struct). */
typedef struct {
  int32_t steps;       /* Krylov columns built in the cycle (j_f) */
  int32_t checks;      /* true-residual evaluations in the cycle */
  int32_t converged;
  int32_t ell;         /* numerical rank of SAW at the cycle's end */
  int32_t kprime;      /* recycle columns produced */
  int32_t kh;          /* recycle columns used by the cycle */
  int32_t flags;       /* bit 0: truncated-SVD path taken; bit 1: breakdown;
                          bit 2: rank lost (SAW's QR, l = 0, the eigenvalue
                          iteration's limit, or bit 3); bit 3: a selected
                          eigenvector was dependent on the ones before it
                          (its Gram-Schmidt remainder below 1e-12 of its norm) */
  int32_t svd_sweeps;  /* Jacobi sweeps of the truncated-SVD path (0 when not taken) */
  double res;          /* true residual at the cycle's last check */
  double sres;         /* sketched residual at the cycle's last step */
  double safety;       /* safety factor after the cycle */
} sdr_cycle_log;

/* Create a handle: fix Algorithm 1's inputs (m, t, k, safety) and the
 * subspace embedding S of Section 3 (Eq. (sketch); here the sparse-sign
 * operator defined by s, zeta and seed, drawn once so that SU and SAU stay
 * valid across a sequence, Section 3.6), and allocate the cycle's storage:
 * the basis V (n_max x (m+1)), SV, SAV (s x m), the recycle triple U, SU,
 * SAU (Section 3.5) and the QR factors of SAW.
 *   p: host pointer to parameters.  n_max: largest n any later call uses.
 *   stream: a cudaStream_t (NULL = legacy default stream).
 *   out: host pointer receiving the handle.
 * Allocates all device workspace on the current device and builds the
 * sketch's per-tile index tables.  Synchronous.
 * Errors: INVALID_ARG (parameter out of range), OOM, CUDA. */
sdr_status sdr_create(const sdr_params* p, int64_t n_max, void* stream, sdr_handle** out);

/* Solve A x = b by restarted GMRES-SDR (Algorithm 1 repeated on the current
 * residual), starting from the iterate in x and from the handle's current
 * recycle space U, SU, SAU (empty for a fresh handle).
 *   A: host pointer to a CSR descriptor of device arrays, A->n <= n_max.
 *   b: device pointer, n entries.   x: device pointer, n entries, in: x0,
 *   out: solution.   stats: host pointer or NULL.
 * On return U, SU, SAU describe the recycle space for the next system.
 * Returns OK, NOT_CONVERGED (x holds the last iterate), BREAKDOWN (a cycle
 * ended with H(j+1, j) = 0 and res >= tol, or a non-finite value appeared;
 * a NaN or an Inf in A, b or x0 is caught before any cycle, x unchanged),
 * INVALID_ARG or CUDA. */
sdr_status sdr_solve(sdr_handle* h, const sdr_csr* A, const double* b, double* x, sdr_stats* stats);

/* Solve count independent systems, one per handle (each handle with its own
 * stream and recycle space; a handle appears at most once): A_i x_i = b_i
 * exactly as sdr_solve would, but driven in lockstep.  In each round the
 * library issues one restart cycle of every unfinished system (on the
 * handles' streams, so the systems' kernels run concurrently) and then reads
 * every issued cycle's outcome; a handle's cycle is replayed from a CUDA graph
 * captured on first use.
 *   hs: host array of count handles (SDR_PREC_F64).  As: host array of count
 *   CSR descriptors.  bs, xs: host arrays of count device pointers.
 *   stats: host array of count entries, or NULL.
 * Returns OK when every system converged, else the first non-OK status of
 * the systems in order (INVALID_ARG / NOT_IMPLEMENTED before any work). */
sdr_status sdr_solve_batch(int32_t count, sdr_handle* const* hs, const sdr_csr* As, const double* const* bs,
                           double* const* xs, sdr_stats* stats);

/* sdr_recycle for count handles (mode as in sdr_recycle), the SAU
 * recomputations of all handles issued before any is waited for.
 *   hs: host array of count handles.  As: host array of count CSR
 *   descriptors (read only in mode 0; may be NULL otherwise).
 * Returns when every handle's stream is idle.  Errors: INVALID_ARG (count
 * < 0, a NULL handle, mode outside 0..2, or in mode 0 a descriptor that
 * fails the sdr_solve checks for a handle with a recycle space), CUDA. */
sdr_status sdr_recycle_batch(int32_t count, sdr_handle* const* hs, const sdr_csr* As, int32_t mode);

/* Prepare the recycle space for the next system in a sequence (Section 3.6).
 *   mode 0 (exact): keep U and SU, recompute SAU = S A_next U with k products
 *          with A_next and k sketches (A_next: host pointer to a CSR
 *          descriptor of device arrays).
 *   mode 1 (inexact): keep SAU as it is (A_next unused, may be NULL).
 *   mode 2: drop the recycle space.
 * A system sequence with a fixed matrix needs no call at all.
 * Synchronous: returns when the new SAU is in place.  Errors: INVALID_ARG
 * (h NULL, mode outside 0..2, or in mode 0 with a non-empty recycle space an
 * A_next that is NULL, has a NULL array, n outside 1..n_max or nnz outside
 * 0..2^31 - 1), RANK (mode 0: the recomputed SAU is numerically
 * rank-deficient, |R_pp| <= s eps max_q ||SAU(:, q)|| in its QR; the recycle
 * space is dropped and the handle stays usable), CUDA. */
sdr_status sdr_recycle(sdr_handle* h, const sdr_csr* A_next, int32_t mode);

/* Release all device memory of the handle and the handle itself (h must not
 * be used afterwards).  h may be NULL. */
sdr_status sdr_destroy(sdr_handle* h);

/* ---- inspection and state transfer ---------------------------------- */

/* y = S x: apply the handle's subspace embedding S (Section 3, Eq. (sketch)) to
 * a length-n vector.
 *   x: device pointer (n entries, 1 <= n <= n_max; for a DCT handle n must be
 *   the size its draws were set for).  y: device pointer (s entries),
 *   overwritten.
 * Synchronous.  Errors: INVALID_ARG (NULL pointer or n out of range), CUDA. */
sdr_status sdr_sketch(sdr_handle* h, const double* x, int64_t n, double* y);

/* y = S x without allocating any device memory.  S is the same hash-defined
 * sparse-sign embedding a handle with these s, zeta and seed applies (for a
 * handle whose n_max equals n the results agree bit for bit).  The paper has
 * no counterpart: this entry point exists for callers that must not let a
 * library allocate device memory, such as code running while another
 * component owns the device's memory (a framework's pool, or a budget fixed at
 * start-up) and latency-critical paths that cannot afford a cudaMalloc, which
 * may synchronise the device.
 *   x: device pointer, n entries (1 <= n <= 2^31 - 1).
 *   y: device pointer, s entries (1 <= s <= 512), overwritten.
 *   zeta: nonzeros per column, 1 <= zeta <= min(s, 32).
 *   stream: a cudaStream_t (NULL = legacy default stream).  The call enqueues
 *   its kernels on it and returns; y is ready when the stream gets there.
 * Non-finite input: if x holds a NaN or an Inf, every y[i] is set to NaN
 * (the call still returns SDR_OK; the caller tests y).  x == 0 gives y == 0.
 * Scratch: one file-scope device array of 8,256 bytes, which every GPU that
 * loads this library keeps until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture.  The kept address is not refreshed after
 * cudaDeviceReset: do not call this entry point again on a device that was
 * reset.  Every call
 * shares the array and clears it before use, so calls whose work overlaps on
 * the GPU (other streams, or other host threads, before an earlier call's
 * kernels have finished) race and corrupt each other's results.
 * Errors: INVALID_ARG for sizes or pointers outside these limits (nothing is
 * launched), CUDA if the address lookup or a launch fails. */
sdr_status sdr_sketch_noalloc(const double* x, int64_t n, int32_t s, int32_t zeta, uint64_t seed, double* y,
                              void* stream);

/* ---- Differentiable solve (the adjoint form) ----------------------------
 * For x = A^{-1} b and a scalar loss L(x), the adjoint method gives
 * dL/db = lambda with A^T lambda = dL/dx, and dL/dA_ij = -lambda_i x_j on the
 * stored entries.  The paper has no counterpart: these calls serve the
 * transposed solves that a gradient needs, each carried out by sdr_solve on a
 * second handle whose recycle space (Section 3.6) persists from call to call.
 *
 * Transposed sparsity pattern of A (A: host pointer to a CSR descriptor of
 * device arrays).  rowptrT (n+1), colT (nnz), perm (nnz): device outputs;
 * the values of A^T are val[perm[q]], q = 0..nnz-1, and each row of colT is
 * sorted by column (deterministic).  work: device scratch of 2n int32.
 * Column indices must lie in [0, n).  Asynchronous on stream.
 * Errors: INVALID_ARG (null pointer, n or nnz out of int32 range), CUDA. */
sdr_status sdr_csr_transpose(const sdr_csr* A, int32_t* rowptrT, int32_t* colT, int32_t* perm, int32_t* work,
                             void* stream);

/* out[q] = val[perm[q]] for q < nnz (device pointers; perm from
 * sdr_csr_transpose).  Asynchronous on stream.  Errors: INVALID_ARG, CUDA. */
sdr_status sdr_gather_values(const double* val, const int32_t* perm, int64_t nnz, double* out, void* stream);

/* grad[p] = -lambda[i] * x[col[p]] for every stored entry p of row i of A
 * (host CSR descriptor of device arrays; lambda, x: device, n entries;
 * grad: device, nnz entries, written).  Asynchronous on stream.
 * Errors: INVALID_ARG, CUDA. */
sdr_status sdr_value_gradient(const sdr_csr* A, const double* lambda, const double* x, double* grad,
                              void* stream);

/* Sketched residual norms of every Arnoldi step of the last sdr_solve, in
 * order, and the per-cycle log.  sres: host pointer with room for cap_steps
 * doubles (may be NULL).  log: host pointer with room for cap_cycles entries
 * (may be NULL).  n_steps / n_cycles: host pointers receiving the counts
 * (may be NULL).  The counts are those kept, not min(count, cap).  Reads host
 * memory only.  Errors: INVALID_ARG (h NULL). */
sdr_status sdr_get_history(sdr_handle* h, double* sres, int32_t cap_steps, int32_t* n_steps,
                           sdr_cycle_log* log, int32_t cap_cycles, int32_t* n_cycles);

/* Set the random draws of a DCT sketch (sketch_kind 1): the subsampled
 * randomised DCT S = sqrt(n/s) P F E of Section 6 for systems of size n.
 *   n: system size (1 <= n <= n_max); every later call must use this n.
 *   signs: host pointer, n entries, each +1 or -1 (the diagonal E).
 *   rows: host pointer, s entries, strictly increasing in [0, n) (the
 *   frequencies P selects).
 * Copies the draws to the device, builds the cosine table, drops the recycle
 * space (sketched with another operator) and returns when done.
 * Errors: INVALID_ARG (not a DCT handle, n out of range, a sign other than
 * +-1, rows not strictly increasing in [0, n)), CUDA. */
sdr_status sdr_set_sketch_draws(sdr_handle* h, int64_t n, const int8_t* signs, const int32_t* rows);

/* Givens sines and cosines of every Arnoldi step of the last sdr_solve, in
 * the order of sdr_get_history (Section 4.5, Theorem on Givens sines and
 * sketched GMRES angles; Section 5, the augmented cycle through the whitened
 * basis).  Step j's rotation has |s_j| = sin of the angle between S r_{j-1}
 * and S A [U V_j], so that ||S r_j|| = |s_j| ||S r_{j-1}||, and
 * |c_j| = sqrt(1 - s_j^2); both are read off the QR of SAW that each step
 * updates (no extra work on the device).  The Corollary that follows the
 * Theorem turns them into a progressive bound on the true residual.
 *   sines, cosines: host pointers with room for cap doubles (either may be
 *   NULL).  n_steps: host pointer receiving the number of steps (may be NULL).
 * Reads host memory only.  Errors: INVALID_ARG (h NULL, cap < 0). */
sdr_status sdr_get_givens(sdr_handle* h, double* sines, double* cosines, int32_t cap, int32_t* n_steps);

/* Current number of recycle columns (0 for a fresh handle; at most k + 1).
 * Errors: INVALID_ARG (h or kdim NULL). */
sdr_status sdr_recycle_dim(sdr_handle* h, int32_t* kdim);

/* Copy the recycle state out: U (device, n x kdim, ld n), SU and SAU
 * (device, s x kdim each, ld s).  Any pointer may be NULL to skip it; n is
 * the length of the system the space belongs to.  Synchronous; nothing is
 * copied when kdim = 0.  Errors: INVALID_ARG (h NULL, n outside 1..n_max),
 * NOT_IMPLEMENTED (a float32 handle), CUDA. */
sdr_status sdr_recycle_export(sdr_handle* h, int64_t n, double* U, double* SU, double* SAU);

/* Replace the recycle state: U (device, n x kdim, ld n); SU and SAU (device,
 * s x kdim) or NULL, in which case the missing sketches are computed from U
 * with A (host pointer to a CSR descriptor; needed only when SAU is NULL).
 * kdim <= k + 1; kdim = 0 empties the space.  U's columns are taken as they
 * are (the next cycle assumes nothing of their scaling).  Synchronous.
 * Errors: INVALID_ARG (h NULL, n outside 1..n_max, kdim out of range, U NULL
 * with kdim > 0, or A invalid when it is needed), RANK (SAU, given or
 * computed, is numerically rank-deficient as in sdr_recycle: Algorithm 1's
 * least squares needs SAW = [SAU, SAV] of full column rank; the space is
 * dropped), NOT_IMPLEMENTED (a float32 handle), CUDA. */
sdr_status sdr_recycle_import(sdr_handle* h, const sdr_csr* A, int64_t n, int32_t kdim,
                              const double* U, const double* SU, const double* SAU);

/* ---- timing of the library's own kernels ---------------------------- */

/* Kernel classes of sdr_kernel_time entries (index = class). */
enum {
  SDR_K_SOLVE_INIT = 0,   /* ||b||, max|b|, ||A||_inf at the start of a solve */
  SDR_K_RESIDUAL0,        /* initial residual b - A x0 with its sketch */
  SDR_K_CYCLE_INIT,       /* S r0, beta (first launch), QR of SAU (second launch): Algorithm 1 set-up */
  SDR_K_SPMV_DOTS,        /* w = A v_j with truncation-window dots */
  SDR_K_UPDATE_SKETCH,    /* truncated-Arnoldi update (the next SpMV sketches its output) */
  SDR_K_STEP_DENSE,       /* QR update of SAW, sketched residual, control */
  SDR_K_CHECK_GEMV,       /* x_trial = x + [U V] y (launched every step, works on checks) */
  SDR_K_CHECK_RESIDUAL,   /* true residual of x_trial (launched every step, works on checks) */
  SDR_K_CYCLE_END,        /* harmonic-Ritz recycling: C = Q^T S[U V] (first of eight parts) */
  SDR_K_RECYCLE_GEMM,     /* U_new = [U V] P */
  SDR_K_RECYCLE_SAU,      /* SAU = S A U for the exact variant (per column) */
  SDR_K_SKETCH,           /* stand-alone sketches (sdr_sketch, SU) */
  SDR_K_CE_RINV,          /* cycle end: R^{-1} */
  SDR_K_CE_M,             /* cycle end: full-rank certificate and M = R^{-1} C */
  SDR_K_CE_SVD,           /* cycle end: truncated SVD (only when not certified) */
  SDR_K_CE_EIG,           /* cycle end: FP32 eigenvalue candidates (Hessenberg + Francis QR) */
  SDR_K_CE_INVIT,         /* cycle end: FP64 inverse iteration per candidate */
  SDR_K_CE_SELECT,        /* cycle end: selection of the k largest |mu| */
  SDR_K_CE_FINISH,        /* cycle end: orthonormal basis Z and P */
  SDR_K_CE_SKETCHES,      /* cycle end: SU, SAU of the new recycle space */
  SDR_K_REFINE,           /* refined form: float32 right-hand side and the float64 update x += d */
  SDR_K_COUNT
};

typedef struct {
  int32_t launches;  /* launches of the class since profiling was enabled */
  int32_t pad;
  double total_ms;   /* summed CUDA-event time between each launch's start and end */
} sdr_kernel_time;

/* enable != 0: bracket every kernel launch with CUDA events on the stream it
 * is launched on and accumulate per-class times (resets the totals); 0: stop.
 * Events serialise nothing but add a record per launch; a profiled call is
 * slower than an unprofiled one.  Errors: INVALID_ARG (h NULL). */
sdr_status sdr_profile(sdr_handle* h, int32_t enable);

/* Copy min(cap, SDR_K_COUNT) per-class totals into out (host pointer, may be
 * NULL); *n receives SDR_K_COUNT.  Errors: INVALID_ARG (h NULL). */
sdr_status sdr_profile_get(sdr_handle* h, sdr_kernel_time* out, int32_t cap, int32_t* n);

/* One launch of a traced call.  start_us and end_us are the CUDA events
 * recorded just before and just after the launch on its stream, in
 * microseconds after the first launch traced since sdr_trace; the span thus
 * includes the time the launch waited for its stream and for free SMs. */
typedef struct {
  int32_t cls;      /* sdr_kernel_class */
  int32_t stream;   /* 0: the handle's main stream, 1: its control stream, 2: another stream */
  double start_us;
  double end_us;
} sdr_trace_entry;

/* cap > 0: while profiling is enabled (sdr_profile), keep a trace entry for
 * each of the next cap launches (clears the earlier trace and takes a new
 * time origin); cap = 0: stop tracing.  Entries are taken when a call
 * collects its event pairs, i.e. before the call returns.
 * Errors: INVALID_ARG (h NULL, cap < 0), CUDA (event creation). */
sdr_status sdr_trace(sdr_handle* h, int32_t cap);

/* Copy min(cap, *n) trace entries into out (host pointer); *n receives the
 * number kept.  Errors: INVALID_ARG (h NULL, cap < 0, out NULL with cap > 0). */
sdr_status sdr_trace_get(sdr_handle* h, sdr_trace_entry* out, int32_t cap, int32_t* n);

/* Human-readable text of a status (static storage). */
const char* sdr_status_string(sdr_status st);

/* SDR_ABI_VERSION of the library. */
int32_t sdr_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SDR_H */
