/*
 * ils.h -- C ABI of a GB300 (sm_103a) solver for the indefinite least squares
 * (ILS) problem
 *
 *     min_x (b - A x)^T J (b - A x),   J = diag(I_p, -I_q),  p + q = m,
 *
 * (Zhang & Li, "Splitting-based randomized iterative methods for solving
 * indefinite least squares problem", Sec. 1, eq. (1.1)).  A = [A_1; A_2] with
 * A_1 p x n and A_2 q x n (Sec. 1.4, eq. (1.4)); the solution is unique and
 * equals (A^T J A)^{-1} A^T J b exactly when A^T J A is symmetric positive
 * definite (eq. (1.2)-(1.3)).  Three methods are provided: SP (Alg. 1),
 * SP-RK-RGS (Alg. 2) and SP-SCD (Alg. 5).
 *
 * Conventions for every entry point:
 *   - Matrices are column-major.  "lda" is the distance in elements between
 *     consecutive columns and must be >= the number of rows.
 *   - Pointers are DEVICE pointers unless the comment says "host".
 *   - Work is ordered on the caller's stream (NULL = the legacy default
 *     stream).  Calls that return an ils_info synchronize that stream before
 *     returning; the others only enqueue work.
 *   - Errors are returned as ils_status; nothing aborts, traps or prints.  A
 *     CUDA error inside a call is returned as ILS_ERR_CUDA.
 *   - A handle is not thread-safe; calls on one handle must not overlap.
 */
#ifndef ILS_H
#define ILS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream. */
typedef struct CUstream_st* ils_stream_t;

typedef struct ils_handle_s* ils_handle;

typedef enum {
  ILS_OK = 0,
  ILS_ERR_INVALID_ARG = 1,    /* bad size, stride, pointer or option */
  ILS_ERR_NOT_SPD = 2,        /* condition (1.3) fails: A_1^T A_1 or H = A^T J A failed its pivot test
                                 (explicit route), or the estimated rho(Abar1^{-1} Abar2) >= 1
                                 (matrix-free route with options.estimate) */
  ILS_ERR_NO_CONVERGENCE = 3, /* max_outer reached; x holds the last iterate */
  ILS_ERR_NONFINITE = 4,      /* a NaN/Inf appeared in the input or the iteration */
  ILS_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out */
  ILS_ERR_CUDA = 6,           /* a CUDA runtime call failed */
  ILS_ERR_OOM = 7             /* device allocation failed */
} ils_status;

typedef enum {
  ILS_SP = 0,        /* Alg. 1: x_{k+1} = B x_k + c, B = (A_1^T A_1)^{-1} A_2^T A_2 */
  ILS_SP_RK_RGS = 1, /* Alg. 2: inner RK step on A_1^T w = bhat, RGS step on A_1 z = w */
  ILS_SP_SCD = 2     /* Alg. 5: inner sampling coordinate descent on (A_1^T A_1) beta = bhat */
} ils_method;

typedef enum {
  ILS_FP64 = 0,        /* every product in FP64 (the paper's arithmetic) */
  ILS_FP32_REFINE = 1, /* SP method: FP64-accurate Grams; the correction sweeps use
                          P = Abar1^{-1} and B = P Abar2 in FP32 with FP32 accumulation.
                          P comes from the FP32 Gauss-Jordan inverse of Abar1 (single dense
                          handles; beyond one cooperative wave of its tiles, from an FP32
                          Cholesky factor), or from the FP64 Cholesky factor when
                          options.factor64 != 0, on the matrix-free route and on batch
                          handles; an FP32 pivot that fails falls back to FP64.  Each step's
                          residual bbar - H x is FP64 (iterative refinement), so the FP64
                          stopping test still decides.  Also SP-RK-RGS on a sparse A (see
                          ils_setup_csr). */
  ILS_BF16_REFINE = 2  /* as ILS_FP32_REFINE with B held in BF16 (FP32 accumulation) */
} ils_precision;

typedef enum {
  ILS_GRAM_FP64 = 0, /* A_1^T A_1 with FP64 fused multiply-adds */
  ILS_GRAM_SPLIT = 1 /* A_1^T A_1 to FP64 accuracy from exact integer slice products on tensor cores */
} ils_gram_mode;

typedef struct {
  int32_t method;      /* ils_method */
  int32_t precision;   /* ils_precision */
  int32_t gram;        /* ils_gram_mode */
  int32_t timing;      /* != 0: time the setup phases with CUDA events (see ils_get_timings) */
  int64_t max_outer;   /* outer-iteration cap; default 20000 (Sec. 5) */
  int64_t max_inner;   /* inner-step cap per outer iteration (randomized methods); 0 = 200 n */
  double theta;        /* inner stop: ||bhat - Abar1 z|| <= theta ||bbar - H x_k||; default 0.1 */
  int64_t check_every; /* RK-RGS inner residual test period in steps; 0 = n */
  int32_t scd_sampler; /* SP-SCD: 0 = rank sampler equal in law to Alg. 5 steps 7-9, 1 = greedy
                          (alpha = n, the Motzkin rule).  SP-RK-RGS: 2 = draw j2 = j1 (SP-RCD) */
  int32_t sweeps;      /* mixed precision: SP sweeps per FP64 refinement step; 0 = 3 */
  uint64_t seed;       /* Philox4x32-10 key for the randomized methods */
  int32_t route;       /* SP only: 0 auto, 1 explicit B = P Abar2, 2 matrix-free (stream A_2 every
                          step, never form Abar2; n <= 512).  Auto takes the route with the lower
                          modelled cost, setup + expected streams, from rates measured once per
                          process (the first auto setup of a process synchronizes and runs about a
                          millisecond of calibration kernels on synthetic data; see ils_route_model). */
  int32_t chain_ctas;  /* SP-RK-RGS on a sparse A: CTAs per inner chain.  0 = auto (the smallest
                          thread-block cluster of 1, 2, 4 or 8 CTAs whose shared memory holds
                          w and e, else one CTA with w and e in global memory); 1, 2, 4, 8 =
                          that cluster size; -1 = one CTA, vectors in global memory. */
  /* ---- fields below were added after the first release; ils_options_default sets them ---- */
  int32_t stop_rule;   /* ils_stop_rule: how `tol` of the solve calls is read (default relres) */
  int32_t estimate;    /* Lanczos estimates at setup (ils_info.rho_est, kappa_est, err_bound):
                          0 = none, 1 = rho(Abar1^{-1} Abar2) and kappa_2(A^T J A), 2 = kappa only
                          (the matrix-free route always estimates both).  ILS_STOP_ERR_BOUND
                          with 0 takes 2.  Estimates need n <= 4096 (else INVALID_ARG) */
  int32_t alpha_mode;  /* SP-SCD: 0 = alpha ~ U{1..n} each step (Alg. 5), 1 = fixed alpha_fixed
                          (Sec. 4: alpha = n is the greedy Motzkin rule, alpha = 1 a uniform pick) */
  int32_t sampler;     /* SP-RK-RGS column draws from ||A_1(:,j)||^2 / ||A_1||_F^2: 0 = inverse CDF
                          (the oracle's parity mode), 1 = Vose alias table (same law, O(1) draws) */
  int64_t alpha_fixed; /* 1 <= alpha_fixed <= n when alpha_mode = 1 */
  int32_t warm_inner;  /* randomized methods: != 0 starts each inner solve at x_k (z = x_k,
                          w = A_1 x_k; beta = x_k) instead of 0 (the paper's step); not in the paper */
  int32_t inner_form;  /* dense SP-RK-RGS: 0 = column form of Alg. 2 (O(p) per step), 1 = Gram form
                          (w = A_1 y carried as g = Abar1 y, h = Abar1 z: O(n) per step, same
                          iterates in exact arithmetic); not in the paper */
  const char* tune_cache; /* [host] file that keeps the sweep autotuner's choices between
                          processes: read at each mixed-precision setup (entries tuned on another
                          GPU model are ignored), rewritten after each new tuning; NULL = none.
                          The path is copied at setup */
  int64_t wait_limit_ns; /* bound in nanoseconds on each grid-barrier wait of the one-launch
                          mixed-precision solve; 0 = 1 s (the setup kernels keep their own 1-4 s
                          bounds).  A wait that runs out ends the kernel and the solve returns
                          ILS_ERR_TIMEOUT; the handle stays usable */
  int32_t lanczos_steps; /* Lanczos steps of the estimates; 0 = 24 (the extreme Ritz values of
                          these spectra settle to well under 1% by then) */
  int32_t factor64;    /* mixed precision, single dense handle: != 0 forms P = Abar1^{-1} from the
                          FP64 Cholesky factor of Abar1 and tests H by FP64 Cholesky (the
                          factorization stays FP64), instead of the FP32 Gauss-Jordan inverse */
  int32_t reserved0;
  double theta_decay;  /* randomized methods: the inner stop of outer iteration k uses
                          theta_k = max(theta * theta_decay^k, theta_min) (a schedule; not in the
                          paper); 1 (the default) or 0 keeps theta; 0 <= theta_decay <= 1 */
  double theta_min;    /* the schedule's floor (>= 0); default 0 */
} ils_options;

typedef enum {
  ILS_STOP_RELRES = 0,   /* stop once relres = ||A^T J (b - A x_k)|| / ||A^T J b|| <= tol */
  ILS_STOP_PAPER_RR = 1, /* Sec. 5's rule: stop once RR = relres^2 <= tol (e.g. tol = 1e-6) */
  ILS_STOP_ERR_BOUND = 2 /* stop once kappa_est * relres <= tol: kappa_2(H) relres bounds
                            ||x - x*|| / ||x*||, so tol is the target relative error */
} ils_stop_rule;

typedef enum { ILS_ROUTE_AUTO = 0, ILS_ROUTE_EXPLICIT = 1, ILS_ROUTE_MATRIX_FREE = 2 } ils_route;

typedef struct {
  int64_t outer_iters;  /* IT in the paper's tables (mixed precision: total SP sweeps) */
  int64_t inner_iters;  /* IT-inner: total inner steps over all outer iterations */
  int64_t refinements;  /* FP64 refinement steps (mixed precision), 0 otherwise */
  double relres;        /* ||A^T J (b - A x)|| / ||A^T J b|| of the returned x (FP64) */
  int32_t status;       /* ils_status of this solve */
  int32_t reserved;
  double err_bound;     /* kappa_est * relres: bounds ||x - x*|| / ||x*|| (Theorem 2.1's setting:
                           x - x* = -H^{-1} r and ||x*|| >= ||bbar|| / ||H||); 0 without estimates */
  double rho_est;       /* Lanczos estimate of rho(Abar1^{-1} Abar2), the SP contraction factor of
                           Theorem 2.1 (Ritz values lie inside the spectrum: rho_est <= rho up to
                           rounding); 0 without estimates */
  double kappa_est;     /* Lanczos estimate of kappa_2(A^T J A) (<= the true value up to rounding) */
  double t_setup_ms;    /* the handle's last setup on the device (CUDA events; options.timing) */
  double t_solve_ms;    /* wall time of this solve call, host clock */
  double t_inner_ms;    /* randomized methods: device time of the inner chains of the first
                           right-hand side (globaltimer), else 0 */
} ils_info;

/* Fill *o with the defaults above (method SP, FP64, FP64 Gram, max_outer 20000,
 * theta 0.1, seed 0).  Host only.  Returns ILS_ERR_INVALID_ARG if o is NULL. */
ils_status ils_options_default(ils_options* o);

/* Build a handle for one ILS instance (Alg. 1 steps 2-4; Alg. 2 steps 2-3;
 * Alg. 5 step 2).
 *   h    [host, out] receives the new handle (NULL on failure).
 *   m,n,p,q          A is m x n with m = p + q, p >= n >= 1, q >= 0.
 *   A    m x n, column-major, leading dimension lda >= m, FP64.  Read only; the
 *        handle copies what it needs, so A may be freed once the stream has
 *        passed this call.
 *   o    [host] options, or NULL for the defaults.
 * Work: copies A, forms Abar1 = A_1^T A_1 and Abar2 = A_2^T A_2 (FP64, or FP64-accurate
 * split tensor-core products when options.gram = ILS_GRAM_SPLIT or precision is mixed),
 * tests Abar1 and H = Abar1 - Abar2 for positive definiteness (the SPD test of eq. (1.3)) and
 * forms P = Abar1^{-1}, B = P Abar2.  FP64 handles (and mixed ones with options.factor64)
 * factor both matrices by FP64 Cholesky and form P from the factor; a mixed single dense
 * handle inverts Abar1 by FP32 block Gauss-Jordan elimination and sweeps H the same way
 * (its pivots are the Cholesky pivots), settling a failed FP32 pivot in FP64.  With
 * options.estimate, rho and kappa are estimated by Lanczos (matrix-free route: an estimate
 * rho >= 1 returns NOT_SPD).  Synchronizes the stream once to read the pivot status.
 * Errors: INVALID_ARG, OOM, CUDA, NOT_SPD (handle not created), NONFINITE. */
ils_status ils_setup(ils_handle* h, int64_t m, int64_t n, int64_t p, int64_t q,
                     const double* A, int64_t lda, const ils_options* o, ils_stream_t stream);

/* Build a handle for an instance whose A is sparse, given in CSR (Sec. 5 runs its
 * methods on sparse test matrices; the randomized steps of Alg. 2 read single
 * columns of A_1, which a column-sorted copy serves).
 *   h       [host, out] receives the new handle (NULL on failure).
 *   m,n,p,q as for ils_setup; rows 0..p-1 of A form A_1.
 *   nnz     number of stored entries, 0 <= nnz < 2^31.
 *   rowptr  m + 1 int32: row r holds entries rowptr[r] .. rowptr[r+1]-1; rowptr[0] = 0,
 *           rowptr[m] = nnz, nondecreasing.
 *   colind  nnz int32 column indices in [0, n), no (row, column) pair twice; any order
 *           within a row.
 *   val     nnz FP64 values.
 *   o       [host] options or NULL.  Every method runs in FP64.  precision =
 *           ILS_FP32_REFINE is accepted for ILS_SP (as for dense A) and for
 *           ILS_SP_RK_RGS, whose inner chain then runs in FP32 on the FP64 residual
 *           (x_k += d with Abar1 d = bbar - H x_k approximately); gram and route are ignored.
 * All three arrays are read only during this call's stream work: the handle keeps a
 * column-sorted CSC copy (entries of A_1 first in each column), Abar1 and Abar2 (formed
 * from the rows' outer products in FP64) and the same n x n products as ils_setup.
 * A column may hold at most 4096 entries.  Synchronizes the stream once.
 * Errors: INVALID_ARG (sizes, malformed CSR, a duplicate entry, a column over 4096
 * entries), NONFINITE, NOT_SPD, OOM, CUDA.  ils_refactor does not apply to such a
 * handle (INVALID_ARG). */
ils_status ils_setup_csr(ils_handle* h, int64_t m, int64_t n, int64_t p, int64_t q, int64_t nnz,
                         const int32_t* rowptr, const int32_t* colind, const double* val,
                         const ils_options* o, ils_stream_t stream);

/* Recompute every setup product of h for new matrix values of the same shape
 * (same m, n, p, q), allocating nothing.  Same errors as ils_setup; on
 * NOT_SPD the handle stays valid but must not be used to solve. */
ils_status ils_refactor(ils_handle h, const double* A, int64_t lda, ils_stream_t stream);

/* As ils_refactor without waiting for the setup: the copy of A and every setup product
 * are enqueued on `stream` and the call returns (the first call for a given n on a
 * mixed-precision handle waits once, to tune the sweep shapes).  A is read before any
 * later work on `stream`.  The next ils_solve / ils_solve_many on h, on the same stream,
 * runs behind the setup and then reports the setup's status: a failed setup's status
 * (NOT_SPD, NONFINITE, TIMEOUT, ...) replaces the solve's and x is unspecified; where an
 * FP64 factorization has to settle a failed FP32 pivot test, that solve performs it and
 * solves again.  On a mixed-precision single handle with split Grams the solve's
 * A^T J b (Alg. 1 step 4) runs on a second stream beside the setup's last products, and
 * the FP32 test of H (condition (1.3)) on a third stream beside the solve; with FP32
 * refinement, B = P Abar2 (which the one-cluster solve does not read) is formed on a
 * fourth stream once the solve's own kernels are enqueued, or before any path that reads it.
 * Since that A^T J b may run before the setup ends, the right-hand sides of the next solve
 * must be in place when ils_refactor_async is called (written by earlier work on `stream`
 * or by the host), not by work enqueued between the two calls.
 * Timings (ils_get_timings) are read at that solve.  Errors: INVALID_ARG, CUDA. */
ils_status ils_refactor_async(ils_handle h, const double* A, int64_t lda, ils_stream_t stream);

/* Solve for one right-hand side with the handle's method.
 *   b    length m, FP64.
 *   x    length n, FP64.  In: x0 unless x0_zero != 0.  Out: the solution.
 *   tol  stop once ||A^T J (b - A x_k)|| <= tol ||A^T J b|| (checked before each
 *        outer update, as in Sec. 5) or after max_outer updates; options.stop_rule reads
 *        tol instead as a bound on RR = relres^2 (Sec. 5) or on kappa_est * relres.
 *   info [host, out, may be NULL] iteration counts and the final relres.
 * Synchronizes the stream.  Errors: INVALID_ARG, NO_CONVERGENCE (x = last
 * iterate), NONFINITE, TIMEOUT, CUDA. */
ils_status ils_solve(ils_handle h, const double* b, double* x, int x0_zero, double tol,
                     ils_info* info, ils_stream_t stream);

/* Solve for k right-hand sides at once (columns of B, m x k, leading dimension
 * ldb >= m; X n x k, ldx >= n).  Each column stops on its own tolerance test.
 * info [host, may be NULL] receives the worst column (largest relres; the
 * largest iteration counts).  Synchronizes the stream. */
ils_status ils_solve_many(ils_handle h, int64_t k, const double* B, int64_t ldb, double* X,
                          int64_t ldx, int x0_zero, double tol, ils_info* info,
                          ils_stream_t stream);

/* Copy an internal n x n FP64 product of the handle into dst (device, column-major,
 * leading dimension ldd >= n): which = 0 Abar1, 1 Abar2, 2 FP64 Cholesky factor L of
 * Abar1 (lower triangle; the strict upper triangle of dst is set to 0; formed on demand,
 * synchronizing the handle's stream, where the setup factored Abar1 in FP32 only), 3 P = Abar1^{-1},
 * 4 B = P Abar2.  P and B are formed only by FP64 SP handles; Abar2 and B only on the
 * explicit route (a matrix-free handle streams A_2 instead); asking a handle for a matrix it
 * does not form is INVALID_ARG.  For tests and diagnostics.
 * Errors: INVALID_ARG, CUDA. */
ils_status ils_get_matrix(ils_handle h, int which, double* dst, int64_t ldd, ils_stream_t stream);

/* Setup phase times of the last ils_setup / ils_refactor on h, in milliseconds,
 * measured with CUDA events on the handle's stream when options.timing != 0
 * (zeros otherwise).  out [host] receives min(count, 14) values:
 *   0 Abar1 Gram, 1 the wait for the Abar2 Gram (its own time where it runs alone; on a
 *     mixed-precision single handle the FP32 copy of Abar1, the Abar2 Gram running on),
 *   2 the factor step: the Cholesky factorizations of Abar1 and H, or on a mixed-precision
 *     single handle the one-launch FP32 inverse of Abar1 (H is tested on another stream),
 *   3 the products that follow (P and B, or B alone after the inverse), with any wait for
 *     the Abar2 Gram (the FP32 test of H of a mixed single handle runs beside them and
 *     the next solve, and is not part of any phase),
 *   4 the whole setup, 5 the copy of A, 6 the tensor-core kernel of the Abar1 Gram alone
 *   (split Grams only);
 * and of the last solve (its first pass of up to 8 right-hand sides):
 *   7 from the end of the setup to the solve's first work on the stream (0 when the solve
 *     was enqueued behind the setup), 8 the solve's work up to its answer (A^T J b, the
 *     iteration and any wait for kappa_est; where the iteration is not one launch, up to
 *     its first chunk), 9 the copy of the answer and of the results to the host;
 * and, on a mixed-precision single handle, 10 the start of the kappa(H) estimate after the
 * start of the setup, 11 its duration (with estimates), 12 the moment both Grams were
 * done for the forming of H and 13 the moment H was formed (both after the start of the
 * setup).
 * Returns the number of values written (at most 14), or -1 on a bad argument. */
int ils_get_timings(ils_handle h, double* out, int count);

/* The launch shape the autotuner picked for the mixed-precision sweep GEMV of an n x n
 * operator with k right-hand sides (bf16 != 0: the BF16 copy of B): *warps per CTA and
 * *blocks CTAs.  The first mixed-precision setup of a given n (rounded up to 32) times
 * 1, 2, 4 and 8 warps per CTA with one, two or four rows per warp on its own operators
 * and keeps the fastest for the rest of the process (k classes: k <= 2 and k > 2).
 * Returns 1 when a tuned shape exists, else 0 (the default shape is then used).  Host
 * only; warps and blocks may be NULL. */
int ils_tuned_shape(int64_t n, int64_t k, int bf16, int* warps, int* blocks);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles, all threads).  Host only. */
int64_t ils_kernel_launches(void);

/* ---- Batches of independent problems (uneven m, n, p, q) ---------------------------------- */

typedef struct ils_batch_s* ils_batch;

/* One problem of a batch: A is m x n, column-major, leading dimension lda >= m, FP64,
 * device memory; rows 0..p-1 form A_1 and rows p..m-1 form A_2. */
typedef struct {
  int64_t m, n, p, q;
  const double* A;
  int64_t lda;
} ils_problem;

/* Set up `count` independent problems (probs is a host array) with the same options.
 * Each problem is set up exactly as by ils_setup; the problems' kernels are spread over
 * internal streams so they run concurrently, ordered after the work already on `stream`;
 * the call returns when every setup has finished.  On any failure nothing is kept and the
 * first failing status is returned (INVALID_ARG, OOM, CUDA, NOT_SPD, NONFINITE). */
ils_status ils_batch_setup(ils_batch* b, int64_t count, const ils_problem* probs, const ils_options* o,
                           ils_stream_t stream);

/* Solve k right-hand sides for every problem of the batch.  B and X are host arrays of
 * `count` device pointers: B[i] is m_i x k (leading dimension ldb[i] >= m_i, or m_i when
 * ldb is NULL) and X[i] is n_i x k (ldx[i] >= n_i, or n_i when ldx is NULL).  x0_zero and
 * tol as in ils_solve_many.  infos [host, may be NULL] receives one ils_info per problem.
 * The work is ordered after `stream` and `stream` waits for it; the call synchronizes.
 * Returns ILS_OK or the first non-OK problem status. */
ils_status ils_batch_solve(ils_batch b, int64_t k, const double* const* B, const int64_t* ldb, double* const* X,
                           const int64_t* ldx, int x0_zero, double tol, ils_info* infos, ils_stream_t stream);

/* Record one batch solve as a CUDA graph, to be replayed by ils_batch_run with a single
 * graph launch (the batched form of the spec design: every problem's kernels, on
 * the batch's internal streams, in one launch).  Nothing is computed by this call.
 *   refactor  != 0: each replay first recomputes every setup product from the A pointers
 *             given to ils_batch_setup (their contents may change between replays, their
 *             addresses and shapes may not); 0: the products of the last setup are used.
 *   k         right-hand sides per problem, 1 <= k <= 8.
 *   B, ldb, X, ldx, x0_zero, tol  as in ils_batch_solve; these device buffers are baked
 *             into the graph, so every replay reads B and writes X at the same addresses.
 *   steps     outer steps recorded per problem (each returns at once once its problem
 *             has converged); a problem that needs more is finished by ils_batch_run on
 *             the host-driven path.
 *   stream    must not be the legacy default stream (it cannot be captured).
 * Replaces any earlier capture of the batch.  Errors: INVALID_ARG, CUDA. */
ils_status ils_batch_capture(ils_batch b, int refactor, int64_t k, const double* const* B, const int64_t* ldb,
                             double* const* X, const int64_t* ldx, int x0_zero, double tol, int64_t steps,
                             ils_stream_t stream);

/* Replay the captured batch solve on `stream` and synchronize it; problems that had not
 * converged within the captured steps continue on the host-driven path.  infos [host,
 * may be NULL] receives one ils_info per problem (a refactor's NOT_SPD or NONFINITE is
 * reported there).  Returns ILS_OK or the first non-OK problem status; INVALID_ARG when
 * nothing was captured. */
ils_status ils_batch_run(ils_batch b, ils_info* infos, ils_stream_t stream);

/* The handle of problem i (owned by the batch; for ils_get_matrix and diagnostics), or
 * NULL when i is out of range. */
ils_handle ils_batch_handle(ils_batch b, int64_t i);

/* Release the batch and every handle it owns.  NULL is ignored. */
void ils_batch_destroy(ils_batch b);

/* ---- Learned warm start ---------------------------------------------------------------------
 * A three-layer perceptron x0 = net(theta) for parametric right-hand sides b(theta):
 *   z1 = W1 theta + b1, h1 = gelu(z1), z2 = W2 h1 + b2, h2 = gelu(z2), y = W3 h2 + b3,
 *   x0 = mu + sigma * y  (mu, sigma: per-coordinate mean and deviation of the training
 *   targets), gelu(z) = z Phi(z).  The paper has no counterpart.  Weights are FP32 and
 *   trained on the GPU by this library's kernels (mean-squared error on standardized
 *   targets, Adam); inference runs in BF16 or FP32.  Parameters are stored flat: W1
 *   (d_hidden x d_in, row-major), b1, W2 (d_hidden x d_hidden), b2, W3 (d_out x d_hidden),
 *   b3.  Samples are contiguous: theta is d_in x count and targets/outputs d_out x count,
 *   column-major. */
typedef struct ils_mlp_s* ils_mlp;

/* New network with weights and biases ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) drawn from
 * Philox4x32-10 keyed by `seed`; mu = 0, sigma = 1.  Errors: INVALID_ARG, OOM, CUDA. */
ils_status ils_mlp_create(ils_mlp* net, int64_t d_in, int64_t d_hidden, int64_t d_out, uint64_t seed,
                          ils_stream_t stream);
/* Number of FP32 parameters (-1 for NULL). */
int64_t ils_mlp_num_params(ils_mlp net);
/* Copy the flat FP32 parameters to / from device memory. */
ils_status ils_mlp_get_params(ils_mlp net, float* dst, ils_stream_t stream);
ils_status ils_mlp_set_params(ils_mlp net, const float* src, ils_stream_t stream);
/* Mean over count x d_out entries of (y - (T - mu)/sigma)^2 for 1 <= count <= 1024 samples
 * (loss, host, FP64) and its gradient with respect to the flat parameters (grad, device,
 * FP32).  Synchronizes the stream. */
ils_status ils_mlp_loss_grad(ils_mlp net, int64_t count, const float* theta, const double* T, double* loss,
                             float* grad, ils_stream_t stream);
/* Set mu, sigma from the targets T (d_out x count, FP64) and run `epochs` passes of Adam
 * (lr; beta1 0.9, beta2 0.999, eps 1e-8) over minibatches of `batch` <= 1024 consecutive
 * samples.  final_loss [host, may be NULL]: loss of the last minibatch seen.  Synchronizes. */
ils_status ils_mlp_train(ils_mlp net, int64_t count, const float* theta, const double* T, int64_t epochs,
                         int64_t batch, double lr, double* final_loss, ils_stream_t stream);
/* X(:, i) = net(theta(:, i)) for count samples (X d_out x count, ldx >= d_out, FP64);
 * bf16 != 0 runs the layers in BF16 with FP32 accumulation.  Non-finite outputs are 0. */
ils_status ils_mlp_forward(ils_mlp net, int64_t count, const float* theta, double* X, int64_t ldx, int bf16,
                           ils_stream_t stream);
/* Solve for k parametric right-hand sides B(:, i) = b(theta(:, i)) starting from the
 * network's prediction (BF16 inference), as ils_solve_many with x0 = net(theta).  Since the
 * iteration converges from any start, the prediction only changes the iteration count.
 * Requires d_in of the net = rows of theta and d_out = n.  net = NULL uses the network set by
 * ils_set_warmstart (INVALID_ARG when none is set). */
ils_status ils_solve_param(ils_handle h, ils_mlp net, int64_t k, const float* theta, const double* B, int64_t ldb,
                           double* X, int64_t ldx, double tol, ils_info* info, ils_stream_t stream);
void ils_mlp_destroy(ils_mlp net);

/* Attach a network to the handle (the handle does not own it; NULL detaches): a later
 * ils_solve_param with net = NULL starts from this network's prediction.  Checks that the
 * network's output size equals n.  Host only.  Errors: INVALID_ARG. */
ils_status ils_set_warmstart(ils_handle h, ils_mlp net);

/* Gram product C = X^T X (FP64) without any device allocation.  The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc (for
 * example code that runs under stream capture with allocation forbidden, or inside a
 * host application whose allocator owns all device memory).
 *   K, n  X is K x n, column-major, leading dimension ldx >= max(K, 1); 1 <= n <= 1024
 *         (larger n is rejected with ILS_ERR_INVALID_ARG).  K = 0 gives C = 0.
 *   C     n x n, column-major, ldc >= n; both triangles are written.
 * The split-K partial sums live in a fixed 16 MiB array (2^21 doubles) inside the
 * library's device memory, resident on every GPU that loads the library until the
 * process exits; when they would not fit, the call uses fewer, longer K slices.  The
 * first call on each device looks up that array's device address (with that device
 * current), so make the first call on a device before any stream capture; the address
 * stays valid for the CUDA context current at that call (a context torn down and created
 * again, for example by cudaDeviceReset, needs a new process).  Every call
 * shares the array: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race on it and must be serialized by the caller.  Enqueues
 * work only; nothing is synchronized.  Errors: INVALID_ARG, CUDA. */
ils_status ils_gram_noalloc(int64_t K, int64_t n, const double* X, int64_t ldx, double* C, int64_t ldc,
                            ils_stream_t stream);

/* v = A_2^T (A_2 x) for one vector (length n in, length n out, FP64, device) by the
 * handle's one-pass stream over its row-major copy of A_2: prec 0 streams the FP64-accurate
 * copy (FP64 on an FP64 handle; on a mixed-precision handle the double-FP32 copy, each
 * entry as its FP32 rounding plus the FP32 rounding of the rest, carried in double-FP32
 * arithmetic), 1 the FP32 copy, 2 the BF16 copy (FP32 accumulation); the copy must exist
 * (matrix-free route; the low-precision copy in the matching mixed precision).  For tests
 * and bandwidth measurements.  Errors: INVALID_ARG, CUDA. */
ils_status ils_aq_product(ils_handle h, const double* x, double* v, int prec, ils_stream_t stream);

/* The last automatic route decision (options.route = auto) of this process, host only.  out
 * receives min(count, 9) values: the modelled extra cost of the explicit route and of the
 * matrix-free route in seconds (explicit: Abar2 = A_2^T A_2 by the Gram route of the
 * handle's precision plus B = P Abar2; matrix-free: the row-major copies of A_2 plus the
 * expected streams of a solve), the measured split-digit Gram rate and FP64 Gram rate (flop/s
 * in p n^2 units), the measured stream rates of the FP64, FP32 and BF16 copies (bytes/s), the
 * copy rate (bytes/s), and 1 if the matrix-free route was taken.  The paper has no
 * counterpart (its SP forms B).  Returns the number of values written, -1 on a bad argument. */
int ils_route_model(double* out, int count);

/* Change options.wait_limit_ns of an existing handle (0 restores the default).  Host only.
 * Errors: INVALID_ARG. */
ils_status ils_set_wait_limit(ils_handle h, int64_t limit_ns);

/* Diagnostic: record the column indices the randomized inner chain of the first right-hand
 * side picks in the first outer iteration of each later solve: SP-SCD writes j_t at picks[t]
 * (Alg. 5 step 9), SP-RK-RGS writes j1 at picks[2t] and j2 at picks[2t + 1] (Alg. 2 steps 8
 * and 10); steps beyond capacity are not recorded.  picks is device memory owned by the
 * caller (int32, capacity entries); NULL stops recording.  Dense handles only.
 * Errors: INVALID_ARG. */
ils_status ils_record_picks(ils_handle h, int32_t* picks, int64_t capacity);

/* Release everything the handle owns (stream-ordered on the stream it was
 * created with).  NULL is ignored. */
void ils_destroy(ils_handle h);

/* Description of the last CUDA failure that made a call of this thread return
 * ILS_ERR_CUDA (the failing call and the CUDA error string); "" if none.  Host only. */
const char* ils_last_error(void);

/* Static, human-readable name of a status code.  Host only. */
const char* ils_status_string(ils_status st);

#ifdef __cplusplus
}
#endif

#endif /* ILS_H */
