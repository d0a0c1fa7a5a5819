// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ils.h"

namespace ils {

// Device-side state of one iterative solve, updated by the kernels themselves so
// the outer loop needs no host round trip until it ends.
struct SolveState {
  int32_t done;       // all columns finished (converged, cap reached or non-finite)
  int32_t cur;        // which of the two iterate buffers holds x_k
  int32_t status;     // ils_status of the solve
  int32_t pad0;
  int64_t iters;      // outer updates made so far (max over columns)
  int64_t max_outer;
  int64_t inner_total;
  uint32_t counter;   // arrival counter of the last-block reduction
  uint32_t pad1;
};

constexpr int kMaxRhsPerPass = 8;  // right-hand sides carried per iteration launch

// The results of a pass, gathered on the device into one block so that a single copy
// brings them to the host: the solve state, then per right-hand side ||r||^2, ||bbar||^2,
// outer and inner iterations, then the inner chain time.  Byte offsets:
constexpr size_t kResSt = 0, kResRr = 64, kResBn = kResRr + 8 * kMaxRhsPerPass,
                 kResIters = kResBn + 8 * kMaxRhsPerPass, kResInner = kResIters + 8 * kMaxRhsPerPass,
                 kResInnerNs = kResInner + 8 * kMaxRhsPerPass, kResBytes = kResInnerNs + 64;
static_assert(sizeof(SolveState) <= kResRr, "state slot");
struct ResultGather {
  const SolveState* st;
  const double* rr;
  const double* bn;
  const int64_t* iters;
  const int64_t* inner;
  const unsigned long long* inner_ns;  // may be null
  void* out;                           // kResBytes on the device
  int64_t k;
};

// Record a failed CUDA call for ils_last_error (this thread) and clear CUDA's sticky error
// state; returns ILS_ERR_CUDA.
ils_status record_cuda_error(cudaError_t e, const char* what, int line);

// Accessors of the handle for the other translation units.
int64_t handle_n(ils_handle h);
ils_mlp handle_warm_net(ils_handle h);
void handle_set_warm_net(ils_handle h, ils_mlp net);

// Host-side count of kernel launches made by this library (reported by ils_kernel_launches).
void note_launch(int64_t count = 1);

// ---- dense FP64 building blocks (dense_f64.cu) -------------------------------------------

// C = X^T Y with X (K x n1, ldx) and Y (K x n2, ldy) column-major, FP64 FMA.
// Rows r >= sign_split of Y are negated (sign_split = K for a plain product), which
// forms A^T J B in one pass.  sym: n1 == n2, X == Y, only upper tiles are computed and
// the result is mirrored.  trans_out: C is written transposed.  work must hold
// gemm_tn_work_elems(...) doubles when splits > 1.
size_t gemm_tn_work_elems(int64_t K, int64_t n1, int64_t n2, bool sym, int* splits_out);
cudaError_t gemm_tn_f64(int64_t K, int64_t n1, int64_t n2, const double* X, int64_t ldx,
                        const double* Y, int64_t ldy, int64_t sign_split, double* C,
                        int64_t ldc, bool sym, bool trans_out, double* work, cudaStream_t s);

// Symmetric C = X^T X like gemm_tn_f64, with the split-K partial sums limited to
// work_cap_elems doubles of the given work array (fewer, longer K slices if needed).
cudaError_t gemm_tn_f64_capped(int64_t K, int64_t n, const double* X, int64_t ldx, double* C, int64_t ldc,
                               double* work, size_t work_cap_elems, cudaStream_t s);

// out(:,c) = A^T J b(:,c) for k right-hand sides: A m x n (lda), B m x k (ldb),
// rows >= p carry the minus sign of J.  out is n x k (ldo).
cudaError_t rhs_bar_f64(int64_t m, int64_t n, int64_t p, int64_t k, const double* A, int64_t lda,
                        const double* B, int64_t ldb, double* out, int64_t ldo, cudaStream_t s);

// Y(:,c) = M^T X(:,c) for an n x n column-major M (so row i of M^T is column i of M).
cudaError_t gemv_cols_f64(int64_t n, int64_t k, const double* M, int64_t ldm, const double* X,
                          int64_t ldx, double* Y, int64_t ldy, cudaStream_t s);

// In-place blocked Cholesky of the lower triangles of `count` (1 or 2) n x n matrices
// (ld n), factored together.  inv_diag[i] (length n) receives 1 / L_jj.  stash: count x
// 1024 scratch elements.  status (device int) is set to ILS_ERR_NOT_SPD or
// ILS_ERR_NONFINITE on a bad pivot of any matrix.
cudaError_t cholesky_f64_batch(int64_t n, int count, double* const* mats, double* const* inv_diag, double* stash,
                               int32_t* status, cudaStream_t s);

// Cholesky of one FP32 matrix in place (lower triangle; inv_diag gets 1 / L_ii).  Up to
// n = 768 it is one data-driven launch and `stash` (1024 floats) holds its chunk flags;
// larger n takes the panel launches above.  Status as above.
cudaError_t cholesky_f32(int64_t n, float* M, float* inv_diag, float* stash, int32_t* status, cudaStream_t s);
// Two FP32 matrices in one launch, each with its own status word (stash: 2048 floats).
cudaError_t cholesky_f32_pair(int64_t n, float* M0, float* M1, float* inv0, float* inv1, float* stash,
                              int32_t* status0, int32_t* status1, cudaStream_t s);

// X := L^{-1} X (lower = forward) then, if both, X := L^{-T} X.  X n x k (ldx).
cudaError_t trsm_lower_f64(int64_t n, int64_t k, const double* L, double* X, int64_t ldx,
                           bool forward, bool backward, cudaStream_t s);
cudaError_t trsm_lower_f32(int64_t n, int64_t k, const float* L, float* X, int64_t ldx,
                           bool forward, bool backward, cudaStream_t s);
// Same solves by 32-row blocks with explicit inverses of L's 32 x 32 diagonal blocks
// (written to Dinv, ceil(n/32) * 1024 elements); the right-hand sides of a CTA stay in
// shared memory with one 32 x n panel of L (n <= 708 in FP64, 1422 in FP32).
cudaError_t trsm_binv_f64(int64_t n, int64_t k, const double* L, double* Dinv, double* X, int64_t ldx,
                          bool forward, bool backward, cudaStream_t s);
// Dinv = inverses of the 32 x 32 diagonal blocks of the lower-triangular L (block after block).
cudaError_t diag_block_inverse_f32(int64_t n, const float* L, float* Dinv, cudaStream_t s);
cudaError_t trsm_binv_f32(int64_t n, int64_t k, const float* L, float* Dinv, float* X, int64_t ldx,
                          bool forward, bool backward, cudaStream_t s);

// dst (m x n, ld m) = src (m x n, ld lda), both device memory.
cudaError_t copy_matrix_f64(int64_t m, int64_t n, const double* src, int64_t lda, double* dst, cudaStream_t s);

// Elementwise helpers.
cudaError_t set_identity_f64(int64_t n, double* M, int64_t ld, cudaStream_t s);
cudaError_t axpby_mat_f64(int64_t n, double alpha, const double* X, double beta, const double* Y,
                          double* Z, cudaStream_t s);
// Z = X - Y (n x n, FP64) and its FP32 rounding Z32, in one pass.
cudaError_t diff_mat_f64_f32(int64_t n, const double* X, const double* Y, double* Z, float* Z32, cudaStream_t s);  // Z = alpha X + beta Y, n*n contiguous
cudaError_t copy_lower_zero_upper_f64(int64_t n, const double* L, double* dst, int64_t ldd,
                                      cudaStream_t s);
cudaError_t sq_norms_cols_f64(int64_t n, int64_t k, const double* X, int64_t ldx, double* out,
                              cudaStream_t s);

// One outer step for up to kMaxRhsPerPass columns.  For every unfinished column it
// forms the residual r_k = bbar - H x_k of Sec. 5's stopping test and either
//   mode 0 (SP, Alg. 1 step 6):        x_{k+1} = B x_k + c  (M = B^T, addv = c), or
//   mode 1 (randomized, Alg. 2 step 5 / Alg. 5 step 4): bhat = Abar2 x_k + bbar
//          (M = Abar2, addv = bbar), written to bhat_out for the inner chain, or
//   mode 2 (mixed-precision refinement): r_k itself is written to bhat_out and x_k stays
//          in place (the correction kernels update it);
//   mode 3 (matrix-free SP): with v = A_2^T (A_2 x_k) given in vvec, r_k = bbar + v - Abar1 x_k
//          (H = Abar1) and x_{k+1} = P (v + bbar) (M = P);
//   mode 4 (matrix-free refinement): r_k = bbar + v - Abar1 x_k written to bhat_out, x_k in
//          place.
// See dense_f64.cu for the completion protocol.
struct SpIterArgs {
  int64_t n, k;
  int32_t mode;
  int32_t pad;
  const double* Bt;    // M, column-major n x n: column i = row i of the operator
  const double* H;     // A^T J A (symmetric)
  const double* cvec;  // addv, n x k
  const double* bbar;  // n x k
  const double* bnorm2;  // k
  double* X0;          // n x k iterate buffers
  double* X1;
  double* bhat_out;    // n x k (modes 1, 2, 4)
  const double* vvec;  // n x k: A_2^T (A_2 x_k) (modes 3, 4)
  double tol2;         // squared relres target (tol^2, or tol for Sec. 5's RR rule)
  const double* tol_scale;  // device scalar multiplying tol2 (1 / kappa_est^2 for the error-bound
                            // rule), or nullptr
  int64_t wait_ns;          // bound on the grid-barrier waits of the one-launch solve; 0 = 1 s
  double theta2;       // theta^2 (mode 1): inner target = theta_k^2 ||r_k||^2 with
  double theta_decay;  // theta_k = max(theta theta_decay^k, theta_min) (theta_decay 0 or 1: theta)
  double theta_min2;
  double* col_target2; // k (mode 1)
  int32_t* col_done;   // k flags
  double* col_rr;      // k: ||r||^2 of each column's returned iterate
  int64_t* col_iters;  // k
  double* partials;    // gridDim x k
  SolveState* st;
};
cudaError_t sp_iterate_f64(const SpIterArgs& a, cudaStream_t s);

struct MixedArgs;
// The mixed-precision refinement of one right-hand side (explicit route), every outer step
// up to st->max_outer, in one cooperative launch (solve_fused.cu); same state and results
// as sp_iterate_f64 (mode 2) + mixed_correct per step.  `sync`: 4 words.
// cudaErrorNotSupported when k != 1 or cooperative launch is unavailable.
// phase 0: the whole solve; 1: provisional, stopping on tol2 alone (col_done = 2 when that
// is met: ||r||^2 and r of x are kept); 2: resume after a provisional launch with the final
// rule (tol2 * tol_scale), refining on if the kept residual fails it.
// b_ready: where B = P Abar2 is formed off the stream, fn(ctx, &ev) yields the event that
// orders it (enqueuing its formation first where the setup deferred it); the launch makes
// the stream wait for it before any kernel that reads B (the one-cluster kernel with A2_32
// does not, and never calls fn).  fn null: B is formed on the stream already.
struct BReady {
  cudaError_t (*fn)(void* ctx, cudaEvent_t* ev) = nullptr;
  void* ctx = nullptr;
};
cudaError_t mixed_solve_fused(const SpIterArgs& sa, const MixedArgs& ma, int precision, uint32_t* sync,
                              cudaStream_t s, int phase = 0, BReady b_ready = BReady());
int sp_iterate_blocks(int64_t n);

// Copy the final iterate buffer (chosen on the device) into the user's X.
cudaError_t copy_final_f64(int64_t n, int64_t k, const double* X0, const double* X1,
                           const SolveState* st, double* X, int64_t ldx, cudaStream_t s, const ResultGather* gather = nullptr);

// ---- FP64-accurate Gram from exact integer slice products on tcgen05 (gram_split_tc.cu) ----
struct GramSplitWork {
  size_t slice_elems = 0;    // BF16 slices
  size_t partial_elems = 0;  // partial products (FP32 values in a buffer of this many doubles)
  size_t exps = 0;           // int exponents
};
GramSplitWork gram_split_work(int64_t K, int64_t n);
// C = A^T A for the K x n column-major A (lda), both triangles written.  err (device int)
// is set to 1 on a tensor-pipeline timeout and 2 on a non-finite input.  mma_begin /
// mma_end, when set, are recorded on s around the tensor-core launch alone.  With a_copy,
// A is also copied there (leading dimension ld_copy), by the digit split where it can, and
// `copied` (if set) is recorded once the copy is complete.
cudaError_t gram_split_tc(int64_t K, int64_t n, const double* A, int64_t lda, double* C, int64_t ldc,
                          void* slices, double* partial, int* exps, int32_t* err, cudaStream_t s,
                          cudaEvent_t mma_begin = nullptr, cudaEvent_t mma_end = nullptr, double* a_copy = nullptr,
                          int64_t ld_copy = 0, cudaEvent_t copied = nullptr);
// The two Grams C1 = A1^T A1 (K1 x n) and C2 = A2^T A2 (K2 x n) with their tensor-core
// products in one launch: the digit splits run on s1 and s2 (A2's recorded by ev_split2),
// the shared product kernel on s1 (ev_mma after it), the reductions on s1 and s2.  The
// digit buffers, partials and exponents are per Gram; copy1 / copy2 (ld_copy) receive the
// copies of A1 and A2, copied1 is recorded on s1 after A1's.
cudaError_t gram_split_pair_tc(int64_t K1, int64_t K2, int64_t n, const double* A1, int64_t lda1, const double* A2,
                               int64_t lda2, double* C1, double* C2, int64_t ldc, void* slices1, void* slices2,
                               double* partial1, double* partial2, int* exps1, int* exps2, int32_t* err,
                               cudaStream_t s1, cudaStream_t s2, cudaEvent_t ev_split2, cudaEvent_t ev_mma,
                               cudaEvent_t mma_begin, cudaEvent_t mma_end, double* copy1, double* copy2,
                               int64_t ld_copy, cudaEvent_t copied1);

// General product C = X^T Y (X: K x n1, Y: K x n2) to FP64 accuracy from the same exact digit
// products, on digit slices made by split_digits (rows >= sign_split of the split matrix are
// negated: J's sign for A^T J B).  C0 != nullptr gives C = C0 - X^T Y (C may equal C0).
// partial holds gemm_partial_elems doubles; slices digit_slice_elems BF16 values; err as above.
size_t digit_slice_elems(int64_t K, int64_t n);
size_t gemm_partial_elems(int64_t K, int64_t n1, int64_t n2);
cudaError_t split_digits(int64_t K, int64_t n, const double* A, int64_t lda, int64_t sign_split, void* slices,
                         int* exps, int32_t* err, cudaStream_t s);
cudaError_t gemm_split_tc(int64_t K, int64_t n1, int64_t n2, const void* slicesX, const int* expsX,
                          const void* slicesY, const int* expsY, double* C, int64_t ldc, const double* C0,
                          int64_t ldc0, double* partial, int32_t* err, cudaStream_t s);

// ---- mixed precision for many right-hand sides (wide_mixed.cu) -----------------------------
constexpr int64_t kWideMixedBlock = 1024;  // right-hand sides refined together
struct WideMixedArgs {
  int64_t m, n, p;
  const double* A;       // m x n, ld m
  const double* H;       // A^T J A (FP64)
  const float* P32;      // Abar1^{-1}
  const float* Bt32;     // (P Abar2)^T
  int32_t sweeps;
  int64_t max_outer;     // refinement cap
  double tol2;
  const double* tol_scale;
};
struct WideMixedResult {
  double relres;         // largest relres over the columns
  int64_t refinements;   // largest number of refinement steps
  int32_t status;
};
// h_state: pinned host memory for 3 int32.  Synchronizes s once per refinement step.
cudaError_t wide_mixed_solve(const WideMixedArgs& a, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                             int x0_zero, WideMixedResult* res, int32_t* h_state, cudaStream_t s);

// ---- matrix-free A_2 products (stream.cu) ---------------------------------------------------
// Row-major copy of A_2 (q x n, column-major source with leading dimension lda) with rows
// padded to aq_row_stride(n) elements; prec 0 FP64, 1 FP32, 2 BF16.
int64_t aq_row_stride(int64_t n);
int aq_stream_blocks();
cudaError_t aq_copy_rows(int64_t q, int64_t n, const double* Ac, int64_t lda, void* Ar, int prec, cudaStream_t s);
// v = A_2^T (A_2 x) in one pass; part: aq_stream_blocks() * n accumulators (double for
// prec 0, float otherwise).  n <= 512 in FP64, n <= 1024 otherwise.
cudaError_t aq_product(int64_t q, int64_t n, const void* Ar, int prec, const double* x, void* part, double* v,
                       cudaStream_t s);
// Same product for column c of the current iterate buffer (chosen on the device from st):
// returns at once when the solve is done or column c is finished.
cudaError_t aq_product_iterate(int64_t q, int64_t n, const void* Ar, int prec, const double* X0, const double* X1,
                               const SolveState* st, const int32_t* col_done, int c, void* part, double* v,
                               cudaStream_t s);

// ---- mixed precision with FP64 refinement (mixed.cu) ----------------------------------------
struct MixedArgs {
  int64_t n, k;
  int32_t sweeps;         // SP sweeps per correction (>= 1)
  int32_t pad;
  const double* r;        // n x k FP64 residuals (from the mode-2 outer step)
  float* r32;             // n x k
  float* c32;             // n x k: P r
  float* d32[2];          // n x k ping-pong sweep iterates
  const float* P32;       // Abar1^{-1}
  const float* Bt32;      // (P Abar2)^T
  const void* Bt16;       // BF16 copy of Bt32 (ILS_BF16_REFINE)
  double* X0;
  double* X1;
  const int32_t* col_done;
  SolveState* st;
  // H row-scaled in double-FP32 form for the one-cluster solve (null: not formed this setup)
  const float* Hh;
  const float* Hl;
  const int32_t* He;
  // Abar2 in FP32 (symmetric): where set, the one-cluster solve sweeps d_{s+1} = P (Abar2 d_s + r)
  // instead of B d_s + P r, and need not wait for B
  const float* A2_32;
};
// H(i, j) = 2^He[i] (Hh + Hl)(i, j) with |Hh + Hl| < 1 and Hl the FP32 rounding of what Hh
// leaves: about 48 bits of every entry, kept in FP32 so that H x can run on the FP32 pipe
// (solve_fused.cu).  H is n x n symmetric (row i = column i).
cudaError_t split_rows_df(int64_t n, const double* H, float* Hh, float* Hl, int32_t* He, cudaStream_t s);
constexpr int64_t kClusterSolveMaxN = 512;  // the one-cluster solve: 16 CTAs of 32 rows
// Launch shape of the sweep GEMV: warps per CTA and CTAs (each warp takes whole rows).
struct SweepShape {
  int32_t warps;
  int32_t blocks;
};
// The shape for (n, k, operator type): tuned if ils_tune_sweeps ran for it, else a default.
SweepShape sweep_shape(int64_t n, int64_t k, bool bf16);
// Time the candidate shapes for (n, k) on the handle's operators (P32 and Bt32 or Bt16) and
// cache the fastest, once per process.  Synchronizes `s`; not for use inside a capture.
// cache: a file keeping the choices between processes (read first, rewritten after new tuning), or null.
// Whether the sweep shapes for (n, precision) are tuned in this process.
bool sweeps_tuned(int64_t n, int precision);
cudaError_t tune_sweeps(int64_t n, int precision, const float* P32, const float* Bt32, const void* Bt16,
                        float* scratch_in, float* scratch_out, SolveState* st, cudaStream_t s,
                        const char* cache = nullptr);
// 1 and the tuned shape of (n, k, operator type) if the autotuner has one, else 0.
int ils_tuned_shape_impl(int64_t n, int64_t k, int bf16, int* warps, int* blocks);
// L32/P32/G2_32/Bt32 are n x n FP32 buffers, Bt16 an n x n BF16 buffer (BF16 mode only).
// L is the FP64 Cholesky factor, rounded into L32; L == nullptr means L32 already holds an
// FP32 factor (lower triangle, zeros above).  G2 == nullptr (matrix-free route) forms only P32.
cudaError_t mixed_setup(int64_t n, const double* L, const double* G2, int precision, float* L32, float* P32,
                        float* G2_32, float* Bt32, void* Bt16, float* Dinv32, cudaStream_t s);
// B^T (FP32, and BF16 in BF16 mode) from P32 and Abar2: G2 (FP64) is rounded into G2_32
// first unless it is nullptr (then G2_32 already holds it).
cudaError_t mixed_setup_b(int64_t n, const double* G2, int precision, const float* P32, float* G2_32, float* Bt32,
                          void* Bt16, cudaStream_t s);
cudaError_t mixed_correct(const MixedArgs& a, int precision, cudaStream_t s);

// FP32 GEMM C = alpha op(A) op(B) + beta C (column-major; ta/tb: transposed operand), batched
// over `batch` with element strides sa, sb, sc (mixed.cu).
struct GemmF32 {
  int64_t M, N, K, lda, ldb, ldc, sa, sb, sc;
  const float* A;
  const float* B;
  float* C;
  float alpha, beta;
};
cudaError_t gemm_f32(bool ta, bool tb, const GemmF32& g, int64_t batch, cudaStream_t s);

// ---- explicit SPD inverse (spd_gj.cu) ------------------------------------------------------
// P[i] := A[i]^{-1} for count (1 or 2) n x n FP32 symmetric matrices (both triangles
// stored, column-major) by block Gauss-Jordan elimination in one cooperative launch;
// P[i] == nullptr tests A[i] only.  status[i] gets NOT_SPD / NONFINITE on a failed pivot
// (the FP32 counterpart of the Cholesky pivot test) and TIMEOUT if a flag wait ran out.
// Tiles are 32 x 32 where each gets a CTA of its own, else 64 x 64 (wide_first: 64 x 64
// wherever they fit, fewer CTAs for a launch beside other work).  `scratch` holds
// spd_inverse_scratch_floats(n) floats.  cudaErrorNotSupported when neither fits (nothing
// is enqueued; the caller takes another route).
size_t spd_inverse_scratch_floats(int64_t n);
cudaError_t spd_inverse_f32(int64_t n, int count, const float* const* A, float* const* P, float* scratch,
                            int32_t* const* status, cudaStream_t s, bool wide_first = false);
cudaError_t convert_f64_to_f32(int64_t count, const double* src, float* dst, cudaStream_t s);
// L32 := lower triangle of the n x n FP64 matrix M rounded to FP32, zeros above.
cudaError_t lower_to_f32(int64_t n, const double* M, float* L32, cudaStream_t s);
cudaError_t mixed_correct_mf(const MixedArgs& a, int precision, int64_t q, const void* Aq_lo, void* part, double* v,
                             double* d64, float* t32, cudaStream_t s);

// ---- randomized inner chains (randomized.cu) ----------------------------------------------
struct RandArgs {
  int64_t n, k, m, p;
  const double* A;        // the handle's copy of A, m x n, ld m (A_1 = rows 0..p-1)
  const double* G1;       // Abar1
  const double* norms2;   // ||A_1(:,j)||^2
  const double* inv_norms2;  // 1 / ||A_1(:,j)||^2 (dense handles)
  const double* cum;      // running sum of norms2, left to right
  const double* bhat;     // n x k
  double* X0;
  double* X1;
  const int32_t* col_done;
  const double* col_target2;
  int64_t* col_inner;
  SolveState* st;
  uint64_t seed;
  int64_t chain0;         // chain id of column 0 of this pass
  int64_t max_inner;
  int64_t check_every;
  int32_t greedy;         // SCD: alpha = n
  int32_t same_index;     // RK-RGS: j2 = j1 (the SP-RCD special case)
  int32_t vec_in_smem;    // RK-RGS: w, e in shared memory
  int32_t correction;     // bhat holds r = bbar - H x_k; the chain solves Abar1 d = r from d = 0
                          // and x_k += d in place (sparse RK-RGS in FP32, and the warm inner
                          // start of the dense chains: the start z = x_k of Alg. 2 / beta = x_k of
                          // Alg. 5 in correction form)
  double* vec_scratch;    // RK-RGS: k x 2p when not in shared memory
  int64_t alpha_fixed;    // SCD: 0 = alpha ~ U{1..n} (Alg. 5); else the fixed subset size
  int32_t gram_form;      // dense RK-RGS: Gram-space steps (g = Abar1 y, h = Abar1 z)
  int32_t alias;          // RK-RGS: column draws from the alias table below
  const double* alias_prob;  // n: acceptance probability of column j
  const int32_t* alias_idx;  // n: alias of column j
  int32_t* picks;         // diagnostic: chain 0's picks in outer iteration 0 (or nullptr)
  int64_t picks_cap;
  unsigned long long* inner_ns;  // accumulated device time of chain 0's launches (or nullptr)
};
// Vose alias table of the column law norms2 / sum(norms2) (n <= 16384), one CTA.
cudaError_t alias_table_f64(int64_t n, const double* norms2, double* prob, int32_t* alias, cudaStream_t s);
// Sparse A: column-sorted CSC of all of A; split[j] = entries of column j in rows < p.
struct SparseCols {
  int32_t* colptr;  // n + 1
  int32_t* rowind;  // nnz
  double* val;      // nnz
  float* val32;     // nnz (FP32 copy, mixed precision only; else nullptr)
  int32_t* split;   // n
  // SP-RK-RGS on a thread-block cluster of cs CTAs (cs = 0: one CTA, vectors in global memory)
  int32_t* seg;         // n x (cs + 1): CTA r's entries of column j are seg[j(cs+1)+r] .. seg[j(cs+1)+r+1]-1
  double* inv_norms2;   // n: 1 / ||A_1(:,j)||^2
  void* G1c;            // Abar1 in the chain's precision, leading dimension ldg (16-byte columns)
  int32_t cs;
  int32_t slice;        // rows of A_1 per CTA
  int32_t nres;         // entries of s = bhat - Abar1 z per CTA
  int32_t ldg;
};
cudaError_t sparse_setup(int64_t m, int64_t n, int64_t p, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                         const double* val, SparseCols sc, int32_t* cnt_fill, double* G1, double* G2, int32_t* err,
                         cudaStream_t s);
cudaError_t sparse_rhs_bar(int64_t n, int64_t p, int64_t k, SparseCols sc, const double* B, int64_t ldb, double* out,
                           int64_t ldo, cudaStream_t s);
cudaError_t rkrgs_sparse_chain(const RandArgs& a, SparseCols sc, bool fp32, cudaStream_t s);
// Cluster size for the sparse RK-RGS chain (0 when none fits); *slice = rows of A_1 per CTA.
// want = 0: the smallest size that fits and leaves about col_entries / cs <= 112 entries
// of a column per CTA; else only that size is tried.
int rkrgs_cluster_plan(int64_t n, int64_t p, bool fp32, int want, double col_entries, int32_t* slice,
                       int32_t* nres);
// After the Grams and column norms: the per-CTA column segments, 1/||A_1(:,j)||^2 and the
// padded copy of Abar1 the cluster chain reads.
cudaError_t sparse_chain_prep(int64_t n, SparseCols sc, const double* G1, const double* norms2, bool fp32,
                              cudaStream_t s);

// ---- route choice (route_tune.cu) ------------------------------------------------------------
// Matrix-free or explicit for an SP problem with q rows of A_2 and n columns, by the cost
// model of route_tune.cu with rates measured once per process (synchronizes on first use).
// model (host, may be null) receives 8 values: the explicit and matrix-free costs in seconds,
// the split and FP64 Gram rates (flop/s), the FP64/FP32/BF16 stream rates and the copy rate (B/s).
cudaError_t route_prefers_matrix_free(int64_t q, int64_t n, int precision, bool split_gram, int estimate_steps,
                                      bool* mf, double* model);

// ---- Lanczos estimates (lanczos.cu) -----------------------------------------------------------
// Extreme eigenvalues of C = M2 M1 in the M1 inner product (M1 == nullptr: standard Lanczos on
// the symmetric M2).  M2, M1: n x n symmetric, FP64 (f64 != 0) or FP32.  out (device):
// [0] smallest, [1] largest Ritz value after `steps` steps (<= 256), [2] steps taken.
struct LanczosProblem {
  int64_t n;
  const void* M2;
  const void* M1;
  int32_t m2_f64, m1_f64;
  int32_t steps;
  int32_t pad;
  double* out;
};
// Up to four problems of equal n in one launch, one thread-block cluster each.
cudaError_t lanczos_extremes(int count, const LanczosProblem* probs, cudaStream_t s);
// est[0..7] (see the handle) from the outputs of the kappa (H) and rho problems (either may be null).
// est[7] (status) must be 0 before the first call of a setup; later calls keep a failure.
cudaError_t estimates_finish(const double* kap_out, const double* rho_out, double* est, cudaStream_t s,
                             bool gram_bound = false);
// Matrix-free rho: Lanczos on (A_2^T A_2) P in the P inner product, P FP32 (n <= 512).  w holds
// lz_mf_work_floats(n) floats; lz_mf_vector(n, w) is the FP64 vector t_j whose product
// y = A_2^T (A_2 t_j) each lz_mf_step(j) consumes; lz_mf_finish writes out[0..2] like
// lanczos_extremes.
size_t lz_mf_work_floats(int64_t n);
cudaError_t lz_mf_init(int64_t n, const float* P, float* w, cudaStream_t s);
double* lz_mf_vector(int64_t n, float* w);
cudaError_t lz_mf_step(int64_t n, const float* P, const double* y, float* w, int j, cudaStream_t s);
cudaError_t lz_mf_finish(int64_t n, float* w, double* out, cudaStream_t s);

// norms2 = diag(Abar1), cum its running sum (left to right), inv_norms2 = 1 / norms2 (may be null).
cudaError_t column_cumsum_f64(int64_t n, const double* G1, double* norms2, double* cum, cudaStream_t s,
                              double* inv_norms2 = nullptr);
cudaError_t rand_chain_f64(const RandArgs& a, int method, cudaStream_t s);
bool rkrgs_vec_fits(int64_t n, int64_t p);

}  // namespace ils
