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

// out(:,c) = A^T J b(:,c) for k right-hand sides: A m x n (lda), B m x k (ldb),
// rows >= p carry the minus sign of J.  out is n x k (ldo).
cudaError_t rhs_bar_f64(int64_t m, int64_t n, int64_t p, int64_t k, const double* A, int64_t lda,
                        const double* B, int64_t ldb, double* out, int64_t ldo, cudaStream_t s);

// Y(:,c) = M^T X(:,c) for an n x n column-major M (so row i of M^T is column i of M).
cudaError_t gemv_cols_f64(int64_t n, int64_t k, const double* M, int64_t ldm, const double* X,
                          int64_t ldx, double* Y, int64_t ldy, cudaStream_t s);

// In-place blocked Cholesky of the lower triangle of the n x n matrix L (ld n).
// status (device int) is set to ILS_ERR_NOT_SPD or ILS_ERR_NONFINITE on a bad pivot.
cudaError_t cholesky_f64(int64_t n, double* L, int32_t* status, cudaStream_t s);

// X := L^{-1} X (lower = forward) then, if both, X := L^{-T} X.  X n x k (ldx).
cudaError_t trsm_lower_f64(int64_t n, int64_t k, const double* L, double* X, int64_t ldx,
                           bool forward, bool backward, cudaStream_t s);

// Elementwise helpers.
cudaError_t set_identity_f64(int64_t n, double* M, int64_t ld, cudaStream_t s);
cudaError_t axpby_mat_f64(int64_t n, double alpha, const double* X, double beta, const double* Y,
                          double* Z, cudaStream_t s);  // Z = alpha X + beta Y, n*n contiguous
cudaError_t copy_lower_zero_upper_f64(int64_t n, const double* L, double* dst, int64_t ldd,
                                      cudaStream_t s);
cudaError_t sq_norms_cols_f64(int64_t n, int64_t k, const double* X, int64_t ldx, double* out,
                              cudaStream_t s);

// One SP outer step for up to kMaxRhsPerPass columns (Alg. 1 step 6 with the residual
// test of Sec. 5 on x_k).  See dense_f64.cu for the protocol.
struct SpIterArgs {
  int64_t n, k;
  const double* Bt;    // B^T, column-major n x n: column i = row i of B
  const double* H;     // A^T J A (symmetric)
  const double* cvec;  // n x k
  const double* bbar;  // n x k
  const double* bnorm2;  // k
  double* X0;          // n x k iterate buffers
  double* X1;
  double tol2;         // tol^2
  int32_t* col_done;   // k flags
  double* col_rr;      // k: ||r||^2 of each column's returned iterate
  int64_t* col_iters;  // k
  double* partials;    // gridDim x k
  SolveState* st;
};
cudaError_t sp_iterate_f64(const SpIterArgs& a, cudaStream_t s);
int sp_iterate_blocks(int64_t n);

// Copy the final iterate buffer (chosen on the device) into the user's X.
cudaError_t copy_final_f64(int64_t n, int64_t k, const double* X0, const double* X1,
                           const SolveState* st, double* X, int64_t ldx, cudaStream_t s);

}  // namespace ils
