// Dense FP64 kernels of the SP path: Gram products, A^T J b, Cholesky, triangular
// solves and the SP outer step.  On GB300 FP64 fused multiply-adds issue at about
// 2 per clock per SM (64x below FP32), so every kernel here is FP64-ALU bound and is
// shaped to spread its multiply-adds evenly over all 152 SMs rather than to save
// bandwidth.
#include <algorithm>

#include "ils_internal.h"

namespace ils {
namespace {

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
// C = X^T Y (Gram / GEMM-TN), 64 x 64 output tiles, 16-row k-steps, optional split over K.
// ---------------------------------------------------------------------------------------
constexpr int kTM = 64;
constexpr int kTK = 16;
constexpr int kGemmThreads = 256;

__global__ void __launch_bounds__(kGemmThreads)
gemm_tn_kernel(int64_t K, int64_t n1, int64_t n2, const double* __restrict__ X, int64_t ldx,
               const double* __restrict__ Y, int64_t ldy, int64_t sign_split,
               double* __restrict__ out, int64_t ldo, int sym, int trans_out, int64_t chunk,
               int partial) {
  const int bi = blockIdx.x, bj = blockIdx.y, sidx = blockIdx.z;
  if (sym && bi > bj) return;
  const int64_t i0 = (int64_t)bi * kTM, j0 = (int64_t)bj * kTM;
  const int64_t r_begin = (int64_t)sidx * chunk;
  const int64_t r_end = min(K, r_begin + chunk);
  __shared__ double Xs[kTK][kTM];
  __shared__ double Ys[kTK][kTM];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int lk = tid % kTK, lc = tid / kTK;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTK) {
    const int64_t r = r0 + lk;
    const bool rin = r < r_end;
    const double sg = (r >= sign_split) ? -1.0 : 1.0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int c = lc + 16 * l;
      const int64_t gi = i0 + c, gj = j0 + c;
      Xs[lk][c] = (rin && gi < n1) ? X[r + gi * ldx] : 0.0;
      Ys[lk][c] = (rin && gj < n2) ? sg * Y[r + gj * ldy] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      double xa[4], yb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xa[a] = Xs[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yb[b] = Ys[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
      if (gi >= n1 || gj >= n2) continue;
      if (sym && gi > gj) continue;
      if (partial) {
        out[(size_t)sidx * n1 * n2 + gi + gj * n1] = acc[a][b];
      } else {
        if (trans_out) out[gj + gi * ldo] = acc[a][b];
        else out[gi + gj * ldo] = acc[a][b];
        if (sym && gi != gj) out[gj + gi * ldo] = acc[a][b];
      }
    }
  }
}

__global__ void gemm_reduce_kernel(int64_t n1, int64_t n2, int splits, const double* __restrict__ work,
                                   double* __restrict__ out, int64_t ldo, int sym, int trans_out) {
  const int64_t total = n1 * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = e % n1, gj = e / n1;
    if (sym && gi > gj) continue;
    double v = 0.0;
    for (int s = 0; s < splits; ++s) v += work[(size_t)s * total + e];
    if (trans_out) out[gj + gi * ldo] = v;
    else out[gi + gj * ldo] = v;
    if (sym && gi != gj) out[gj + gi * ldo] = v;
  }
}

void gemm_plan(int64_t K, int64_t n1, int64_t n2, bool sym, int* splits, int64_t* chunk) {
  const int64_t nb1 = (n1 + kTM - 1) / kTM, nb2 = (n2 + kTM - 1) / kTM;
  const int64_t tiles = sym ? nb1 * (nb1 + 1) / 2 : nb1 * nb2;
  const int64_t target = 2 * (int64_t)num_sms();
  int64_t s = (target + tiles - 1) / tiles;
  const int64_t max_s = std::max<int64_t>(1, K / 256);
  s = std::max<int64_t>(1, std::min(s, max_s));
  int64_t ch = (K + s - 1) / s;
  ch = ((ch + kTK - 1) / kTK) * kTK;
  if (ch <= 0) ch = kTK;
  s = (K + ch - 1) / ch;
  if (s < 1) s = 1;
  *splits = (int)s;
  *chunk = ch;
}

// ---------------------------------------------------------------------------------------
// A^T J B for a few right-hand sides: one CTA per column of A.
// ---------------------------------------------------------------------------------------
constexpr int kRhsThreads = 256;

__global__ void __launch_bounds__(kRhsThreads)
rhs_bar_kernel(int64_t m, int64_t n, int64_t p, int64_t k, const double* __restrict__ A, int64_t lda,
               const double* __restrict__ B, int64_t ldb, double* __restrict__ out, int64_t ldo) {
  const int64_t j = blockIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * kMaxRhsPerPass;
  const int kk = (int)((k - c0) < kMaxRhsPerPass ? (k - c0) : kMaxRhsPerPass);
  double acc[kMaxRhsPerPass];
#pragma unroll
  for (int c = 0; c < kMaxRhsPerPass; ++c) acc[c] = 0.0;
  const double* col = A + j * lda;
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
    const double a = (r < p) ? col[r] : -col[r];
#pragma unroll
    for (int c = 0; c < kMaxRhsPerPass; ++c)
      if (c < kk) acc[c] = fma(a, B[r + (c0 + c) * ldb], acc[c]);
  }
  __shared__ double red[kRhsThreads / 32][kMaxRhsPerPass];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kMaxRhsPerPass; ++c) {
    const double v = warp_sum(acc[c]);
    if (lane == 0) red[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kk) {
    double v = 0.0;
    for (int ww = 0; ww < kRhsThreads / 32; ++ww) v += red[ww][threadIdx.x];
    out[j + (c0 + threadIdx.x) * ldo] = v;
  }
}

// Y(:,c) = M^T X(:,c): warp i reduces column i of M against each right-hand side.
constexpr int kGemvWarps = 2;

__global__ void __launch_bounds__(32 * kGemvWarps)
gemv_cols_kernel(int64_t n, int64_t k, const double* __restrict__ M, int64_t ldm,
                 const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * kGemvWarps + w; i < n; i += (int64_t)gridDim.x * kGemvWarps) {
    const double* col = M + i * ldm;
    for (int64_t c0 = 0; c0 < k; c0 += kMaxRhsPerPass) {
      const int kk = (int)((k - c0) < kMaxRhsPerPass ? (k - c0) : kMaxRhsPerPass);
      double acc[kMaxRhsPerPass];
#pragma unroll
      for (int c = 0; c < kMaxRhsPerPass; ++c) acc[c] = 0.0;
      for (int64_t j = lane; j < n; j += 32) {
        const double mv = col[j];
#pragma unroll
        for (int c = 0; c < kMaxRhsPerPass; ++c)
          if (c < kk) acc[c] = fma(mv, X[j + (c0 + c) * ldx], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < kMaxRhsPerPass; ++c) {
        const double v = warp_sum(acc[c]);
        if (lane == 0 && c < kk) Y[i + (c0 + c) * ldy] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Blocked right-looking Cholesky, 32-wide panels.
// ---------------------------------------------------------------------------------------
constexpr int kNB = 32;

__device__ void set_status(int32_t* status, int32_t code) { atomicCAS(status, 0, code); }

__global__ void __launch_bounds__(1024)
potrf_diag_kernel(int64_t n, double* __restrict__ L, int64_t k0, int nb, int32_t* status) {
  __shared__ double s[kNB][kNB + 1];
  const int i = threadIdx.y, j = threadIdx.x;
  s[i][j] = (i < nb && j < nb) ? L[(k0 + i) + (k0 + j) * n] : (i == j ? 1.0 : 0.0);
  for (int c = 0; c < nb; ++c) {
    __syncthreads();
    if (i == c && j == c) {
      double d = s[c][c];
      if (!isfinite(d)) {
        set_status(status, ILS_ERR_NONFINITE);
        d = 1.0;
      } else if (!(d > 0.0)) {
        set_status(status, ILS_ERR_NOT_SPD);
        d = 1.0;
      }
      s[c][c] = sqrt(d);
    }
    __syncthreads();
    if (j == c && i > c) s[i][c] /= s[c][c];
    __syncthreads();
    if (j > c && i >= j) s[i][j] = fma(-s[i][c], s[j][c], s[i][j]);
  }
  __syncthreads();
  if (i < nb && j < nb && i >= j) L[(k0 + i) + (k0 + j) * n] = s[i][j];
}

// Rows below the diagonal block: L21 = A21 L11^{-T}, one thread per row.
__global__ void __launch_bounds__(128)
trsm_panel_kernel(int64_t n, double* __restrict__ L, int64_t k0, int nb) {
  __shared__ double l11[kNB][kNB + 1];
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int a = e % kNB, b = e / kNB;
    l11[a][b] = (a < nb && b < nb && a >= b) ? L[(k0 + a) + (k0 + b) * n] : 0.0;
  }
  __syncthreads();
  const int64_t i = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) x[c] = (c < nb) ? L[i + (k0 + c) * n] : 0.0;
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    if (c < nb) {
      double v = x[c];
#pragma unroll
      for (int d = 0; d < kNB; ++d)
        if (d < c) v = fma(-x[d], l11[c][d], v);
      x[c] = v / l11[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    if (c < nb) L[i + (k0 + c) * n] = x[c];
}

// Trailing update A22 -= L21 L21^T on lower 32 x 32 tiles.
__global__ void __launch_bounds__(256)
syrk_trailing_kernel(int64_t n, double* __restrict__ L, int64_t k0, int nb) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bi < bj) return;
  const int64_t k1 = k0 + nb;
  const int64_t ri0 = k1 + (int64_t)bi * kNB, rj0 = k1 + (int64_t)bj * kNB;
  __shared__ double Pi[kNB][kNB + 1];
  __shared__ double Pj[kNB][kNB + 1];
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e % kNB, c = e / kNB;
    Pi[r][c] = (ri0 + r < n && c < nb) ? L[(ri0 + r) + (k0 + c) * n] : 0.0;
    Pj[r][c] = (rj0 + r < n && c < nb) ? L[(rj0 + r) + (k0 + c) * n] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = 0; c < nb; ++c) {
    const double pj = Pj[tx][c];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = fma(Pi[ty + 8 * a][c], pj, acc[a]);
  }
  const int64_t gj = rj0 + tx;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t gi = ri0 + ty + 8 * a;
    if (gi < n && gj < n && gi >= gj) L[gi + gj * n] -= acc[a];
  }
}

// ---------------------------------------------------------------------------------------
// Triangular solves with many right-hand sides: one warp per right-hand side,
// the vector kept in shared memory.
// ---------------------------------------------------------------------------------------
constexpr int kTrsmWarps = 4;

__global__ void __launch_bounds__(32 * kTrsmWarps)
trsm_kernel(int64_t n, int64_t k, const double* __restrict__ L, double* __restrict__ X, int64_t ldx,
            int fwd, int bwd) {
  extern __shared__ double smem_y[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * kTrsmWarps + w;
  if (col >= k) return;
  double* y = smem_y + (size_t)w * n;
  double* xc = X + col * ldx;
  for (int64_t r = lane; r < n; r += 32) y[r] = xc[r];
  __syncwarp();
  if (fwd) {
    for (int64_t i = 0; i < n; ++i) {
      const double yi = y[i] / L[i + i * n];
      __syncwarp();
      if (lane == 0) y[i] = yi;
      const double* li = L + i * n;
      for (int64_t r = i + 1 + lane; r < n; r += 32) y[r] = fma(-li[r], yi, y[r]);
      __syncwarp();
    }
  }
  if (bwd) {
    for (int64_t i = n - 1; i >= 0; --i) {
      const double* li = L + i * n;
      double s = 0.0;
      for (int64_t r = i + 1 + lane; r < n; r += 32) s = fma(li[r], y[r], s);
      s = warp_sum(s);
      if (lane == 0) y[i] = (y[i] - s) / li[i];
      __syncwarp();
    }
  }
  for (int64_t r = lane; r < n; r += 32) xc[r] = y[r];
}

__global__ void set_identity_kernel(int64_t n, double* M, int64_t ld) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    M[i + j * ld] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void axpby_kernel(int64_t total, double alpha, const double* X, double beta, const double* Y,
                             double* Z) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    Z[e] = alpha * X[e] + beta * Y[e];
}

__global__ void copy_lower_kernel(int64_t n, const double* L, double* D, int64_t ldd) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    D[i + j * ldd] = (i >= j) ? L[i + j * n] : 0.0;
  }
}

__global__ void sq_norms_kernel(int64_t n, int64_t k, const double* X, int64_t ldx, double* out) {
  const int64_t c = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = X[r + c * ldx];
    s = fma(v, v, s);
  }
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[c] = t;
  }
}

// ---------------------------------------------------------------------------------------
// SP outer step.  Each launch, for every unfinished column c:
//   r_k = bbar - H x_k (the residual of Sec. 5's stopping test, on x_k),
//   x_{k+1} = B x_k + c (Alg. 1 step 6),
// with x_k and x_{k+1} in two ping-pong buffers.  The last CTA to arrive sums the
// per-CTA ||r_k||^2 partials and decides: a column whose residual passes the test (or
// that reached max_outer, or went non-finite) is finished with x_k; when every column
// is finished the solve is done and later launches return at once.
// ---------------------------------------------------------------------------------------
constexpr int kIterWarps = 2;

__global__ void __launch_bounds__(32 * kIterWarps) sp_iter_kernel(SpIterArgs a) {
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done)) return;
  const int cur = *((volatile int32_t*)&st->cur);
  const double* __restrict__ x = cur ? a.X1 : a.X0;
  double* __restrict__ xn = cur ? a.X0 : a.X1;
  const int64_t n = a.n;
  const int k = (int)a.k;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ int32_t done_c[kMaxRhsPerPass];
  if (threadIdx.x < kMaxRhsPerPass) done_c[threadIdx.x] = (threadIdx.x < k) ? a.col_done[threadIdx.x] : 1;
  __syncthreads();
  double rpart[kMaxRhsPerPass];
#pragma unroll
  for (int c = 0; c < kMaxRhsPerPass; ++c) rpart[c] = 0.0;

  for (int64_t i = (int64_t)blockIdx.x * kIterWarps + w; i < n; i += (int64_t)gridDim.x * kIterWarps) {
    const double* brow = a.Bt + i * n;
    const double* hrow = a.H + i * n;
    double ab[kMaxRhsPerPass], ah[kMaxRhsPerPass];
#pragma unroll
    for (int c = 0; c < kMaxRhsPerPass; ++c) ab[c] = ah[c] = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
      const double bv = brow[j], hv = hrow[j];
#pragma unroll
      for (int c = 0; c < kMaxRhsPerPass; ++c) {
        if (c < k) {
          const double xv = x[j + c * n];
          ab[c] = fma(bv, xv, ab[c]);
          ah[c] = fma(hv, xv, ah[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kMaxRhsPerPass; ++c) {
      const double sb = warp_sum(ab[c]);
      const double sh = warp_sum(ah[c]);
      if (lane == 0 && c < k) {
        if (done_c[c]) {
          xn[i + c * n] = x[i + c * n];
        } else {
          if (a.mode == 0) xn[i + c * n] = sb + a.cvec[i + c * n];
          else a.bhat_out[i + c * n] = sb + a.cvec[i + c * n];
          const double r = a.bbar[i + c * n] - sh;
          rpart[c] = fma(r, r, rpart[c]);
        }
      }
    }
  }
  __shared__ double red[kIterWarps][kMaxRhsPerPass];
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < kMaxRhsPerPass; ++c) red[w][c] = rpart[c];
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double v = 0.0;
    for (int ww = 0; ww < kIterWarps; ++ww) v += red[ww][threadIdx.x];
    a.partials[(int64_t)blockIdx.x * k + threadIdx.x] = v;
  }
  __threadfence();
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ int32_t newly_done[kMaxRhsPerPass];
  __shared__ int all_done;
  if (threadIdx.x == 0) {
    int all = 1;
    const int64_t it = st->iters;
    for (int c = 0; c < k; ++c) {
      newly_done[c] = 0;
      if (done_c[c]) continue;
      double rr = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) rr += __ldcg(&a.partials[(int64_t)b * k + c]);
      const bool finite = isfinite(rr);
      const bool conv = finite && rr <= a.tol2 * a.bnorm2[c];
      if (!finite || conv || it >= st->max_outer) {
        a.col_done[c] = 1;
        a.col_rr[c] = rr;
        a.col_iters[c] = it;
        newly_done[c] = 1;
        if (!finite) atomicCAS(&st->status, 0, ILS_ERR_NONFINITE);
        else if (!conv) atomicCAS(&st->status, 0, ILS_ERR_NO_CONVERGENCE);
      } else {
        all = 0;
        if (a.mode == 1) a.col_target2[c] = a.theta2 * rr;
      }
    }
    all_done = all;
    if (all) {
      st->done = 1;  // the answer of every column is in buffer `cur`
    } else {
      st->cur = cur ^ 1;
      st->iters = it + 1;
    }
    st->counter = 0u;
  }
  __syncthreads();
  if (!all_done) {
    // Columns that finished now keep x_k: copy it over the x_{k+1} just written.
    for (int c = 0; c < k; ++c) {
      if (!newly_done[c]) continue;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xn[i + c * n] = x[i + c * n];
    }
  }
}

__global__ void copy_final_kernel(int64_t n, int64_t k, const double* X0, const double* X1,
                                  const SolveState* st, double* X, int64_t ldx) {
  const double* src = st->cur ? X1 : X0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, c = e / n;
    X[i + c * ldx] = src[i + c * n];
  }
}

int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  const int64_t cap = 8 * (int64_t)num_sms();
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------
size_t gemm_tn_work_elems(int64_t K, int64_t n1, int64_t n2, bool sym, int* splits_out) {
  int splits;
  int64_t chunk;
  gemm_plan(K, n1, n2, sym, &splits, &chunk);
  if (splits_out) *splits_out = splits;
  return splits > 1 ? (size_t)splits * (size_t)n1 * (size_t)n2 : 0;
}

cudaError_t gemm_tn_f64(int64_t K, int64_t n1, int64_t n2, const double* X, int64_t ldx, const double* Y,
                        int64_t ldy, int64_t sign_split, double* C, int64_t ldc, bool sym, bool trans_out,
                        double* work, cudaStream_t s) {
  if (n1 <= 0 || n2 <= 0) return cudaSuccess;
  if (K <= 0) {
    // Empty block (for example q = 0): the product is the zero matrix.
    if (trans_out) return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * n2, n1, s);
    return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * n1, n2, s);
  }
  int splits;
  int64_t chunk;
  gemm_plan(K, n1, n2, sym, &splits, &chunk);
  dim3 grid((unsigned)((n1 + kTM - 1) / kTM), (unsigned)((n2 + kTM - 1) / kTM), (unsigned)splits);
  const bool partial = splits > 1;
  gemm_tn_kernel<<<grid, kGemmThreads, 0, s>>>(K, n1, n2, X, ldx, Y, ldy, sign_split, partial ? work : C,
                                                ldc, sym ? 1 : 0, trans_out ? 1 : 0, chunk, partial ? 1 : 0);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !partial) return e;
  gemm_reduce_kernel<<<grid_for(n1 * n2, 256), 256, 0, s>>>(n1, n2, splits, work, C, ldc, sym ? 1 : 0,
                                                            trans_out ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gemm_tn_f64_capped(int64_t K, int64_t n, const double* X, int64_t ldx, double* C, int64_t ldc,
                               double* work, size_t work_cap_elems, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (K <= 0) return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * n, n, s);
  int splits;
  int64_t chunk;
  gemm_plan(K, n, n, true, &splits, &chunk);
  const int64_t cap = (int64_t)(work_cap_elems / ((size_t)n * (size_t)n));
  if (splits > 1 && splits > cap) {
    // Fewer, longer K slices so the partial sums fit in the caller's scratch.
    const int64_t sp = std::max<int64_t>(1, cap);
    chunk = ((K + sp - 1) / sp + kTK - 1) / kTK * kTK;
    splits = (int)((K + chunk - 1) / chunk);
  }
  dim3 grid((unsigned)((n + kTM - 1) / kTM), (unsigned)((n + kTM - 1) / kTM), (unsigned)splits);
  const bool partial = splits > 1;
  gemm_tn_kernel<<<grid, kGemmThreads, 0, s>>>(K, n, n, X, ldx, X, ldx, K, partial ? work : C, ldc, 1, 0, chunk,
                                                partial ? 1 : 0);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !partial) return e;
  gemm_reduce_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(n, n, splits, work, C, ldc, 1, 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t rhs_bar_f64(int64_t m, int64_t n, int64_t p, int64_t k, const double* A, int64_t lda, const double* B,
                        int64_t ldb, double* out, int64_t ldo, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  dim3 grid((unsigned)n, (unsigned)((k + kMaxRhsPerPass - 1) / kMaxRhsPerPass));
  rhs_bar_kernel<<<grid, kRhsThreads, 0, s>>>(m, n, p, k, A, lda, B, ldb, out, ldo);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gemv_cols_f64(int64_t n, int64_t k, const double* M, int64_t ldm, const double* X, int64_t ldx,
                          double* Y, int64_t ldy, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + kGemvWarps - 1) / kGemvWarps, 16 * (int64_t)num_sms());
  gemv_cols_kernel<<<blocks, 32 * kGemvWarps, 0, s>>>(n, k, M, ldm, X, ldx, Y, ldy);
  note_launch();
  return cudaGetLastError();
}

cudaError_t cholesky_f64(int64_t n, double* L, int32_t* status, cudaStream_t s) {
  for (int64_t k0 = 0; k0 < n; k0 += kNB) {
    const int nb = (int)std::min<int64_t>(kNB, n - k0);
    potrf_diag_kernel<<<1, dim3(kNB, kNB), 0, s>>>(n, L, k0, nb, status);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t rest = n - k0 - nb;
    if (rest <= 0) break;
    trsm_panel_kernel<<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(n, L, k0, nb);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned nt = (unsigned)((rest + kNB - 1) / kNB);
    syrk_trailing_kernel<<<dim3(nt, nt), 256, 0, s>>>(n, L, k0, nb);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t trsm_lower_f64(int64_t n, int64_t k, const double* L, double* X, int64_t ldx, bool forward,
                           bool backward, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * (size_t)n * kTrsmWarps;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  trsm_kernel<<<(unsigned)((k + kTrsmWarps - 1) / kTrsmWarps), 32 * kTrsmWarps, smem, s>>>(
      n, k, L, X, ldx, forward ? 1 : 0, backward ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_identity_f64(int64_t n, double* M, int64_t ld, cudaStream_t s) {
  set_identity_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(n, M, ld);
  note_launch();
  return cudaGetLastError();
}

cudaError_t axpby_mat_f64(int64_t n, double alpha, const double* X, double beta, const double* Y, double* Z,
                          cudaStream_t s) {
  axpby_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(n * n, alpha, X, beta, Y, Z);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_lower_zero_upper_f64(int64_t n, const double* L, double* dst, int64_t ldd, cudaStream_t s) {
  copy_lower_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(n, L, dst, ldd);
  note_launch();
  return cudaGetLastError();
}

cudaError_t sq_norms_cols_f64(int64_t n, int64_t k, const double* X, int64_t ldx, double* out, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  sq_norms_kernel<<<(unsigned)k, 256, 0, s>>>(n, k, X, ldx, out);
  note_launch();
  return cudaGetLastError();
}

int sp_iterate_blocks(int64_t n) {
  const int64_t want = (n + kIterWarps - 1) / kIterWarps;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 4 * (int64_t)num_sms()));
}

cudaError_t sp_iterate_f64(const SpIterArgs& a, cudaStream_t s) {
  sp_iter_kernel<<<sp_iterate_blocks(a.n), 32 * kIterWarps, 0, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_final_f64(int64_t n, int64_t k, const double* X0, const double* X1, const SolveState* st,
                           double* X, int64_t ldx, cudaStream_t s) {
  copy_final_kernel<<<grid_for(n * k, 256), 256, 0, s>>>(n, k, X0, X1, st, X, ldx);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
