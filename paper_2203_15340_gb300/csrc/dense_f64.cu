// Dense FP64 kernels of the SP path: Gram products, A^T J b, Cholesky, triangular
// solves and the SP outer step.  On GB300 FP64 fused multiply-adds issue at about
// 2 per clock per SM (64x below FP32), so every kernel here is FP64-ALU bound and is
// shaped to spread its multiply-adds evenly over all 152 SMs rather than to save
// bandwidth.
#include <algorithm>
#include <cmath>

#include <type_traits>

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

// dst[e] = src(e) for e in [tid, total) stepping by nthr, with 8 loads in flight per thread
// (a plain load-store loop would wait one L2 round trip per element).
template <typename T, typename F>
__device__ __forceinline__ void batched_copy(T* dst, int64_t total, int tid, int nthr, F src) {
  int64_t e = tid;
  for (; e + 7 * (int64_t)nthr < total; e += 8 * (int64_t)nthr) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = src(e + u * (int64_t)nthr);
#pragma unroll
    for (int u = 0; u < 8; ++u) dst[e + u * (int64_t)nthr] = v[u];
  }
  for (; e < total; e += nthr) dst[e] = src(e);
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
    const int64_t gi = (uint32_t)e % (uint32_t)n1, gj = (uint32_t)e / (uint32_t)n1;  // n1 * n2 < 2^31
    if (sym && gi > gj) continue;
    double v = 0.0;
    for (int s = 0; s < splits; ++s) v += work[(size_t)s * total + e];
    if (trans_out) out[gj + gi * ldo] = v;
    else out[gi + gj * ldo] = v;
    if (sym && gi != gj) out[gj + gi * ldo] = v;
  }
}

// K-split of the GEMM grid.  The kernel is FP64-issue bound, so the split is chosen to
// give every one of the SMs the same number of CTAs (ties: fewer slices), with at least
// two CTAs per SM and at least 64 K rows per slice.
void gemm_plan(int64_t K, int64_t n1, int64_t n2, bool sym, int* splits, int64_t* chunk) {
  const int64_t nb1 = (n1 + kTM - 1) / kTM, nb2 = (n2 + kTM - 1) / kTM;
  const int64_t tiles = sym ? nb1 * (nb1 + 1) / 2 : nb1 * nb2;
  const int64_t sms = num_sms();
  const int64_t s_min = std::max<int64_t>(1, (2 * sms + tiles - 1) / tiles);
  const int64_t s_max = std::max<int64_t>(1, std::min<int64_t>(32, K / 64));
  int64_t best_s = 1, best_ch = ((K + kTK - 1) / kTK) * kTK;
  double best_eff = -1.0;
  for (int64_t s = std::min(s_min, s_max); s <= s_max; ++s) {
    int64_t ch = ((K + s - 1) / s + kTK - 1) / kTK * kTK;
    if (ch <= 0) ch = kTK;
    const int64_t se = (K + ch - 1) / ch;
    const int64_t ctas = tiles * se;
    const double waves = (double)ctas / (double)sms;
    const double eff = waves / std::ceil(waves);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best_s = se;
      best_ch = ch;
    }
    if (eff >= 0.98) break;
  }
  *splits = (int)best_s;
  *chunk = best_ch;
}

// ---------------------------------------------------------------------------------------
// A^T J B for a few right-hand sides: one CTA per column of A.
// ---------------------------------------------------------------------------------------
constexpr int kRhsThreads = 256;

template <int KR>
__global__ void __launch_bounds__(kRhsThreads)
rhs_bar_kernel(int64_t m, int64_t n, int64_t p, int64_t k, const double* __restrict__ A, int64_t lda,
               const double* __restrict__ B, int64_t ldb, double* __restrict__ out, int64_t ldo) {
  const int64_t j = blockIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * kMaxRhsPerPass;
  // Four interleaved partial sums per right-hand side keep FP64 latency (64 cycles per
  // dependent FMA) and the loads overlapped.
  double acc[KR][4];
#pragma unroll
  for (int c = 0; c < KR; ++c)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[c][u] = 0.0;
  const double* col = A + j * lda;
  const int64_t stride = blockDim.x;
  // Rows of A_1 add, rows of A_2 subtract: two passes with the sign fixed at compile time,
  // so it folds into the FMA instead of costing an FP64 negation per element.
  auto pass = [&](int64_t r0, int64_t r1, auto neg) {
    int64_t r = r0 + threadIdx.x;
    for (; r + 3 * stride < r1; r += 4 * stride) {
      double av[4], bv[KR][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = col[r + u * stride];
#pragma unroll
        for (int c = 0; c < KR; ++c) bv[c][u] = B[r + u * stride + c * ldb];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < KR; ++c) acc[c][u] = fma(decltype(neg)::value ? -av[u] : av[u], bv[c][u], acc[c][u]);
    }
    for (; r < r1; r += stride) {
      const double a = col[r];
#pragma unroll
      for (int c = 0; c < KR; ++c) acc[c][0] = fma(decltype(neg)::value ? -a : a, B[r + c * ldb], acc[c][0]);
    }
  };
  pass(0, p, std::false_type{});
  pass(p, m, std::true_type{});
  __shared__ double red[kRhsThreads / 32][kMaxRhsPerPass];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < KR; ++c) {
    const double v = warp_sum((acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3]));
    if (lane == 0) red[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < KR) {
    double v = 0.0;
    for (int ww = 0; ww < kRhsThreads / 32; ++ww) v += red[ww][threadIdx.x];
    out[j + (c0 + threadIdx.x) * ldo] = v;
  }
}

// Y(:,c) = M^T X(:,c): warp i reduces column i of M against each right-hand side.
constexpr int kGemvWarps = 2;

template <int KR>
__global__ void __launch_bounds__(32 * kGemvWarps)
gemv_cols_kernel(int64_t n, const double* __restrict__ M, int64_t ldm, const double* __restrict__ X, int64_t ldx,
                 double* __restrict__ Y, int64_t ldy) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * kGemvWarps + w; i < n; i += (int64_t)gridDim.x * kGemvWarps) {
    const double* col = M + i * ldm;
    double acc[KR];
#pragma unroll
    for (int c = 0; c < KR; ++c) acc[c] = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
      const double mv = col[j];
#pragma unroll
      for (int c = 0; c < KR; ++c) acc[c] = fma(mv, X[j + c * ldx], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < KR; ++c) {
      const double v = warp_sum(acc[c]);
      if (lane == 0) Y[i + c * ldy] = v;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Blocked right-looking Cholesky, 32-wide panels, for a batch of matrices at once
// (blockIdx.z selects the matrix).  On GB300 one warp issues FP64 fused multiply-adds at
// about one per 64 cycles (the SM's FP64 rate is about 2 lanes per clock over its four
// sub-partitions), so no FP64 stage may rest on a single warp: every kernel spreads its
// multiply-adds over several warps and CTAs.  Two launches per panel:
//   chol_panel_kernel  every CTA factors the 32 x 32 diagonal block in shared memory
//                      (4 warps; redundantly, so no CTA waits for another), CTA 0 stores
//                      it, and each warp then solves one row of L21 = A21 L11^{-T} with
//                      the 32 columns spread over its lanes;
//   syrk16_kernel      A22 -= L21 L21^T on 16 x 16 lower tiles, 4 warps per tile.
// Division by a pivot is multiplication by its reciprocal square root.
// ---------------------------------------------------------------------------------------
constexpr int kNB = 32;
constexpr int kPanelWarps = 4;

template <typename T>
struct CholBatch {
  T* M[2];         // matrices (ld n), lower triangles factored in place
  T* inv_diag[2];  // 1 / L_ii, filled panel by panel
  T* stash[2];     // 32 x 32 factored diagonal block of the current panel
  int32_t* status;
};

// Pivot test: NONFINITE, NOT_SPD or 0.  FP64 looks at the bit pattern (integer pipes, not
// the scarce FP64 one); FP32 compares directly.
__device__ __forceinline__ int pivot_code(double d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
  if (((bits >> 52) & 0x7ffull) == 0x7ffull) return ILS_ERR_NONFINITE;
  if ((bits >> 63) != 0ull || bits == 0ull) return ILS_ERR_NOT_SPD;
  return 0;
}
__device__ __forceinline__ int pivot_code(float d) {
  if (!isfinite(d)) return ILS_ERR_NONFINITE;
  if (!(d > 0.f)) return ILS_ERR_NOT_SPD;
  return 0;
}
__device__ __forceinline__ double rsqrt_t(double d) { return rsqrt(d); }
__device__ __forceinline__ float rsqrt_t(float d) { return rsqrtf(d); }

__device__ void set_status(int32_t* status, int32_t code) { atomicCAS(status, 0, code); }

template <typename T>
__global__ void __launch_bounds__(32 * kPanelWarps)
chol_panel_kernel(int64_t n, CholBatch<T> cb, int64_t k0, int nb) {
  T* L = cb.M[blockIdx.z];
  T* inv = cb.inv_diag[blockIdx.z];
  __shared__ T a[kNB][kNB + 1];
  __shared__ T rinv[kNB];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int r = e & 31, c = e >> 5;
    a[r][c] = (r < nb && c < nb && r >= c) ? L[(k0 + r) + (k0 + c) * n] : (r == c ? T(1) : T(0));
  }
  __syncthreads();
  // Pivot c: every thread reads a[c][c] and forms rs = 1/sqrt(a_cc) itself, then
  // a[i][j] -= a[i][c] a[j][c] rs^2 for c < j <= i (lane = column j, warps take rows in
  // turn).  Column c is scaled by rs one pivot later, once nobody reads it unscaled.
  for (int c = 0; c < kNB; ++c) {
    __syncthreads();
    if (c > 0 && w == 0 && lane >= c - 1) a[lane][c - 1] *= rinv[c - 1];
    T d = a[c][c];
    const int code = pivot_code(d);
    if (code != 0) {
      if (tid == 0 && blockIdx.x == 0) set_status(cb.status, code);
      d = T(1);
    }
    const T rs = rsqrt_t(d);
    if (tid == 0) rinv[c] = rs;
    const int j = lane;
    if (j > c) {
      const T tj = a[j][c] * (rs * rs);
      for (int i = j + ((w - j) % kPanelWarps + kPanelWarps) % kPanelWarps; i < kNB; i += kPanelWarps)
        a[i][j] = fma(-a[i][c], tj, a[i][j]);
    }
  }
  __syncthreads();
  if (w == 0 && lane >= kNB - 1) a[lane][kNB - 1] *= rinv[kNB - 1];
  __syncthreads();
  // The factored block goes to the stash, and into L only when this CTA is the only one:
  // other CTAs of the launch may start late and still have to read the unfactored block.
  // The trailing-update launch that follows moves the stash into L.
  if (blockIdx.x == 0) {
    T* stash = cb.stash[blockIdx.z];
    for (int e = tid; e < kNB * kNB; e += blockDim.x) {
      const int r = e & 31, c = e >> 5;
      stash[e] = a[r][c];
      if (gridDim.x == 1 && r < nb && c < nb && r >= c) L[(k0 + r) + (k0 + c) * n] = a[r][c];
    }
    if (tid < nb) inv[k0 + tid] = rinv[tid];
  }
  // Rows of L21, two per warp at a time: x_c = (a_c - sum_{d<c} x_d l_cd) / l_cc with the
  // columns over the lanes.  The grid holds at most one CTA per SM, so the redundant
  // factorizations above never share an SM's FP64 pipes.
  const int64_t stride = (int64_t)gridDim.x * kPanelWarps;
  for (int64_t row = k0 + nb + (int64_t)blockIdx.x * kPanelWarps + w; row < n; row += 2 * stride) {
    const int64_t row2 = row + stride;
    const bool two = row2 < n;
    T x = lane < nb ? L[row + (k0 + lane) * n] : T(0);
    T y = (two && lane < nb) ? L[row2 + (k0 + lane) * n] : T(0);
    for (int c = 0; c < nb; ++c) {
      const T xc = __shfl_sync(0xffffffffu, x, c) * rinv[c];
      const T yc = __shfl_sync(0xffffffffu, y, c) * rinv[c];
      if (lane == c) {
        x = xc;
        y = yc;
      } else if (lane > c) {
        const T l = a[lane][c];
        x = fma(-xc, l, x);
        y = fma(-yc, l, y);
      }
    }
    if (lane < nb) {
      L[row + (k0 + lane) * n] = x;
      if (two) L[row2 + (k0 + lane) * n] = y;
    }
  }
}

// Trailing update A22 -= L21 L21^T on lower 16 x 16 tiles (two elements per thread).
template <typename T>
__global__ void __launch_bounds__(128)
syrk16_kernel(int64_t n, CholBatch<T> cb, int64_t k0, int nb) {
  T* L = cb.M[blockIdx.z];
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bi == 0 && bj == 0) {  // the panel's factored diagonal block, kept aside by the panel launch
    const T* stash = cb.stash[blockIdx.z];
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
      const int r = e & 31, c = e >> 5;
      if (r < nb && c < nb && r >= c) L[(k0 + r) + (k0 + c) * n] = stash[e];
    }
  }
  if (bi < bj) return;
  const int64_t k1 = k0 + nb;
  const int64_t ri0 = k1 + (int64_t)bi * 16, rj0 = k1 + (int64_t)bj * 16;
  __shared__ T Pi[16][kNB + 1];
  __shared__ T Pj[16][kNB + 1];
  for (int e = threadIdx.x; e < 16 * kNB; e += blockDim.x) {
    const int r = e & 15, c = e >> 4;
    Pi[r][c] = (ri0 + r < n && c < nb) ? L[(ri0 + r) + (k0 + c) * n] : T(0);
    Pj[r][c] = (rj0 + r < n && c < nb) ? L[(rj0 + r) + (k0 + c) * n] : T(0);
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // ty in 0..7
  T acc0 = T(0), acc1 = T(0);
#pragma unroll 8
  for (int c = 0; c < kNB; ++c) {
    const T pj = Pj[tx][c];
    acc0 = fma(Pi[ty][c], pj, acc0);
    acc1 = fma(Pi[ty + 8][c], pj, acc1);
  }
  const int64_t gj = rj0 + tx;
  const int64_t gi0 = ri0 + ty, gi1 = ri0 + ty + 8;
  if (gi0 < n && gj < n && gi0 >= gj) L[gi0 + gj * n] -= acc0;
  if (gi1 < n && gj < n && gi1 >= gj) L[gi1 + gj * n] -= acc1;
}

// ---------------------------------------------------------------------------------------
// Triangular solves with many right-hand sides: one warp per right-hand side, the vector
// kept in shared memory.  The blocked kernel stages each 32-column panel of L (rows i0..n-1)
// in shared memory once per 32 substitution steps, so a step reads L from shared memory
// instead of paying an L2 round trip; the simple kernel is the fallback when the panel does
// not fit.
// ---------------------------------------------------------------------------------------
constexpr int kTrsmWarps = 4;

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(32 * kTrsmWarps)
trsm_kernel(int64_t n, int64_t k, const T* __restrict__ L, T* __restrict__ X, int64_t ldx, int fwd, int bwd) {
  extern __shared__ __align__(16) unsigned char smem_raw_t[];
  T* smem_y = reinterpret_cast<T*>(smem_raw_t);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * kTrsmWarps + w;
  if (col >= k) return;
  T* y = smem_y + (size_t)w * n;
  T* xc = X + col * ldx;
  for (int64_t r = lane; r < n; r += 32) y[r] = xc[r];
  __syncwarp();
  if (fwd) {
    for (int64_t i = 0; i < n; ++i) {
      const T yi = y[i] / L[i + i * n];
      __syncwarp();
      if (lane == 0) y[i] = yi;
      const T* li = L + i * n;
      for (int64_t r = i + 1 + lane; r < n; r += 32) y[r] = fma(-li[r], yi, y[r]);
      __syncwarp();
    }
  }
  if (bwd) {
    for (int64_t i = n - 1; i >= 0; --i) {
      const T* li = L + i * n;
      T s = T(0);
      for (int64_t r = i + 1 + lane; r < n; r += 32) s = fma(li[r], y[r], s);
      s = warp_sum_t(s);
      if (lane == 0) y[i] = (y[i] - s) / li[i];
      __syncwarp();
    }
  }
  for (int64_t r = lane; r < n; r += 32) xc[r] = y[r];
}

template <typename T>
__global__ void __launch_bounds__(32 * kTrsmWarps)
trsm_blocked_kernel(int64_t n, int64_t k, const T* __restrict__ L, T* __restrict__ X, int64_t ldx, int fwd, int bwd) {
  extern __shared__ __align__(16) unsigned char smem_raw_t[];
  T* panel = reinterpret_cast<T*>(smem_raw_t);  // 32 columns x n rows (rows i0..n-1 used)
  T* ys = panel + (size_t)32 * n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * kTrsmWarps + w;
  const bool valid = col < k;
  T* y = ys + (size_t)w * n;
  if (valid)
    for (int64_t r = lane; r < n; r += 32) y[r] = X[r + col * ldx];
  const int nblk = (int)((n + 31) / 32);
  auto load_panel = [&](int64_t i0, int nb) {
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
      const T* src = L + (i0 + c) * n;
      T* dst = panel + (size_t)c * n;
      for (int64_t r = i0 + threadIdx.x; r < n; r += blockDim.x) dst[r] = src[r];
    }
    __syncthreads();
  };
  if (fwd) {
    for (int b = 0; b < nblk; ++b) {
      const int64_t i0 = (int64_t)b * 32;
      const int nb = (int)((n - i0) < 32 ? (n - i0) : 32);
      load_panel(i0, nb);
      if (valid) {
        for (int c = 0; c < nb; ++c) {
          const int64_t i = i0 + c;
          const T* pc = panel + (size_t)c * n;
          const T yi = y[i] / pc[i];
          __syncwarp();
          if (lane == 0) y[i] = yi;
          for (int64_t r = i + 1 + lane; r < n; r += 32) y[r] = fma(-pc[r], yi, y[r]);
          __syncwarp();
        }
      }
    }
  }
  if (bwd) {
    for (int b = nblk - 1; b >= 0; --b) {
      const int64_t i0 = (int64_t)b * 32;
      const int nb = (int)((n - i0) < 32 ? (n - i0) : 32);
      load_panel(i0, nb);
      if (valid) {
        for (int c = nb - 1; c >= 0; --c) {
          const int64_t i = i0 + c;
          const T* pc = panel + (size_t)c * n;
          T s = T(0);
          for (int64_t r = i + 1 + lane; r < n; r += 32) s = fma(pc[r], y[r], s);
          s = warp_sum_t(s);
          if (lane == 0) y[i] = (y[i] - s) / pc[i];
          __syncwarp();
        }
      }
    }
  }
  if (valid)
    for (int64_t r = lane; r < n; r += 32) X[r + col * ldx] = y[r];
}

// Inverses of the 32 x 32 diagonal blocks of a lower-triangular L (ld n): block b is stored
// column-major at Dinv + b * 1024.  Thread j forms column j of the inverse by forward
// substitution, X_jj = 1 / L_jj and X_ij = -(sum_{j <= k < i} L_ik X_kj) / L_ii.
template <typename T>
__global__ void __launch_bounds__(32) diag_block_inverse_kernel(int64_t n, const T* __restrict__ L, T* __restrict__ Dinv) {
  __shared__ T Lb[32][33];
  __shared__ T X[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int nb = (int)((n - i0) < 32 ? (n - i0) : 32);
  const int j = threadIdx.x;
  for (int a = 0; a < 32; ++a) Lb[a][j] = (a < nb && j < nb && a >= j) ? L[(i0 + a) + (i0 + j) * n] : (a == j ? T(1) : T(0));
  __syncthreads();
  // Right-looking: x = e_j; for k = j..31: x_k /= L_kk, then x_{k+1..} -= L(k+1..,k) x_k.
  T x[32];
#pragma unroll
  for (int a = 0; a < 32; ++a) x[a] = (a == j) ? T(1) : T(0);
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    if (kk >= j) {
      x[kk] = x[kk] / Lb[kk][kk];
#pragma unroll
      for (int a = kk + 1; a < 32; ++a) x[a] = fma(-Lb[a][kk], x[kk], x[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 32; ++a) X[a][j] = x[a];
  for (int a = 0; a < 32; ++a) Dinv[(size_t)blockIdx.x * 1024 + a + j * 32] = X[a][j];
}

// X := L^{-1} X and/or L^{-T} X by 32-row block substitution with the diagonal-block
// inverses: T = X_I - sum_{J<I} L_IJ X_J, X_I = Dinv_I T (and the transposed sweep
// backwards).  Each CTA owns CT right-hand sides, kept in shared memory; one thread per
// (row of the block, right-hand side).
template <typename T, int CT>
__global__ void __launch_bounds__(32 * CT)
trsm_binv_kernel(int64_t n, int64_t k, const T* __restrict__ L, const T* __restrict__ Dinv, T* __restrict__ X,
                 int64_t ldx, int fwd, int bwd) {
  extern __shared__ __align__(16) unsigned char smem_raw_b[];
  T* Xs = reinterpret_cast<T*>(smem_raw_b);      // CT columns of length n
  T* Pn = Xs + (size_t)CT * n;                   // one block row / block column of L: 32 x n
  __shared__ T Db[32][33];
  __shared__ T Tm[32][CT];
  const int r = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int nthr = 32 * CT;
  const int64_t col = (int64_t)blockIdx.x * CT + c;
  const bool cvalid = col < k;
  for (int64_t e = r; e < n; e += 32) Xs[(size_t)c * n + e] = cvalid ? X[e + col * ldx] : T(0);
  const int nblk = (int)((n + 31) / 32);
  auto load_dinv = [&](int64_t ib) {
    for (int e = threadIdx.x; e < 1024; e += nthr) Db[e & 31][e >> 5] = Dinv[(size_t)ib * 1024 + e];
  };
  if (fwd) {
    for (int I = 0; I < nblk; ++I) {
      const int64_t i0 = (int64_t)I * 32, cols = i0;  // L(i0..i0+31, 0..i0-1), stored Pn[col * 32 + row]
      __syncthreads();
      batched_copy(Pn, cols * 32, threadIdx.x, nthr, [&](int64_t e) {
        const int64_t cc = e >> 5, rr = e & 31;
        return (i0 + rr < n) ? L[(i0 + rr) + cc * n] : T(0);
      });
      load_dinv(I);
      __syncthreads();
      const int64_t gi = i0 + r;
      T acc = (gi < n) ? Xs[(size_t)c * n + gi] : T(0);
      const T* xc = Xs + (size_t)c * n;
#pragma unroll 8
      for (int64_t cc = 0; cc < cols; ++cc) acc = fma(-Pn[cc * 32 + r], xc[cc], acc);
      Tm[r][c] = acc;
      __syncthreads();
      T out = T(0);
#pragma unroll 8
      for (int b = 0; b < 32; ++b) out = fma(Db[r][b], Tm[b][c], out);
      if (gi < n) Xs[(size_t)c * n + gi] = out;
    }
  }
  if (bwd) {
    for (int I = nblk - 1; I >= 0; --I) {
      const int64_t i0 = (int64_t)I * 32, j0 = i0 + 32;
      const int64_t rows = n > j0 ? n - j0 : 0;  // L(j0..n-1, i0..i0+31), stored Pn[b * rows + row]
      __syncthreads();
      batched_copy(Pn, rows * 32, threadIdx.x, nthr, [&](int64_t e) {
        const int64_t b = e / rows, rr = e - b * rows;
        return (i0 + b < n) ? L[(j0 + rr) + (i0 + b) * n] : T(0);
      });
      load_dinv(I);
      __syncthreads();
      const int64_t gi = i0 + r;
      T acc = (gi < n) ? Xs[(size_t)c * n + gi] : T(0);
      const T* xc = Xs + (size_t)c * n + j0;
      const T* pr = Pn + (size_t)r * rows;
#pragma unroll 8
      for (int64_t e = 0; e < rows; ++e) acc = fma(-pr[e], xc[e], acc);
      Tm[r][c] = acc;
      __syncthreads();
      T out = T(0);
#pragma unroll 8
      for (int b = 0; b < 32; ++b) out = fma(Db[b][r], Tm[b][c], out);
      if (gi < n) Xs[(size_t)c * n + gi] = out;
    }
  }
  __syncthreads();
  if (cvalid)
    for (int64_t e = r; e < n; e += 32) X[e + col * ldx] = Xs[(size_t)c * n + e];
}

__global__ void set_identity_kernel(int64_t n, double* M, int64_t ld) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (uint32_t)e % (uint32_t)n, j = (uint32_t)e / (uint32_t)n;  // n * n < 2^31
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
    const int64_t i = (uint32_t)e % (uint32_t)n, j = (uint32_t)e / (uint32_t)n;  // n * n < 2^31
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

template <int KR>
__global__ void __launch_bounds__(32 * kIterWarps) sp_iter_kernel(SpIterArgs a) {
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done)) return;
  const int cur = *((volatile int32_t*)&st->cur);
  const double* __restrict__ x = cur ? a.X1 : a.X0;
  double* __restrict__ xn = cur ? a.X0 : a.X1;
  const int64_t n = a.n;
  constexpr int k = KR;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ int32_t done_c[kMaxRhsPerPass];
  if (threadIdx.x < kMaxRhsPerPass) done_c[threadIdx.x] = (threadIdx.x < k) ? a.col_done[threadIdx.x] : 1;
  __syncthreads();
  double rpart[KR];
#pragma unroll
  for (int c = 0; c < KR; ++c) rpart[c] = 0.0;

  for (int64_t i = (int64_t)blockIdx.x * kIterWarps + w; i < n; i += (int64_t)gridDim.x * kIterWarps) {
    const double* brow = a.Bt + i * n;
    const double* hrow = a.H + i * n;
    double ab[KR], ah[KR];
#pragma unroll
    for (int c = 0; c < KR; ++c) ab[c] = ah[c] = 0.0;
    double ab2[KR], ah2[KR];
#pragma unroll
    for (int c = 0; c < KR; ++c) ab2[c] = ah2[c] = 0.0;
    int64_t j = lane;
    if (a.mode == 3) {
      // matrix-free SP: ab = P (v + bbar), ah = Abar1 x
      for (; j < n; j += 32) {
        const double bv = brow[j], hv = hrow[j];
#pragma unroll
        for (int c = 0; c < KR; ++c) {
          ab[c] = fma(bv, a.vvec[j + c * n] + a.bbar[j + c * n], ab[c]);
          ah[c] = fma(hv, x[j + c * n], ah[c]);
        }
      }
    } else if (a.mode != 2 && a.mode != 4) {
      for (; j + 32 < n; j += 64) {
        const double bv = brow[j], hv = hrow[j], bv2 = brow[j + 32], hv2 = hrow[j + 32];
#pragma unroll
        for (int c = 0; c < KR; ++c) {
          const double xv = x[j + c * n], xv2 = x[j + 32 + c * n];
          ab[c] = fma(bv, xv, ab[c]);
          ah[c] = fma(hv, xv, ah[c]);
          ab2[c] = fma(bv2, xv2, ab2[c]);
          ah2[c] = fma(hv2, xv2, ah2[c]);
        }
      }
      for (; j < n; j += 32) {
        const double bv = brow[j], hv = hrow[j];
#pragma unroll
        for (int c = 0; c < KR; ++c) {
          const double xv = x[j + c * n];
          ab[c] = fma(bv, xv, ab[c]);
          ah[c] = fma(hv, xv, ah[c]);
        }
      }
    } else {
      for (; j + 32 < n; j += 64) {
        const double hv = hrow[j], hv2 = hrow[j + 32];
#pragma unroll
        for (int c = 0; c < KR; ++c) {
          ah[c] = fma(hv, x[j + c * n], ah[c]);
          ah2[c] = fma(hv2, x[j + 32 + c * n], ah2[c]);
        }
      }
      for (; j < n; j += 32) {
        const double hv = hrow[j];
#pragma unroll
        for (int c = 0; c < KR; ++c) ah[c] = fma(hv, x[j + c * n], ah[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < KR; ++c) {
      ab[c] += ab2[c];
      ah[c] += ah2[c];
    }
#pragma unroll
    for (int c = 0; c < KR; ++c) {
      const double sb = (a.mode != 2 && a.mode != 4) ? warp_sum(ab[c]) : 0.0;
      const double sh = warp_sum(ah[c]);
      if (lane == 0) {
        const bool inplace = a.mode == 2 || a.mode == 4;
        if (done_c[c]) {
          if (!inplace) xn[i + c * n] = x[i + c * n];
        } else {
          const double r = a.bbar[i + c * n] - sh + ((a.mode >= 3) ? a.vvec[i + c * n] : 0.0);
          if (a.mode == 0) xn[i + c * n] = sb + a.cvec[i + c * n];
          else if (a.mode == 1) a.bhat_out[i + c * n] = sb + a.cvec[i + c * n];
          else if (a.mode == 3) xn[i + c * n] = sb;
          else a.bhat_out[i + c * n] = r;
          rpart[c] = fma(r, r, rpart[c]);
        }
      }
    }
  }
  __shared__ double red[kIterWarps][KR];
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < KR; ++c) red[w][c] = rpart[c];
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
  // ||r_k||^2 per column: every thread of the last CTA adds a strided share of the per-CTA
  // partials (a serial sum would chain gridDim.x dependent FP64 additions).
  __shared__ double rr_w[kIterWarps][KR];
#pragma unroll
  for (int c = 0; c < KR; ++c) {
    double v = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) v += __ldcg(&a.partials[(int64_t)b * k + c]);
    v = warp_sum(v);
    if (lane == 0) rr_w[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    const int64_t it = st->iters;
    for (int c = 0; c < k; ++c) {
      newly_done[c] = 0;
      if (done_c[c]) continue;
      double rr = 0.0;
      for (int ww = 0; ww < kIterWarps; ++ww) rr += rr_w[ww][c];
      const bool finite = isfinite(rr);
      const bool conv = finite && rr <= a.tol2 * (a.tol_scale ? *a.tol_scale : 1.0) * a.bnorm2[c];
      if (!finite || conv || it >= st->max_outer) {
        a.col_done[c] = 1;
        a.col_rr[c] = rr;
        a.col_iters[c] = it;
        newly_done[c] = 1;
        if (!finite) atomicCAS(&st->status, 0, ILS_ERR_NONFINITE);
        else if (!conv) atomicCAS(&st->status, 0, ILS_ERR_NO_CONVERGENCE);
      } else {
        all = 0;
        if (a.mode == 1 || a.mode == 2) {
          double th2 = a.theta2;  // the schedule: theta_k^2 = max(theta^2 decay^(2k), theta_min^2)
          if (a.theta_decay > 0.0 && a.theta_decay < 1.0)
            th2 = fmax(a.theta2 * pow(a.theta_decay, 2.0 * (double)it), a.theta_min2);
          a.col_target2[c] = th2 * rr;
        }
      }
    }
    all_done = all;
    if (all) {
      st->done = 1;  // the answer of every column is in buffer `cur`
    } else {
      if (a.mode != 2 && a.mode != 4) st->cur = cur ^ 1;  // modes 2 and 4 update x in place
      st->iters = it + 1;
    }
    st->counter = 0u;
  }
  __syncthreads();
  if (!all_done && a.mode != 2 && a.mode != 4) {
    // Columns that finished now keep x_k: copy it over the x_{k+1} just written.
    for (int c = 0; c < k; ++c) {
      if (!newly_done[c]) continue;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xn[i + c * n] = x[i + c * n];
    }
  }
}

__global__ void copy_final_kernel(int64_t n, int64_t k, const double* X0, const double* X1,
                                  const SolveState* st, double* X, int64_t ldx, ResultGather g) {
  const double* src = st->cur ? X1 : X0;
  if (g.out && blockIdx.x == 0 && threadIdx.x < 32) {  // the pass's results, for one copy to the host
    char* out = static_cast<char*>(g.out);
    const int t = threadIdx.x;
    if (t < (int)(sizeof(SolveState) / 4)) reinterpret_cast<uint32_t*>(out + kResSt)[t] = reinterpret_cast<const uint32_t*>(g.st)[t];
    if (t < g.k) {
      reinterpret_cast<double*>(out + kResRr)[t] = g.rr[t];
      reinterpret_cast<double*>(out + kResBn)[t] = g.bn[t];
      reinterpret_cast<int64_t*>(out + kResIters)[t] = g.iters[t];
      reinterpret_cast<int64_t*>(out + kResInner)[t] = g.inner[t];
    }
    if (t == 0) *reinterpret_cast<unsigned long long*>(out + kResInnerNs) = g.inner_ns ? *g.inner_ns : 0ull;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (uint32_t)e % (uint32_t)n, c = (uint32_t)e / (uint32_t)n;
    X[i + c * ldx] = src[i + c * n];
  }
}

// ---------------------------------------------------------------------------------------
// FP32 Cholesky in one launch (n <= kDfMaxN): left-looking, data-driven at the grain of
// 32-row chunks.  CTA j owns the 32-column panel j; its warp w owns the chunks t = w,
// w + 8, ... (rows 32j + 32t .. + 31, one row per lane, the 32 columns in registers).
// A chunk is updated by every earlier panel k as soon as the chunk of panel k covering
// the same rows is published (A_j(t) -= L_k(t') L_k(j)^T, where L_k(j) is panel k's
// 32 x 32 block in the rows of block j, staged in shared memory by warp 0, which reads it
// anyway for chunk 0), then solved against the factored diagonal block and published
// under its own flag.  Warp 0 factors the diagonal block (lane = row, each pivot's column
// broadcast by shuffles) as soon as chunk 0 is updated.  The next panel's diagonal block
// therefore waits only for one chunk of this panel, not for the whole panel, and the
// n^3/3 multiply-adds are spread over the CTAs' warps without any launch boundary.
// A chunk's flag is set only after its stores are fenced; waiting warps read it through
// L2.  Every wait is bounded: past the limit the warp records TIMEOUT, raises the abort
// word (which releases every other waiter) and returns.
// ---------------------------------------------------------------------------------------
constexpr int kDfWarps = 8;
constexpr int kDfThreads = 32 * kDfWarps;
constexpr int64_t kDfMaxN = 768;  // the staged 32 x 32 blocks of all earlier panels fit in shared memory

struct DfArgs {
  float* M[2];
  float* inv_diag[2];
  uint32_t* flags[2];  // flags[i][k * npanels + t]: chunk t of panel k stored; [npanels^2]: abort
  int32_t* status[2];
  int64_t n;
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t ld_acquire_smem(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_smem(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// One warp waits until *flag != 0 (global when `global`, else this CTA's shared memory).
// Returns false on abort or after about 1 s (then TIMEOUT is recorded and abort raised).
__device__ __forceinline__ bool df_wait_warp(const uint32_t* flag, bool global, uint32_t* abort_word,
                                             int32_t* status) {
  int res = 1;
  if ((threadIdx.x & 31) == 0) {
    uint64_t t0 = 0;
    for (uint32_t spin = 0;; ++spin) {
      // Relaxed polls; the fence after a poll that sees the flag makes it an acquire.
      if ((global ? ld_relaxed_u32(flag) : ld_acquire_smem(flag)) != 0u) {
        if (global) asm volatile("fence.acq_rel.gpu;" ::: "memory");
        break;
      }
      if ((spin & 15u) == 15u) {
        if (ld_acquire_u32(abort_word) != 0u) {
          res = 0;
          break;
        }
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > 1000000000ull) {
          atomicCAS(status, 0, (int32_t)ILS_ERR_TIMEOUT);
          atomicExch(abort_word, 1u);
          res = 0;
          break;
        }
      }
      if (spin >= 64u) __nanosleep(32);
    }
  }
  res = __shfl_sync(0xffffffffu, res, 0);
  __syncwarp();
  return res != 0;
}

__global__ void __launch_bounds__(kDfThreads)
chol_dataflow_f32_kernel(DfArgs a) {
  extern __shared__ __align__(16) float df_smem[];
  const int mat = blockIdx.y;
  float* L = a.M[mat];
  uint32_t* flags = a.flags[mat];
  int32_t* status = a.status[mat];
  const int64_t n = a.n;
  const int np = (int)((n + 31) / 32);
  uint32_t* abort_word = flags + (size_t)np * np;
  const int j = blockIdx.x;
  const int64_t c0 = 32 * (int64_t)j;
  const int nb = (int)(n - c0 < 32 ? n - c0 : 32);
  const int nchunks = (int)((n - c0 + 31) / 32);
  float* W = df_smem;                     // [k][kk][c] = L(c0 + c, 32k + kk)
  float* LT = W + (size_t)np * 1024;      // [c][d] = L11(d, c)
  float* rinv = LT + 1024;                // 1 / L11(c, c)
  uint32_t* wready = reinterpret_cast<uint32_t*>(rinv + 32);  // [k]: W block k staged
  uint32_t* l11_ready = wready + np;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i <= np; i += kDfThreads) wready[i] = 0u;
  __syncthreads();

  for (int t = w; t < nchunks; t += kDfWarps) {
    const int64_t r = c0 + 32 * (int64_t)t + lane;  // this lane's row
    const bool live = r < n;
    float acc[32];
    if (t == 0) {
      // Lower part of the diagonal block; past a ragged end it acts as an identity block.
#pragma unroll
      for (int c = 0; c < 32; ++c)
        acc[c] = (c < nb && lane < nb) ? (lane >= c ? L[r + (c0 + c) * n] : 0.f) : (lane == c ? 1.f : 0.f);
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = live ? L[r + (c0 + c) * n] : 0.f;
    }
    // Updates from the earlier panels, each once its chunk over these rows is stored.
    for (int k = 0; k < j; ++k) {
      if (!df_wait_warp(flags + (size_t)k * np + (j - k + t), true, abort_word, status)) return;
      const float* Lk = L + 32 * (int64_t)k * n;
      float lk[32];
#pragma unroll
      for (int kk = 0; kk < 32; ++kk) lk[kk] = live ? __ldcg(Lk + r + kk * n) : 0.f;
      float* Wk = W + (size_t)k * 1024;
      if (t == 0) {
        // These rows are panel k's block in the rows of block j: stage it for the other warps.
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) Wk[kk * 32 + lane] = lk[kk];
        __syncwarp();
        if (lane == 0) st_release_smem(wready + k, 1u);
        __syncwarp();
      } else if (!df_wait_warp(wready + k, false, abort_word, status)) {
        return;
      }
#pragma unroll
      for (int kk = 0; kk < 32; ++kk) {
        const float4* w4 = reinterpret_cast<const float4*>(Wk + kk * 32);
#pragma unroll
        for (int c4 = 0; c4 < 8; ++c4) {
          const float4 v = w4[c4];
          acc[4 * c4 + 0] = fmaf(-lk[kk], v.x, acc[4 * c4 + 0]);
          acc[4 * c4 + 1] = fmaf(-lk[kk], v.y, acc[4 * c4 + 1]);
          acc[4 * c4 + 2] = fmaf(-lk[kk], v.z, acc[4 * c4 + 2]);
          acc[4 * c4 + 3] = fmaf(-lk[kk], v.w, acc[4 * c4 + 3]);
        }
      }
    }
    if (t == 0) {
      // Diagonal block, lane i = row i.  Pivot c: every lane posts a_ic to a shared column
      // buffer; with d = a_cc and rs = 1/sqrt(d): l_cc = d rs, l_ic = a_ic rs, and
      // a_ij -= (a_ic rs^2) a_jc for j > c, a_jc read back from the buffer (4 at a time).
      float* colbuf = LT;  // the factor's column buffer until the factor is written there
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        colbuf[(c & 1) * 32 + lane] = acc[c];
        __syncwarp();
        float d = colbuf[(c & 1) * 32 + c];
        const int code = pivot_code(d);
        if (code != 0) {
          if (lane == 0) set_status(status, code);
          d = 1.f;
        }
        const float rs = rsqrtf(d);
        const float ti = lane > c ? acc[c] * (rs * rs) : 0.f;
        acc[c] = lane > c ? acc[c] * rs : (lane == c ? d * rs : 0.f);
        if (lane == 0) rinv[c] = rs;
        const float4* col4 = reinterpret_cast<const float4*>(colbuf + (c & 1) * 32);
#pragma unroll
        for (int q = (c + 1) / 4; q < 8; ++q) {
          const float4 v = col4[q];
          if (4 * q + 0 > c) acc[4 * q + 0] = fmaf(-ti, v.x, acc[4 * q + 0]);
          if (4 * q + 1 > c) acc[4 * q + 1] = fmaf(-ti, v.y, acc[4 * q + 1]);
          if (4 * q + 2 > c) acc[4 * q + 2] = fmaf(-ti, v.z, acc[4 * q + 2]);
          if (4 * q + 3 > c) acc[4 * q + 3] = fmaf(-ti, v.w, acc[4 * q + 3]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int c = 0; c < 32; ++c) LT[c * 32 + lane] = lane >= c ? acc[c] : 0.f;
      __syncwarp();
      if (lane == 0) st_release_smem(l11_ready, 1u);
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < nb && lane < nb && lane >= c) L[r + (c0 + c) * n] = acc[c];
      if (lane < nb) a.inv_diag[mat][c0 + lane] = rinv[lane];
    } else {
      // Rows below the diagonal block: x = a L11^{-T} by forward substitution.
      if (!df_wait_warp(l11_ready, false, abort_word, status)) return;
      const float4* lt4 = reinterpret_cast<const float4*>(LT);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        acc[c] *= rinv[c];
#pragma unroll
        for (int q = (c + 1) / 4; q < 8; ++q) {
          const float4 v = lt4[c * 8 + q];
          if (4 * q + 0 > c) acc[4 * q + 0] = fmaf(-acc[c], v.x, acc[4 * q + 0]);
          if (4 * q + 1 > c) acc[4 * q + 1] = fmaf(-acc[c], v.y, acc[4 * q + 1]);
          if (4 * q + 2 > c) acc[4 * q + 2] = fmaf(-acc[c], v.z, acc[4 * q + 2]);
          if (4 * q + 3 > c) acc[4 * q + 3] = fmaf(-acc[c], v.w, acc[4 * q + 3]);
        }
      }
      if (live) {
#pragma unroll
        for (int c = 0; c < 32; ++c) L[r + (c0 + c) * n] = acc[c];
      }
      // The warp barrier orders every lane's stores before lane 0's release.
      __syncwarp();
      if (lane == 0) st_release_u32(flags + (size_t)j * np + t, 1u);
    }
  }
}

size_t df_smem_bytes(int64_t n) {
  const size_t np = (size_t)((n + 31) / 32);
  return sizeof(float) * (np * 1024 + 1024 + 32) + sizeof(uint32_t) * (np + 1);
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
  for (int64_t c0 = 0; c0 < k; c0 += kMaxRhsPerPass) {
    const int kk = (int)std::min<int64_t>(kMaxRhsPerPass, k - c0);
    const double* Bc = B + c0 * ldb;  // the kernel indexes columns from 0
    double* Oc = out + c0 * ldo;
    const dim3 grid((unsigned)n, 1);
    switch (kk) {
      case 1: rhs_bar_kernel<1><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
      case 2: rhs_bar_kernel<2><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
      case 3: rhs_bar_kernel<3><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
      case 4: rhs_bar_kernel<4><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
      case 5: rhs_bar_kernel<5><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
      case 6: rhs_bar_kernel<6><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
      case 7: rhs_bar_kernel<7><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
      default: rhs_bar_kernel<8><<<grid, kRhsThreads, 0, s>>>(m, n, p, kk, A, lda, Bc, ldb, Oc, ldo); break;
    }
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t gemv_cols_f64(int64_t n, int64_t k, const double* M, int64_t ldm, const double* X, int64_t ldx,
                          double* Y, int64_t ldy, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + kGemvWarps - 1) / kGemvWarps, 16 * (int64_t)num_sms());
  for (int64_t c0 = 0; c0 < k; c0 += kMaxRhsPerPass) {
    const int kk = (int)std::min<int64_t>(kMaxRhsPerPass, k - c0);
    const double* Xc = X + c0 * ldx;
    double* Yc = Y + c0 * ldy;
    switch (kk) {
      case 1: gemv_cols_kernel<1><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
      case 2: gemv_cols_kernel<2><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
      case 3: gemv_cols_kernel<3><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
      case 4: gemv_cols_kernel<4><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
      case 5: gemv_cols_kernel<5><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
      case 6: gemv_cols_kernel<6><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
      case 7: gemv_cols_kernel<7><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
      default: gemv_cols_kernel<8><<<blocks, 32 * kGemvWarps, 0, s>>>(n, M, ldm, Xc, ldx, Yc, ldy); break;
    }
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// dst (m x n, ld m) = src (m x n, ld lda).  Contiguous 16-byte moves when both layouts
// allow (a 2D memcpy between device buffers runs at about a third of the copy bandwidth).
__global__ void copy_matrix_kernel(int64_t m, int64_t n, const double* __restrict__ src, int64_t lda,
                                   double* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (lda == m && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const int64_t pairs = m * n / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pairs; i += stride) d2[i] = __ldcs(s2 + i);
    if ((m * n) & 1) {
      if (blockIdx.x == 0 && threadIdx.x == 0) dst[m * n - 1] = src[m * n - 1];
    }
    return;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n; e += stride) {
    const int64_t j = e / m, i = e - j * m;
    dst[e] = src[i + j * lda];
  }
}

cudaError_t copy_matrix_f64(int64_t m, int64_t n, const double* src, int64_t lda, double* dst, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const int64_t work = (m * n + 1) / 2;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 8 * (int64_t)num_sms()));
  copy_matrix_kernel<<<blocks, 256, 0, s>>>(m, n, src, lda, dst);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t cholesky_batch_t(int64_t n, int count, T* const* mats, T* const* inv_diag, T* stash, int32_t* status,
                             cudaStream_t s) {
  if (count < 1 || count > 2) return cudaErrorInvalidValue;
  CholBatch<T> cb;
  for (int i = 0; i < 2; ++i) {
    cb.M[i] = mats[i < count ? i : 0];
    cb.inv_diag[i] = inv_diag[i < count ? i : 0];
    cb.stash[i] = stash + (size_t)(i < count ? i : 0) * kNB * kNB;
  }
  cb.status = status;
  for (int64_t k0 = 0; k0 < n; k0 += kNB) {
    const int nb = (int)std::min<int64_t>(kNB, n - k0);
    const int64_t rest = n - k0 - nb;
    const int64_t per_matrix = std::max<int64_t>(1, num_sms() / count);
    const unsigned panel_ctas =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((rest + kPanelWarps - 1) / kPanelWarps, per_matrix));
    chol_panel_kernel<T><<<dim3(panel_ctas, 1, count), 32 * kPanelWarps, 0, s>>>(n, cb, k0, nb);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (rest <= 0) break;
    const unsigned nt = (unsigned)((rest + 15) / 16);
    syrk16_kernel<T><<<dim3(nt, nt, count), 128, 0, s>>>(n, cb, k0, nb);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t cholesky_f64_batch(int64_t n, int count, double* const* mats, double* const* inv_diag, double* stash,
                               int32_t* status, cudaStream_t s) {
  return cholesky_batch_t<double>(n, count, mats, inv_diag, stash, status, s);
}

cudaError_t cholesky_f32_df(int64_t n, int count, float* const* mats, float* const* inv_diag, float* stash,
                            int32_t* const* status, cudaStream_t s) {
  // The stash holds the chunk flags: npanels^2 + 1 words per matrix, 1024 words apart.
  const int npanels = (int)((n + 31) / 32);
  DfArgs a;
  for (int i = 0; i < 2; ++i) {
    const int src = i < count ? i : 0;
    a.M[i] = mats[src];
    a.inv_diag[i] = inv_diag[src];
    a.flags[i] = reinterpret_cast<uint32_t*>(stash) + 1024 * src;
    a.status[i] = status[src];
  }
  a.n = n;
  cudaError_t e = cudaMemsetAsync(stash, 0, sizeof(uint32_t) * (1024 * (count - 1) + npanels * npanels + 1), s);
  if (e != cudaSuccess) return e;
  static const cudaError_t attr_err = cudaFuncSetAttribute(
      chol_dataflow_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)df_smem_bytes(kDfMaxN));
  if (attr_err != cudaSuccess) return attr_err;
  // Cooperative launch: all panels' CTAs are resident together, so a CTA waiting for an
  // earlier panel never holds the SM that panel needs.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)npanels, (unsigned)count, 1);
  cfg.blockDim = dim3(kDfThreads, 1, 1);
  cfg.dynamicSmemBytes = df_smem_bytes(n);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, chol_dataflow_f32_kernel, a);
  note_launch();
  return e;
}

cudaError_t cholesky_f32(int64_t n, float* M, float* inv_diag, float* stash, int32_t* status, cudaStream_t s) {
  float* mats[2] = {M, M};
  float* invd[2] = {inv_diag, inv_diag};
  if (n > 0 && n <= kDfMaxN) {
    int32_t* st[2] = {status, status};
    return cholesky_f32_df(n, 1, mats, invd, stash, st, s);
  }
  return cholesky_batch_t<float>(n, 1, mats, invd, stash, status, s);
}

cudaError_t cholesky_f32_pair(int64_t n, float* M0, float* M1, float* inv0, float* inv1, float* stash,
                              int32_t* status0, int32_t* status1, cudaStream_t s) {
  if (n > 0 && n <= kDfMaxN) {
    float* mats[2] = {M0, M1};
    float* invd[2] = {inv0, inv1};
    int32_t* st[2] = {status0, status1};
    return cholesky_f32_df(n, 2, mats, invd, stash, st, s);
  }
  cudaError_t e = cholesky_f32(n, M0, inv0, stash, status0, s);
  if (e != cudaSuccess) return e;
  return cholesky_f32(n, M1, inv1, stash, status1, s);
}


template <typename T>
cudaError_t trsm_lower_t(int64_t n, int64_t k, const T* L, T* X, int64_t ldx, bool forward, bool backward,
                         cudaStream_t s);

template <typename T>
cudaError_t trsm_binv_t(int64_t n, int64_t k, const T* L, T* Dinv, T* X, int64_t ldx, bool forward, bool backward,
                        cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  constexpr int CT0 = sizeof(T) == 8 ? 4 : 8;
  if (sizeof(T) * (size_t)n * (CT0 + 32) > 200 * 1024)  // panel does not fit: per-step solver
    return trsm_lower_t<T>(n, k, L, X, ldx, forward, backward, s);
  const int nblk = (int)((n + 31) / 32);
  diag_block_inverse_kernel<T><<<nblk, 32, 0, s>>>(n, L, Dinv);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // FP64 is issue-bound: 4 right-hand sides per CTA spread the work over more SMs.
  constexpr int CT = sizeof(T) == 8 ? 4 : 8;
  const size_t smem = sizeof(T) * (size_t)n * (CT + 32);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 0) {  // static shared arrays count against the same limit
    e = cudaFuncSetAttribute(trsm_binv_kernel<T, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  trsm_binv_kernel<T, CT><<<(unsigned)((k + CT - 1) / CT), 32 * CT, smem, s>>>(n, k, L, Dinv, X, ldx,
                                                                             forward ? 1 : 0, backward ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t trsm_lower_t(int64_t n, int64_t k, const T* L, T* X, int64_t ldx, bool forward, bool backward,
                         cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((k + kTrsmWarps - 1) / kTrsmWarps);
  const size_t blocked = sizeof(T) * (size_t)n * (32 + kTrsmWarps);
  if (blocked <= 200 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(trsm_blocked_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(blocked, 48 * 1024));
    if (e != cudaSuccess) return e;
    trsm_blocked_kernel<T><<<grid, 32 * kTrsmWarps, blocked, s>>>(n, k, L, X, ldx, forward ? 1 : 0,
                                                                  backward ? 1 : 0);
    note_launch();
    return cudaGetLastError();
  }
  const size_t smem = sizeof(T) * (size_t)n * kTrsmWarps;
  if (smem > 0) {  // static shared arrays count against the same limit
    cudaError_t e = cudaFuncSetAttribute(trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  trsm_kernel<T><<<grid, 32 * kTrsmWarps, smem, s>>>(n, k, L, X, ldx, forward ? 1 : 0, backward ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t trsm_lower_f64(int64_t n, int64_t k, const double* L, double* X, int64_t ldx, bool forward,
                           bool backward, cudaStream_t s) {
  return trsm_lower_t<double>(n, k, L, X, ldx, forward, backward, s);
}

cudaError_t trsm_lower_f32(int64_t n, int64_t k, const float* L, float* X, int64_t ldx, bool forward,
                           bool backward, cudaStream_t s) {
  return trsm_lower_t<float>(n, k, L, X, ldx, forward, backward, s);
}

cudaError_t diag_block_inverse_f32(int64_t n, const float* L, float* Dinv, cudaStream_t s) {
  diag_block_inverse_kernel<float><<<(unsigned)((n + 31) / 32), 32, 0, s>>>(n, L, Dinv);
  note_launch();
  return cudaGetLastError();
}

cudaError_t trsm_binv_f64(int64_t n, int64_t k, const double* L, double* Dinv, double* X, int64_t ldx, bool forward,
                          bool backward, cudaStream_t s) {
  return trsm_binv_t<double>(n, k, L, Dinv, X, ldx, forward, backward, s);
}

cudaError_t trsm_binv_f32(int64_t n, int64_t k, const float* L, float* Dinv, float* X, int64_t ldx, bool forward,
                          bool backward, cudaStream_t s) {
  return trsm_binv_t<float>(n, k, L, Dinv, X, ldx, forward, backward, s);
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

__global__ void hdiff_kernel(int64_t total, const double* __restrict__ X, const double* __restrict__ Y,
                             double* __restrict__ Z, float* __restrict__ Z32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double z = X[e] - Y[e];
    Z[e] = z;
    Z32[e] = (float)z;
  }
}

cudaError_t diff_mat_f64_f32(int64_t n, const double* X, const double* Y, double* Z, float* Z32, cudaStream_t s) {
  hdiff_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(n * n, X, Y, Z, Z32);
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
  const int blocks = sp_iterate_blocks(a.n);
  switch ((int)a.k) {
    case 1: sp_iter_kernel<1><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
    case 2: sp_iter_kernel<2><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
    case 3: sp_iter_kernel<3><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
    case 4: sp_iter_kernel<4><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
    case 5: sp_iter_kernel<5><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
    case 6: sp_iter_kernel<6><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
    case 7: sp_iter_kernel<7><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
    default: sp_iter_kernel<8><<<blocks, 32 * kIterWarps, 0, s>>>(a); break;
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_final_f64(int64_t n, int64_t k, const double* X0, const double* X1, const SolveState* st,
                           double* X, int64_t ldx, cudaStream_t s, const ResultGather* gather) {
  ResultGather g = {};
  if (gather) g = *gather;
  copy_final_kernel<<<grid_for(n * k, 256), 256, 0, s>>>(n, k, X0, X1, st, X, ldx, g);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
