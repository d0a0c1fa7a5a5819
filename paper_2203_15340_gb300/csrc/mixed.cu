// Mixed-precision SP with FP64 residual refinement.
//
// Each refinement step computes the residual r = bbar - H x in FP64 (H = Abar1 - Abar2
// from the FP64-accurate split Gram products), then solves H d = r approximately with
// `sweeps` SP iterations (Alg. 1 applied to the correction equation)
//     d_1 = P r,   d_{s+1} = B d_s + P r,
// where P = Abar1^{-1} and B = P Abar2 are held in FP32 (or B in BF16) and every product
// accumulates in FP32, and finally updates x += d in FP64.  The correction error per
// step is about rho(B)^sweeps plus the low-precision error of P and B times kappa, so the
// FP64 residual test of Sec. 5 is reached in a few steps while the O(n^2) sweeps run at
// FP32/BF16 speed.
#include <cuda_bf16.h>

#include <algorithm>

#include <cstdio>
#include <map>
#include <string>
#include <mutex>

#include "ils_internal.h"

namespace ils {
namespace {

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void f64_to_f32_kernel(int64_t count, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

__global__ void f32_to_bf16_kernel(int64_t count, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = __float2bfloat16_rn(src[e]);
}

// Operator element loads for the sweep GEMV (FP32 or BF16 storage, FP32 arithmetic).
__device__ __forceinline__ float ld_op(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ld_op(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

// out(:,c) = M^T v(:,c) (+ add(:,c)); column i of M is row i of the operator.  KR is the
// number of right-hand sides, fixed at compile time so no predicated work is issued.  Each
// warp takes whole rows; the launch shape (warps per CTA, CTAs) is picked by tune_sweeps,
// and the result does not depend on it (every row is reduced in the same order).
// v may be the FP64 residual itself (the first sweep of a refinement step reads it
// directly); with update_x the sweep also adds its result to the FP64 iterate of the
// unfinished columns (the last sweep of the step).
template <typename TM, typename TV, int KR>
__global__ void __launch_bounds__(256) sweep_kernel(MixedArgs a, const TM* __restrict__ M,
                                                    const TV* __restrict__ v,
                                                    const float* __restrict__ add,
                                                    float* __restrict__ out, int update_x) {
  if (*((volatile int32_t*)&a.st->done)) return;
  const int64_t n = a.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* x = update_x ? (*((volatile int32_t*)&a.st->cur) ? a.X1 : a.X0) : nullptr;
  for (int64_t i = (int64_t)blockIdx.x * nw + w; i < n; i += (int64_t)gridDim.x * nw) {
    const TM* col = M + i * n;
    float acc[KR];
#pragma unroll
    for (int c = 0; c < KR; ++c) acc[c] = 0.f;
    for (int64_t j = lane; j < n; j += 32) {
      const float mv = ld_op(col, j);
#pragma unroll
      for (int c = 0; c < KR; ++c) acc[c] = fmaf(mv, (float)v[j + c * n], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < KR; ++c) {
      const float sv = warp_sum_f(acc[c]);
      if (lane == 0) {
        const float o = sv + (add ? add[i + c * n] : 0.f);
        out[i + c * n] = o;
        if (update_x && !a.col_done[c]) x[i + c * n] += (double)o;
      }
    }
  }
}

template <typename TM, typename TV = float>
void launch_sweep(const MixedArgs& a, SweepShape sh, const TM* M, const TV* v, const float* add, float* out,
                  cudaStream_t s, int update_x = 0) {
  const dim3 grid((unsigned)sh.blocks), block((unsigned)(32 * sh.warps));
  switch ((int)a.k) {
    case 1: sweep_kernel<TM, TV, 1><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
    case 2: sweep_kernel<TM, TV, 2><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
    case 3: sweep_kernel<TM, TV, 3><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
    case 4: sweep_kernel<TM, TV, 4><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
    case 5: sweep_kernel<TM, TV, 5><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
    case 6: sweep_kernel<TM, TV, 6><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
    case 7: sweep_kernel<TM, TV, 7><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
    default: sweep_kernel<TM, TV, 8><<<grid, block, 0, s>>>(a, M, v, add, out, update_x); break;
  }
  note_launch();
}

__global__ void residual_to_f32_kernel(MixedArgs a) {
  if (*((volatile int32_t*)&a.st->done)) return;
  const int64_t total = a.n * a.k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)((uint32_t)e / (uint32_t)a.n);
    a.r32[e] = a.col_done[c] ? 0.f : (float)a.r[e];
  }
}

// x += d for the unfinished columns (FP64 update of the refinement step).
__global__ void refine_update_kernel(MixedArgs a, const float* __restrict__ d) {
  if (*((volatile int32_t*)&a.st->done)) return;
  double* x = *((volatile int32_t*)&a.st->cur) ? a.X1 : a.X0;
  const int64_t total = a.n * a.k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)((uint32_t)e / (uint32_t)a.n);
    if (!a.col_done[c]) x[e] += (double)d[e];
  }
}

// d64 = (double) d32 for the unfinished columns (the stream reads FP64 vectors).
__global__ void widen_kernel(MixedArgs a, const float* __restrict__ d, double* __restrict__ d64) {
  if (*((volatile int32_t*)&a.st->done)) return;
  const int64_t total = a.n * a.k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    d64[e] = (double)d[e];
}

// t32 = (float) v + r32 (the right-hand side P is applied to in a matrix-free sweep).
__global__ void sweep_rhs_kernel(MixedArgs a, const double* __restrict__ v, float* __restrict__ t32) {
  if (*((volatile int32_t*)&a.st->done)) return;
  const int64_t total = a.n * a.k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    t32[e] = (float)v[e] + a.r32[e];
}

int grid_small(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 1024)); }

}  // namespace

// ---------------------------------------------------------------------------------------
// FP32 GEMM for the setup products: C = alpha op(A) op(B) + beta C, column-major, batched
// over blockIdx.z with element strides.  64 x 64 tiles, 16-deep K slices in shared
// memory, a 4 x 4 register tile per thread (two float4 shared-memory loads per 16 FMAs).
// ---------------------------------------------------------------------------------------

// Shared-memory tiles are [k][64] with the 4-float groups of a row permuted by k (an XOR
// swizzle): a warp's stores hit 32 different banks whichever operand layout it copies, and
// a float4 read of 4 consecutive m (or n) stays contiguous.
__device__ __forceinline__ int swz(int mn, int k) { return (((mn >> 2) ^ (k & 7)) << 2) | (mn & 3); }

// Element e (0..2047) of a 64 x 32 operand slice: which (mn, k) it is.  kfast = the
// operand's k index is contiguous in memory; then a warp covers 8 k x 4 mn (four 32-byte
// sectors), otherwise 32 consecutive mn.
template <bool kfast>
__device__ __forceinline__ void slice_pos(int e, int& mn, int& k) {
  if (kfast) {
    const int rest = e >> 5;
    k = (e & 7) + 8 * (rest & 3);
    mn = ((e >> 3) & 3) + 4 * (rest >> 2);
  } else {
    mn = e & 63;
    k = e >> 6;
  }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_f32_kernel(GemmF32 g) {
  constexpr int BK = 32;
  __shared__ __align__(16) float As[BK][64];
  __shared__ __align__(16) float Bs[BK][64];
  const float* A = g.A + (int64_t)blockIdx.z * g.sa;
  const float* B = g.B + (int64_t)blockIdx.z * g.sb;
  float* C = g.C + (int64_t)blockIdx.z * g.sc;
  const int64_t m0 = (int64_t)blockIdx.x * 64, n0 = (int64_t)blockIdx.y * 64;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  float acc[4][4] = {};
  float ra[8], rb[8];  // the next K slice, fetched while the current one is multiplied
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = t + 256 * r;
      int mm, kk, nn, kb;
      slice_pos<TA>(e, mm, kk);
      slice_pos<!TB>(e, nn, kb);
      const int64_t gm = m0 + mm, gk = k0 + kk, gn = n0 + nn, gkb = k0 + kb;
      ra[r] = (gm < g.M && gk < g.K) ? (TA ? A[gk + gm * g.lda] : A[gm + gk * g.lda]) : 0.f;
      rb[r] = (gn < g.N && gkb < g.K) ? (TB ? B[gn + gkb * g.ldb] : B[gkb + gn * g.ldb]) : 0.f;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = t + 256 * r;
      int mm, kk, nn, kb;
      slice_pos<TA>(e, mm, kk);
      slice_pos<!TB>(e, nn, kb);
      As[kk][swz(mm, kk)] = ra[r];
      Bs[kb][swz(nn, kb)] = rb[r];
    }
  };
  fetch(0);
  stash();
  __syncthreads();
  for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
    const bool more = k0 + BK < g.K;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][swz(4 * ty, kk)]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][swz(4 * tx, kk)]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (more) {
      stash();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + 4 * ty + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + 4 * tx + j;
      if (gn >= g.N) continue;
      float* c = C + gm + gn * g.ldc;
      *c = g.beta == 0.f ? g.alpha * acc[i][j] : fmaf(g.alpha, acc[i][j], g.beta * *c);
    }
  }
}

cudaError_t gemm_f32(bool ta, bool tb, const GemmF32& g, int64_t batch, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((g.M + 63) / 64), (unsigned)((g.N + 63) / 64), (unsigned)batch);
  if (ta && !tb) gemm_f32_kernel<true, false><<<grid, 256, 0, s>>>(g);
  else if (!ta && !tb) gemm_f32_kernel<false, false><<<grid, 256, 0, s>>>(g);
  else if (!ta && tb) gemm_f32_kernel<false, true><<<grid, 256, 0, s>>>(g);
  else gemm_f32_kernel<true, true><<<grid, 256, 0, s>>>(g);
  note_launch();
  return cudaGetLastError();
}

// L32 = lower triangle of L (FP64 -> FP32), zeros above.
__global__ void lower_f32_kernel(int64_t n, const double* __restrict__ L, float* __restrict__ L32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (uint32_t)e % (uint32_t)n, j = (uint32_t)e / (uint32_t)n;
    L32[e] = i >= j ? (float)L[e] : 0.f;
  }
}

cudaError_t lower_to_f32(int64_t n, const double* M, float* L32, cudaStream_t s) {
  lower_f32_kernel<<<grid_small(n * n), 256, 0, s>>>(n, M, L32);
  note_launch();
  return cudaGetLastError();
}

// Diagonal 32 x 32 blocks of X := their inverses (Dinv, stored block after block).
__global__ void place_diag_f32_kernel(int64_t n, const float* __restrict__ Dinv, float* __restrict__ X) {
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
    const int a = e & 31, b = e >> 5;
    if (i0 + a < n && i0 + b < n) X[(i0 + a) + (i0 + b) * n] = Dinv[(size_t)blockIdx.x * 1024 + a + 32 * b];
  }
}

// X := L^{-1} in place (X holds L, lower, zeros above; W is n x n scratch).  Starting
// from inverted 32 x 32 diagonal blocks, adjacent s x s inverted blocks are merged into
// 2s x 2s ones: [A 0; L21 C]^{-1} has off-diagonal block -C^{-1} L21 A^{-1}, two GEMMs
// per merge, all merges of one size in one batched launch.
cudaError_t tri_inverse_f32(int64_t n, float* X, float* W, float* Dinv, cudaStream_t s) {
  const int nblk = (int)((n + 31) / 32);
  cudaError_t e = diag_block_inverse_f32(n, X, Dinv, s);
  if (e != cudaSuccess) return e;
  place_diag_f32_kernel<<<nblk, 256, 0, s>>>(n, Dinv, X);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int64_t sz = 32; sz < n; sz *= 2) {
    const int64_t full = n / (2 * sz);         // merges with two full sz blocks
    const int64_t tail0 = full * 2 * sz;       // a last, shorter merge starts here
    for (int part = 0; part < 2; ++part) {
      const int64_t i0 = part == 0 ? 0 : tail0;
      const int64_t batch = part == 0 ? full : (tail0 + sz < n ? 1 : 0);
      if (batch == 0) continue;
      const int64_t s2 = part == 0 ? sz : n - tail0 - sz;  // rows of the lower block
      const int64_t stride = 2 * sz * (n + 1);
      const int64_t a11 = i0 + i0 * n, a21 = (i0 + sz) + i0 * n, a22 = (i0 + sz) + (i0 + sz) * n;
      GemmF32 g1{s2, sz, sz, n, n, n, stride, stride, stride, X + a21, X + a11, W + a21, 1.f, 0.f};
      if ((e = gemm_f32(false, false, g1, batch, s)) != cudaSuccess) return e;   // W21 = L21 A^{-1}
      GemmF32 g2{s2, sz, s2, n, n, n, stride, stride, stride, X + a22, W + a21, X + a21, -1.f, 0.f};
      if ((e = gemm_f32(false, false, g2, batch, s)) != cudaSuccess) return e;   // X21 = -C^{-1} W21
    }
  }
  return cudaSuccess;
}

cudaError_t convert_f64_to_f32(int64_t count, const double* src, float* dst, cudaStream_t s) {
  f64_to_f32_kernel<<<grid_small(count), 256, 0, s>>>(count, src, dst);
  note_launch();
  return cudaGetLastError();
}

cudaError_t mixed_setup(int64_t n, const double* L, const double* G2, int precision, float* L32, float* P32,
                        float* G2_32, float* Bt32, void* Bt16, float* Dinv32, cudaStream_t s) {
  const int64_t nn = n * n;
  if (L) {
    lower_f32_kernel<<<grid_small(nn), 256, 0, s>>>(n, L, L32);
    note_launch();
  }
  if (G2) {
    f64_to_f32_kernel<<<grid_small(nn), 256, 0, s>>>(nn, G2, G2_32);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // P = L^{-T} L^{-1} in FP32 from the Cholesky factor: L32 := L^{-1} (P32 serves as the
  // merge scratch), then P = (L^{-1})^T L^{-1}.
  if ((e = tri_inverse_f32(n, L32, P32, Dinv32, s)) != cudaSuccess) return e;
  GemmF32 gp{n, n, n, n, n, n, 0, 0, 0, L32, L32, P32, 1.f, 0.f};
  if ((e = gemm_f32(true, false, gp, 1, s)) != cudaSuccess) return e;
  if (!G2) return cudaSuccess;  // matrix-free route: B is never formed
  return mixed_setup_b(n, nullptr, precision, P32, G2_32, Bt32, Bt16, s);
}

// C = A B for n x n column-major FP32 matrices: 32 x 32 output tiles (n = 500 gives 256
// CTAs, more than the 64 of the 64 x 64 kernel), 2 x 2 outputs per thread, 32-deep K
// slices in shared memory with the next slice fetched into registers meanwhile.
__global__ void __launch_bounds__(256) gemm_nn32_f32_kernel(int64_t n, const float* __restrict__ A,
                                                            const float* __restrict__ B, float* __restrict__ C) {
  __shared__ __align__(16) float As[32][33];  // [k][m]
  __shared__ __align__(16) float Bs[32][33];  // [k][n]
  const int64_t m0 = (int64_t)blockIdx.x * 32, n0 = (int64_t)blockIdx.y * 32;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[2][2] = {};
  float ra[4], rb[4];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int lo = e & 31, hi = e >> 5;  // A: (m = lo, k = hi); B: (k = lo, n = hi)
      ra[q] = (m0 + lo < n && k0 + hi < n) ? A[(m0 + lo) + (k0 + hi) * n] : 0.f;
      rb[q] = (k0 + lo < n && n0 + hi < n) ? B[(k0 + lo) + (n0 + hi) * n] : 0.f;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int lo = e & 31, hi = e >> 5;
      As[hi][lo] = ra[q];
      Bs[lo][hi] = rb[q];
    }
  };
  fetch(0);
  stash();
  __syncthreads();
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
    const bool more = k0 + 32 < n;
    if (more) fetch(k0 + 32);
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
      const float a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
      const float b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
    if (more) {
      stash();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int64_t gm = m0 + 2 * ty + i, gn = n0 + 2 * tx + j;
      if (gm < n && gn < n) C[gm + gn * n] = acc[i][j];
    }
}

cudaError_t mixed_setup_b(int64_t n, const double* G2, int precision, const float* P32, float* G2_32, float* Bt32,
                          void* Bt16, cudaStream_t s) {
  const int64_t nn = n * n;
  cudaError_t e;
  if (G2) {
    f64_to_f32_kernel<<<grid_small(nn), 256, 0, s>>>(nn, G2, G2_32);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // B^T = Abar2 P (both symmetric), so column i of B^T is row i of B = P Abar2.
  const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
  gemm_nn32_f32_kernel<<<grid, 256, 0, s>>>(n, G2_32, P32, Bt32);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (precision == ILS_BF16_REFINE) {
    f32_to_bf16_kernel<<<grid_small(nn), 256, 0, s>>>(nn, Bt32, static_cast<__nv_bfloat16*>(Bt16));
    note_launch();
    e = cudaGetLastError();
  }
  return e;
}

// ---------------------------------------------------------------------------------------
// Sweep-shape autotuner.  For each (n rounded up to 32, k class, operator type) the first
// setup that needs it times every candidate shape on the handle's own operators and keeps
// the fastest for the rest of the process.  Candidates: 1, 2, 4 or 8 warps per CTA, with
// one, two or four rows per warp in the first wave (CTAs = ceil(n / (warps x rows))).
// ---------------------------------------------------------------------------------------
namespace {
struct TuneKey {
  int64_t nb;
  int kc;
  int bf16;
  bool operator<(const TuneKey& o) const {
    return nb != o.nb ? nb < o.nb : (kc != o.kc ? kc < o.kc : bf16 < o.bf16);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, SweepShape> g_tune;

TuneKey tune_key(int64_t n, int64_t k, bool bf16) { return TuneKey{(n + 31) / 32, k <= 2 ? 1 : 8, bf16 ? 1 : 0}; }

SweepShape default_shape(int64_t n) {
  return SweepShape{2, (int32_t)std::max<int64_t>(1, std::min<int64_t>((n + 1) / 2, 1024))};
}

template <typename TM>
cudaError_t time_shape(const MixedArgs& a, SweepShape sh, const TM* M, const float* v, float* out, cudaStream_t s,
                       float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    for (int r = 0; r < 2; ++r) launch_sweep<TM>(a, sh, M, v, nullptr, out, s);
    cudaEventRecord(e0, s);
    for (int r = 0; r < 5; ++r) launch_sweep<TM>(a, sh, M, v, nullptr, out, s);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e == cudaSuccess ? cudaGetLastError() : e;
}
}  // namespace

// The autotuner's choices kept in a text file between processes: a header line naming the
// GPU (model and SM count; a file from another GPU is ignored) and one line per key,
// "nb k_class bf16 warps blocks".
std::string tune_device_tag() {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "";
  }
  std::string name(prop.name);
  for (char& c : name)
    if (c == ' ' || c == '\n') c = '_';
  return "ils-sweep-tune-v1 " + std::to_string(prop.multiProcessorCount) + " " + name;
}

void load_tune_cache(const char* path) {
  if (!path || !*path) return;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  const std::string tag = tune_device_tag();
  if (!std::fgets(line, sizeof(line), f) || tag.empty() || std::string(line).rfind(tag, 0) != 0) {
    std::fclose(f);
    return;
  }
  long long nb;
  int kc, bf, w, b;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  while (std::fscanf(f, "%lld %d %d %d %d", &nb, &kc, &bf, &w, &b) == 5) {
    if (nb < 1 || (kc != 1 && kc != 8) || (bf != 0 && bf != 1) || (w != 1 && w != 2 && w != 4 && w != 8) || b < 1)
      continue;  // a damaged line is ignored
    g_tune.emplace(TuneKey{nb, kc, bf}, SweepShape{w, b});
  }
  std::fclose(f);
}

void save_tune_cache(const char* path) {
  if (!path || !*path) return;
  const std::string tag = tune_device_tag();
  if (tag.empty()) return;
  const std::string tmp = std::string(path) + ".tmp";
  std::FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "%s\n", tag.c_str());
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : g_tune)
      std::fprintf(f, "%lld %d %d %d %d\n", (long long)kv.first.nb, kv.first.kc, kv.first.bf16, kv.second.warps,
                   kv.second.blocks);
  }
  const bool ok = std::fclose(f) == 0;
  if (ok) std::rename(tmp.c_str(), path);
  else std::remove(tmp.c_str());
}

SweepShape sweep_shape(int64_t n, int64_t k, bool bf16) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(tune_key(n, k, bf16));
  return it != g_tune.end() ? it->second : default_shape(n);
}

bool sweeps_tuned(int64_t n, int precision) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  bool all = g_tune.count(tune_key(n, 1, false)) && g_tune.count(tune_key(n, 8, false));
  if (precision == ILS_BF16_REFINE) all = all && g_tune.count(tune_key(n, 1, true)) && g_tune.count(tune_key(n, 8, true));
  return all;
}

cudaError_t tune_sweeps(int64_t n, int precision, const float* P32, const float* Bt32, const void* Bt16,
                        float* scratch_in, float* scratch_out, SolveState* st, cudaStream_t s, const char* cache) {
  load_tune_cache(cache);
  const bool all = sweeps_tuned(n, precision);
  if (all) {  // tuned earlier in this process: the file still receives every key
    save_tune_cache(cache);  // takes g_tune_mu itself
    return cudaSuccess;
  }
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(SolveState), s);  // done = 0: the kernels run
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(scratch_in, 0, sizeof(float) * n * kMaxRhsPerPass, s)) != cudaSuccess) return e;
  for (int bf = 0; bf < 2; ++bf) {
    const bool bf16 = bf == 1;
    if (bf16 && precision != ILS_BF16_REFINE) continue;
    for (int64_t k : {1, 8}) {
      const TuneKey key = tune_key(n, k, bf16);
      {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (g_tune.count(key)) continue;
      }
      MixedArgs a{};
      a.n = n;
      a.k = k;
      a.st = st;
      SweepShape best = default_shape(n);
      float best_ms = 1e30f;
      for (int warps : {1, 2, 4, 8}) {
        for (int rows : {1, 2, 4}) {
          const SweepShape sh{warps, (int32_t)std::max<int64_t>(1, (n + warps * rows - 1) / (warps * rows))};
          float ms = 0.f;
          e = bf16 ? time_shape<__nv_bfloat16>(a, sh, static_cast<const __nv_bfloat16*>(Bt16), scratch_in,
                                               scratch_out, s, &ms)
                   : time_shape<float>(a, sh, Bt32 ? Bt32 : P32, scratch_in, scratch_out, s, &ms);
          if (e != cudaSuccess) return e;
          if (ms < best_ms) {
            best_ms = ms;
            best = sh;
          }
        }
      }
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[key] = best;
    }
  }
  save_tune_cache(cache);
  return cudaSuccess;
}

int ils_tuned_shape_impl(int64_t n, int64_t k, int bf16, int* warps, int* blocks) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(tune_key(n, k, bf16 != 0));
  if (it == g_tune.end()) return 0;
  if (warps) *warps = it->second.warps;
  if (blocks) *blocks = it->second.blocks;
  return 1;
}

// One refinement step after the residual launch: r32, d_1 = P r, d_{s+1} = B d_s + P r, x += d.
cudaError_t mixed_correct(const MixedArgs& a, int precision, cudaStream_t s) {
  const SweepShape sh32 = sweep_shape(a.n, a.k, false);
  // c = P r, read straight from the FP64 residual (kept in a.c32; also the first iterate
  // d_1); the last sweep adds d to x.
  launch_sweep<float, double>(a, sh32, a.P32, a.r, nullptr, a.c32, s, a.sweeps == 1 ? 1 : 0);
  const float* dcur = a.c32;
  float* bufs[2] = {a.d32[0], a.d32[1]};
  for (int sw = 1; sw < a.sweeps; ++sw) {
    float* dn = bufs[sw & 1];
    const int last = sw + 1 == a.sweeps ? 1 : 0;
    if (precision == ILS_BF16_REFINE)
      launch_sweep<__nv_bfloat16>(a, sweep_shape(a.n, a.k, true), static_cast<const __nv_bfloat16*>(a.Bt16), dcur,
                                  a.c32, dn, s, last);
    else
      launch_sweep<float>(a, sh32, a.Bt32, dcur, a.c32, dn, s, last);
    dcur = dn;
  }
  return cudaGetLastError();
}

}  // namespace ils

namespace ils {

// Matrix-free refinement step: d_1 = P r, d_{s+1} = P (A_2^T A_2 d_s + r) with the product
// streamed from the FP32/BF16 copy of A_2, then x += d.
cudaError_t mixed_correct_mf(const MixedArgs& a, int precision, int64_t q, const void* Aq_lo, void* part, double* v,
                             double* d64, float* t32, cudaStream_t s) {
  residual_to_f32_kernel<<<grid_small(a.n * a.k), 256, 0, s>>>(a);
  note_launch();
  const SweepShape sh32 = sweep_shape(a.n, a.k, false);
  launch_sweep<float>(a, sh32, a.P32, a.r32, nullptr, a.c32, s);
  const float* dcur = a.c32;
  float* bufs[2] = {a.d32[0], a.d32[1]};
  const int prec = precision == ILS_BF16_REFINE ? 2 : 1;
  for (int sw = 1; sw < a.sweeps; ++sw) {
    widen_kernel<<<grid_small(a.n * a.k), 256, 0, s>>>(a, dcur, d64);
    note_launch();
    for (int c = 0; c < (int)a.k; ++c) {
      cudaError_t e = aq_product_iterate(q, a.n, Aq_lo, prec, d64, d64, a.st, a.col_done, c, part, v + c * a.n, s);
      if (e != cudaSuccess) return e;
    }
    sweep_rhs_kernel<<<grid_small(a.n * a.k), 256, 0, s>>>(a, v, t32);
    note_launch();
    float* dn = bufs[sw & 1];
    launch_sweep<float>(a, sh32, a.P32, t32, nullptr, dn, s);
    dcur = dn;
  }
  refine_update_kernel<<<grid_small(a.n * a.k), 256, 0, s>>>(a, dcur);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
