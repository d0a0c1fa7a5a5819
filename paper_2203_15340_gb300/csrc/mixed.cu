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

__global__ void identity_f32_kernel(int64_t n, float* M) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
    M[e] = ((uint32_t)e % (uint32_t)n == (uint32_t)e / (uint32_t)n) ? 1.f : 0.f;
}

// C = X^T Y in FP32 (X, Y n x n column-major): 32 x 32 tiles, one output per thread.
__global__ void __launch_bounds__(256) gemm_tn_f32_kernel(int64_t n, const float* __restrict__ X,
                                                          const float* __restrict__ Y, float* __restrict__ C) {
  __shared__ float Xs[32][33];
  __shared__ float Ys[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // ty in 0..7
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int64_t k = k0 + tx;
      Xs[rr][tx] = (k < n && i0 + rr < n) ? X[k + (i0 + rr) * n] : 0.f;
      Ys[rr][tx] = (k < n && j0 + rr < n) ? Y[k + (j0 + rr) * n] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float yv = Ys[tx][kk];
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a] = fmaf(Xs[ty + 8 * a][kk], yv, acc[a]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t gi = i0 + ty + 8 * a, gj = j0 + tx;
    if (gi < n && gj < n) C[gi + gj * n] = acc[a];
  }
}

// Operator element loads for the sweep GEMV (FP32 or BF16 storage, FP32 arithmetic).
__device__ __forceinline__ float ld_op(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ld_op(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

constexpr int kSweepWarps = 2;

// out(:,c) = M^T v(:,c) (+ add(:,c)); column i of M is row i of the operator.  KR is the
// number of right-hand sides, fixed at compile time so no predicated work is issued.
template <typename TM, int KR>
__global__ void __launch_bounds__(32 * kSweepWarps) sweep_kernel(MixedArgs a, const TM* __restrict__ M,
                                                                 const float* __restrict__ v,
                                                                 const float* __restrict__ add,
                                                                 float* __restrict__ out) {
  if (*((volatile int32_t*)&a.st->done)) return;
  const int64_t n = a.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * kSweepWarps + w; i < n; i += (int64_t)gridDim.x * kSweepWarps) {
    const TM* col = M + i * n;
    float acc[KR];
#pragma unroll
    for (int c = 0; c < KR; ++c) acc[c] = 0.f;
    for (int64_t j = lane; j < n; j += 32) {
      const float mv = ld_op(col, j);
#pragma unroll
      for (int c = 0; c < KR; ++c) acc[c] = fmaf(mv, v[j + c * n], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < KR; ++c) {
      const float sv = warp_sum_f(acc[c]);
      if (lane == 0) out[i + c * n] = sv + (add ? add[i + c * n] : 0.f);
    }
  }
}

template <typename TM>
void launch_sweep(const MixedArgs& a, int blocks, const TM* M, const float* v, const float* add, float* out,
                  cudaStream_t s) {
  switch ((int)a.k) {
    case 1: sweep_kernel<TM, 1><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
    case 2: sweep_kernel<TM, 2><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
    case 3: sweep_kernel<TM, 3><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
    case 4: sweep_kernel<TM, 4><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
    case 5: sweep_kernel<TM, 5><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
    case 6: sweep_kernel<TM, 6><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
    case 7: sweep_kernel<TM, 7><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
    default: sweep_kernel<TM, 8><<<blocks, 32 * kSweepWarps, 0, s>>>(a, M, v, add, out); break;
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

cudaError_t mixed_setup(int64_t n, const double* L, const double* G2, int precision, float* L32, float* P32,
                        float* G2_32, float* Bt32, void* Bt16, float* Dinv32, cudaStream_t s) {
  const int64_t nn = n * n;
  f64_to_f32_kernel<<<grid_small(nn), 256, 0, s>>>(nn, L, L32);
  note_launch();
  if (G2) {
    f64_to_f32_kernel<<<grid_small(nn), 256, 0, s>>>(nn, G2, G2_32);
    note_launch();
  }
  identity_f32_kernel<<<grid_small(nn), 256, 0, s>>>(n, P32);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // P = L^{-T} L^{-1} in FP32 from the FP64 Cholesky factor.
  if ((e = trsm_binv_f32(n, n, L32, Dinv32, P32, n, true, true, s)) != cudaSuccess) return e;
  if (!G2) return cudaSuccess;  // matrix-free route: B is never formed
  // B^T = Abar2 P (both symmetric), so column i of B^T is row i of B = P Abar2.
  const unsigned nt = (unsigned)((n + 31) / 32);
  gemm_tn_f32_kernel<<<dim3(nt, nt), 256, 0, s>>>(n, G2_32, P32, Bt32);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (precision == ILS_BF16_REFINE) {
    f32_to_bf16_kernel<<<grid_small(nn), 256, 0, s>>>(nn, Bt32, static_cast<__nv_bfloat16*>(Bt16));
    note_launch();
    e = cudaGetLastError();
  }
  return e;
}

int mixed_sweep_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kSweepWarps - 1) / kSweepWarps, 1024));
}

// One refinement step after the residual launch: r32, d_1 = P r, d_{s+1} = B d_s + P r, x += d.
cudaError_t mixed_correct(const MixedArgs& a, int precision, cudaStream_t s) {
  residual_to_f32_kernel<<<grid_small(a.n * a.k), 256, 0, s>>>(a);
  note_launch();
  const int blocks = mixed_sweep_blocks(a.n);
  // c = P r  (kept in a.c32; also the first iterate d_1)
  launch_sweep<float>(a, blocks, a.P32, a.r32, nullptr, a.c32, s);
  const float* dcur = a.c32;
  float* bufs[2] = {a.d32[0], a.d32[1]};
  for (int sw = 1; sw < a.sweeps; ++sw) {
    float* dn = bufs[sw & 1];
    if (precision == ILS_BF16_REFINE)
      launch_sweep<__nv_bfloat16>(a, blocks, static_cast<const __nv_bfloat16*>(a.Bt16), dcur, a.c32, dn, s);
    else
      launch_sweep<float>(a, blocks, a.Bt32, dcur, a.c32, dn, s);
    dcur = dn;
  }
  refine_update_kernel<<<grid_small(a.n * a.k), 256, 0, s>>>(a, dcur);
  note_launch();
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
  const int blocks = mixed_sweep_blocks(a.n);
  launch_sweep<float>(a, blocks, a.P32, a.r32, nullptr, a.c32, s);
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
    launch_sweep<float>(a, blocks, a.P32, t32, nullptr, dn, s);
    dcur = dn;
  }
  refine_update_kernel<<<grid_small(a.n * a.k), 256, 0, s>>>(a, dcur);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
