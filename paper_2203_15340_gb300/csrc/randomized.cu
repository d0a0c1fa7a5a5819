// Inner randomized solvers of SP-RK-RGS (Alg. 2 steps 7-12) and SP-SCD (Alg. 5 steps
// 6-12).  Each inner solve is a sequential chain of cheap steps, so one CTA runs one
// chain (one right-hand side) and keeps its vectors in shared memory; independent
// chains run on different SMs.  Random draws come from Philox4x32-10 with the counter
// layout (t_lo, t_hi, k, chain) and key (seed_lo, seed_hi).
#include <cmath>

#include "ils_internal.h"
#include "philox.cuh"

namespace ils {
namespace {

// Smallest j with cum[j] > u * cum[n-1] (inverse CDF of the column law of Alg. 2 steps 8/10).
__device__ __forceinline__ int invcdf_pick(const double* cum, int n, double u) {
  const double thr = u * cum[n - 1];
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cum[mid] > thr) hi = mid;
    else lo = mid + 1;
  }
  return lo < n ? lo : n - 1;
}

// Rank i in 1..n with P(i) = (n+1)/(n i (i+1)): the law of the position (in decreasing
// |r|) of the index Alg. 5 picks when alpha ~ U{1..n} and the alpha-subset is uniform.
__device__ __forceinline__ int scd_rank(double u, int n) {
  const double num = u * (double)n;
  double i = ceil(num / ((double)(n + 1) - num));
  if (i < 1.0) i = 1.0;
  if (i > (double)n) i = (double)n;
  return (int)i;
}

constexpr int kChainThreads = 512;
constexpr int kChainWarps = kChainThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum, result broadcast to every thread.  red has kChainWarps + 1 slots.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // red may still be read from the previous call
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < kChainWarps ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[kChainWarps] = t;
  }
  __syncthreads();
  return red[kChainWarps];
}

// Key order of the SCD selection: larger |r| first, then lower index.  |r| is compared
// through its bit pattern (for non-negative doubles the unsigned integer order is the
// numeric order), so the selection uses the integer pipes, not the scarce FP64 one.
__device__ __forceinline__ bool key_greater(unsigned long long a, int i, unsigned long long b, int j) {
  return a > b || (a == b && i < j);
}

__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// Index of the i-th largest |r_s| (ties to the lowest index) by i rounds of a block
// argmax restricted to keys below the previous round's key.  The expected number of
// rounds under the rank law is about ln(n).  NaN entries are never picked; returns -1 if
// r holds no entry that can be.
__device__ int select_ith_largest(const double* r, int n, int i, unsigned long long* red_a, int* red_i) {
  constexpr unsigned long long kNaN = 0x7ff0000000000000ull;  // keys above this are NaN
  unsigned long long prev_a = ~0ull;
  int prev_i = -1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int round = 0; round < i; ++round) {
    unsigned long long best_a = 0ull;
    int best_i = n;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
      const unsigned long long a = abs_key(r[s]);
      const bool below = a < prev_a || (a == prev_a && s > prev_i);
      if (a <= kNaN && below && key_greater(a, s, best_a, best_i)) {
        best_a = a;
        best_i = s;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long oa = __shfl_xor_sync(0xffffffffu, best_a, o);
      const int oi = __shfl_xor_sync(0xffffffffu, best_i, o);
      if (key_greater(oa, oi, best_a, best_i)) {
        best_a = oa;
        best_i = oi;
      }
    }
    __syncthreads();
    if (lane == 0) {
      red_a[w] = best_a;
      red_i[w] = best_i;
    }
    __syncthreads();
    if (w == 0) {
      unsigned long long a = lane < kChainWarps ? red_a[lane] : 0ull;
      int ii = lane < kChainWarps ? red_i[lane] : n;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long oa = __shfl_xor_sync(0xffffffffu, a, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ii, o);
        if (key_greater(oa, oi, a, ii)) {
          a = oa;
          ii = oi;
        }
      }
      if (lane == 0) {
        red_a[kChainWarps] = a;
        red_i[kChainWarps] = ii;
      }
    }
    __syncthreads();
    prev_a = red_a[kChainWarps];
    prev_i = red_i[kChainWarps];
    if (prev_i >= n) return -1;
  }
  return prev_i;
}

// ---------------------------------------------------------------------------------------
// SP-SCD inner chain (Alg. 5 steps 5-12) for column blockIdx.x of the pass.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kChainThreads) scd_chain_kernel(RandArgs a) {
  const int c = blockIdx.x;
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done) || a.col_done[c]) return;
  const int n = (int)a.n;
  const int cur = *((volatile int32_t*)&st->cur);
  double* xout = (cur ? a.X1 : a.X0) + (size_t)c * n;
  const uint32_t k = (uint32_t)(st->iters - 1);  // outer index of the iterate being built
  extern __shared__ double smem[];
  double* r = smem;
  double* beta = smem + n;
  __shared__ double red[kChainWarps + 1];
  __shared__ unsigned long long red_a[kChainWarps + 1];
  __shared__ int red_i[kChainWarps + 1];
  const double* bhat = a.bhat + (size_t)c * n;
  double part = 0.0;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const double v = bhat[s];  // r_0 = bhat - Abar1 * 0 (step 5)
    r[s] = v;
    beta[s] = 0.0;
    part = fma(v, v, part);
  }
  double rr = block_sum(part, red);
  const double target2 = a.col_target2[c];
  int64_t t = 0;
  for (; t < a.max_inner; ++t) {
    if (rr <= target2) break;
    int i = 1;
    if (!a.greedy) {
      double u0, u1;
      step_uniforms(a.seed, (uint32_t)(a.chain0 + c), k, (uint64_t)t, &u0, &u1);
      i = scd_rank(u0, n);
    }
    const int j = select_ith_largest(r, n, i, red_a, red_i);
    if (j < 0) {
      if (threadIdx.x == 0) atomicCAS(&st->status, 0, ILS_ERR_NONFINITE);
      break;
    }
    const double* gj = a.G1 + (size_t)j * n;
    const double delta = r[j] / gj[j];  // steps 10-11: r_j / Abar1_jj
    __syncthreads();
    if (threadIdx.x == 0) beta[j] += delta;
    part = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
      const double v = fma(-delta, gj[s], r[s]);
      r[s] = v;
      part = fma(v, v, part);
    }
    rr = block_sum(part, red);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) xout[s] = beta[s];  // x_{k+1} = beta (step 13)
  if (threadIdx.x == 0) a.col_inner[c] += t;
}

// ---------------------------------------------------------------------------------------
// SP-RK-RGS inner chain (Alg. 2 steps 6-12) for column blockIdx.x of the pass.
// w (length p) and the maintained e = w - A_1 z live in shared memory when they fit,
// otherwise in a global scratch slice of the chain.  The RGS step reads A_1^T (w - A_1 z)
// restricted to column j2, which is A_1(:,j2)^T e.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kChainThreads) rkrgs_chain_kernel(RandArgs a) {
  const int c = blockIdx.x;
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done) || a.col_done[c]) return;
  const int n = (int)a.n;
  const int64_t p = a.p, m = a.m;
  const int cur = *((volatile int32_t*)&st->cur);
  double* xout = (cur ? a.X1 : a.X0) + (size_t)c * n;
  const uint32_t k = (uint32_t)(st->iters - 1);
  extern __shared__ double smem[];
  double* z = smem;             // n
  double* cum = smem + n;       // n
  double* w;
  double* e;
  if (a.vec_in_smem) {
    w = smem + 2 * n;
    e = w + p;
  } else {
    w = a.vec_scratch + (size_t)c * 2 * p;
    e = w + p;
  }
  __shared__ double red[kChainWarps + 1];
  const double* bhat = a.bhat + (size_t)c * n;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    z[s] = 0.0;
    cum[s] = a.cum[s];
  }
  for (int64_t r = threadIdx.x; r < p; r += blockDim.x) {
    w[r] = 0.0;
    e[r] = 0.0;
  }
  __syncthreads();
  const double target2 = a.col_target2[c];
  const int64_t check = a.check_every;
  int64_t t = 0;
  bool stop = false;
  for (; t < a.max_inner && !stop; ++t) {
    double u0, u1;
    step_uniforms(a.seed, (uint32_t)(a.chain0 + c), k, (uint64_t)t, &u0, &u1);
    const int j1 = invcdf_pick(cum, n, u0);
    const int j2 = a.same_index ? j1 : invcdf_pick(cum, n, u1);
    // RK step on A_1^T w = bhat (step 9).
    const double* a1 = a.A + (size_t)j1 * m;
    double part = 0.0;
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) part = fma(a1[r], w[r], part);
    const double dot1 = block_sum(part, red);
    const double delta = (bhat[j1] - dot1) / a.norms2[j1];
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) {
      const double av = a1[r];
      w[r] = fma(delta, av, w[r]);
      e[r] = fma(delta, av, e[r]);
    }
    // RGS step on A_1 z = w with the updated w (step 11).
    const double* a2 = a.A + (size_t)j2 * m;
    part = 0.0;
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) part = fma(a2[r], e[r], part);
    const double dot2 = block_sum(part, red);
    const double eps = dot2 / a.norms2[j2];
    if (threadIdx.x == 0) z[j2] += eps;
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) e[r] = fma(-eps, a2[r], e[r]);
    if ((t + 1) % check == 0) {
      // Inner stop test: ||bhat - Abar1 z||^2 <= target2.
      __syncthreads();
      part = 0.0;
      for (int row = threadIdx.x; row < n; row += blockDim.x) {
        const double* g = a.G1 + (size_t)row * n;  // column `row` = row `row` (symmetric)
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = fma(g[j], z[j], acc);
        const double rv = bhat[row] - acc;
        part = fma(rv, rv, part);
      }
      const double res2 = block_sum(part, red);
      if (res2 <= target2) stop = true;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) xout[s] = z[s];  // x_{k+1} = z (step 13)
  if (threadIdx.x == 0) a.col_inner[c] += t;
}

// cum[j] = sum_{i <= j} norms2[i], added left to right; norms2 = diag(Abar1).  The
// diagonal is gathered in parallel; one thread then adds it in order, 32 loads at a time.
__global__ void column_cumsum_kernel(int64_t n, const double* G1, double* norms2, double* cum) {
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) norms2[j] = G1[j + j * n];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    double v[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = (j0 + t < n) ? norms2[j0 + t] : 0.0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (j0 + t < n) {
        s += v[t];
        cum[j0 + t] = s;
      }
    }
  }
}

}  // namespace

cudaError_t column_cumsum_f64(int64_t n, const double* G1, double* norms2, double* cum, cudaStream_t s) {
  column_cumsum_kernel<<<1, 256, 0, s>>>(n, G1, norms2, cum);
  note_launch();
  return cudaGetLastError();
}

size_t rkrgs_smem_bytes(int64_t n, int64_t p, bool vec_in_smem) {
  return sizeof(double) * (size_t)(2 * n + (vec_in_smem ? 2 * p : 0));
}

bool rkrgs_vec_fits(int64_t n, int64_t p) { return rkrgs_smem_bytes(n, p, true) <= 200 * 1024; }

cudaError_t rand_chain_f64(const RandArgs& a, int method, cudaStream_t s) {
  if (method == ILS_SP_SCD) {
    const size_t smem = sizeof(double) * 2 * (size_t)a.n;
    if (smem > 0) {  // static shared arrays count against the same limit
      cudaError_t e = cudaFuncSetAttribute(scd_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    scd_chain_kernel<<<(unsigned)a.k, kChainThreads, smem, s>>>(a);
    note_launch();
    return cudaGetLastError();
  }
  const size_t smem = rkrgs_smem_bytes(a.n, a.p, a.vec_in_smem != 0);
  if (smem > 0) {  // static shared arrays count against the same limit
    cudaError_t e = cudaFuncSetAttribute(rkrgs_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  rkrgs_chain_kernel<<<(unsigned)a.k, kChainThreads, smem, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
