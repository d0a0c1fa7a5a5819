// Mixed-precision SP solve of one right-hand side in a single cooperative launch.
//
// Each outer step of the refinement (Sec. 5's residual test, then Alg. 1's SP sweeps on the
// correction equation H d = r) is a chain of matrix-vector products that depend on one
// another: r = bbar - H x (FP64), then d_1 = P r and d_{s+1} = B d_s + d_1 (FP32, or B in
// BF16), then x += d_S.  Launched one kernel per product, each product pays a launch and a
// drain; here every product is one phase of a persistent grid, phases separated by a grid
// barrier.  A warp takes whole rows of a product (the operator's column i is its row i,
// as in the sweep kernel).  After each residual every CTA adds the per-CTA partial sums of
// ||r||^2 in the same fixed order, so all CTAs take the same stop decision; the decision
// rule and the state written at the end are those of the launch-per-product path.
// Barrier waits are bounded (1 s, or the handle's wait limit); past that the CTA records TIMEOUT, marks the solve
// done and raises the abort word, which releases every other waiter.
// Under the error-bound stop the refinement need not wait for kappa_est: a provisional
// launch stops on relres <= tol (necessary, as kappa >= 1), and a second launch, ordered
// after the estimate, applies kappa_est relres <= tol to the stored residual and refines
// on only if that fails.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ils_internal.h"

namespace ils {
namespace {

constexpr int kFsThreads = 256;
constexpr int kFsWarps = kFsThreads / 32;

struct FusedArgs {
  int64_t n;
  int32_t sweeps;
  int32_t bf16;
  const double* H;       // n x n symmetric: column i is row i
  const double* bbar;    // A^T J b
  const double* bnorm2;  // ||bbar||^2
  double tol2;
  const double* tol_scale;  // nullptr or a device scalar multiplying tol2
  double* x;             // the iterate, updated in place
  double* r;             // FP64 residual
  float* c32;            // P r
  float* d32[2];         // sweep iterates
  const float* P32;
  const float* Bt32;
  const __nv_bfloat16* Bt16;
  double* partials;      // one per CTA
  int32_t* col_done;
  double* col_rr;
  int64_t* col_iters;
  SolveState* st;
  uint32_t* sync;        // [0] arrivals, [1] generation, [2] abort
  uint64_t wait_ns;      // bound on each barrier wait
  int32_t phase;         // 0: one launch; 1: provisional (stop on tol2 alone); 2: resume after 1
  const float* Hh;       // the row-scaled double-FP32 H (split_rows_df), for the cluster kernel
  const float* Hl;
  const int32_t* He;
  const float* A2_32;    // Abar2 (FP32): sweeps as P (Abar2 d + r) instead of B d + P r (cluster kernel)
};

__device__ __forceinline__ uint32_t fs_ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t fs_ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier (generation counting); false on abort or timeout.
__device__ bool fs_barrier(const FusedArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int res = 1;
    uint32_t* sync = a.sync;
    const uint32_t gen = fs_ld_relaxed(sync + 1);
    __threadfence();
    if (atomicAdd(sync, 1u) == gridDim.x - 1) {
      sync[0] = 0u;
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      uint64_t t0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      const bool short_bound = a.wait_ns < 100000ull;  // a short bound is checked at every poll
      for (uint32_t spin = 0;; ++spin) {
        if (fs_ld_acquire(sync + 1) != gen) break;
        if (short_bound || (spin & 15u) == 15u) {
          if (fs_ld_acquire(sync + 2) != 0u) {
            res = 0;
            break;
          }
          uint64_t t;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
          if (t - t0 > a.wait_ns) {
            atomicCAS(&a.st->status, 0, (int32_t)ILS_ERR_TIMEOUT);
            atomicExch(&a.st->done, 1);
            atomicExch(sync + 2, 1u);
            res = 0;
            break;
          }
        }
        if (spin >= 64u) __nanosleep(32);
      }
    }
    ok = res;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double fs_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float fs_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float fs_op(const float* M, int64_t e) { return __ldg(M + e); }
__device__ __forceinline__ float fs_op(const __nv_bfloat16* M, int64_t e) { return __bfloat162float(M[e]); }
__device__ __forceinline__ float fs_vec(const double* v, int64_t j) { return (float)__ldcg(v + j); }
__device__ __forceinline__ float fs_vec(const float* v, int64_t j) { return __ldcg(v + j); }

// out = M^T v (+ add) in FP32, a warp per row; with x, also x += out.  The CTA first copies
// v into shared memory (vs, n floats), so a row costs one round of independent loads of its
// operator entries.
template <typename TM, typename TV>
__device__ void fs_sweep(int64_t n, const TM* M, const TV* v, const float* add, float* out, double* x, float* vs) {
  const int lane = threadIdx.x & 31;
  for (int64_t j = threadIdx.x; j < n; j += kFsThreads) vs[j] = fs_vec(v, j);
  __syncthreads();
  const int64_t tw = (int64_t)gridDim.x * kFsWarps;
  for (int64_t i = (int64_t)blockIdx.x * kFsWarps + (threadIdx.x >> 5); i < n; i += tw) {
    const TM* col = M + i * n;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int64_t j = lane;
#pragma unroll 4
    for (; j + 96 < n; j += 128) {
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(fs_op(col, j + 32 * u), vs[j + 32 * u], acc[u]);
    }
    for (; j < n; j += 32) acc[0] = fmaf(fs_op(col, j), vs[j], acc[0]);
    const float s = fs_warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
    if (lane == 0) {
      const float o = s + (add ? __ldcg(add + i) : 0.f);
      out[i] = o;
      if (x) x[i] += (double)o;
    }
  }
}

// The same product with the warp's row of M held in registers (R entries per lane, one row
// per warp, n <= 32 R); vs is zero past n.
template <int R, typename TV>
__device__ void fs_sweep_reg(int64_t n, int64_t i, const float (&m)[R], const TV* v, const float* add, float* out,
                             double* x, float* vs) {
  const int lane = threadIdx.x & 31;
  for (int64_t j = threadIdx.x; j < 32 * R; j += kFsThreads) vs[j] = j < n ? fs_vec(v, j) : 0.f;
  __syncthreads();
  if (i >= n) return;
  float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
  for (int u = 0; u < R; u += 2) {
    acc0 = fmaf(m[u], vs[lane + 32 * u], acc0);
    if (u + 1 < R) acc1 = fmaf(m[u + 1], vs[lane + 32 * (u + 1)], acc1);
  }
  const float s = fs_warp_sum(acc0 + acc1);
  if (lane == 0) {
    const float o = s + (add ? __ldcg(add + i) : 0.f);
    out[i] = o;
    if (x) x[i] += (double)o;
  }
}

// R > 0: every warp owns one row and keeps that row of H, P and B in registers for the
// whole solve (n <= 32 R); R = 0: rows are streamed from L2 in every phase.
template <int R>
__global__ void __launch_bounds__(kFsThreads) mixed_solve_fused_kernel(FusedArgs a) {
  const int64_t n = a.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t tw = (int64_t)gridDim.x * kFsWarps;
  __shared__ double red[kFsWarps];
  __shared__ double s_rr;
  extern __shared__ __align__(16) double fs_vec_smem[];  // n values of the phase's input vector
  double* xs = fs_vec_smem;
  float* vs = reinterpret_cast<float*>(fs_vec_smem);
  if (*((volatile int32_t*)&a.st->done)) return;
  int64_t it = *((volatile int64_t*)&a.st->iters);
  const int64_t max_outer = a.st->max_outer;
  // A provisional launch stops on tol2 alone: tol_scale <= 1, so that is necessary for the
  // final rule, which a resuming launch applies to the stored ||r||^2 of the same x.
  const double target = a.tol2 * (a.tol_scale && a.phase != 1 ? *a.tol_scale : 1.0) * a.bnorm2[0];
  bool resume = a.phase == 2 && *((volatile int32_t*)a.col_done) == 2;
  const int64_t row = (int64_t)blockIdx.x * kFsWarps + w;  // the warp's row (R > 0)
  constexpr int RR = R > 0 ? R : 1;
  double hr[RR];
  float pr[RR], br[RR];
  if (R > 0) {
#pragma unroll
    for (int u = 0; u < RR; ++u) {
      const int64_t j = lane + 32 * u;
      const bool ok = row < n && j < n;
      hr[u] = ok ? __ldg(a.H + row * n + j) : 0.0;
      pr[u] = ok ? __ldg(a.P32 + row * n + j) : 0.f;
      br[u] = ok ? (a.bf16 ? __bfloat162float(a.Bt16[row * n + j]) : __ldg(a.Bt32 + row * n + j)) : 0.f;
    }
  }
  for (;;) {
    double rr;
    if (resume) {  // r and ||r||^2 of this x were left by the provisional launch
      resume = false;
      rr = *((volatile double*)a.col_rr);
    } else {
      // r = bbar - H x (FP64) and this CTA's share of ||r||^2
      double rp = 0.0;
      const int64_t nst = R > 0 ? 32 * R : n;  // staged entries (zero past n)
      for (int64_t j = threadIdx.x; j < nst; j += kFsThreads) xs[j] = j < n ? __ldcg(a.x + j) : 0.0;
      __syncthreads();
      if (R > 0) {
        if (row < n) {
          double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
          for (int u = 0; u < RR; u += 2) {
            acc0 = fma(hr[u], xs[lane + 32 * u], acc0);
            if (u + 1 < RR) acc1 = fma(hr[u + 1], xs[lane + 32 * (u + 1)], acc1);
          }
          const double s = fs_warp_sum(acc0 + acc1);
          if (lane == 0) {
            const double r = a.bbar[row] - s;
            a.r[row] = r;
            rp = r * r;
          }
        }
      }
      for (int64_t i = (int64_t)blockIdx.x * kFsWarps + w; R == 0 && i < n; i += tw) {
        const double* hrow = a.H + i * n;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int64_t j = lane;
#pragma unroll 4
        for (; j + 96 < n; j += 128) {
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] = fma(__ldg(hrow + j + 32 * u), xs[j + 32 * u], acc[u]);
        }
        for (; j < n; j += 32) acc[0] = fma(__ldg(hrow + j), xs[j], acc[0]);
        const double s = fs_warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
        if (lane == 0) {
          const double r = a.bbar[i] - s;
          a.r[i] = r;
          rp = fma(r, r, rp);
        }
      }
      if (lane == 0) red[w] = rp;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kFsWarps; ++k) t += red[k];
        a.partials[blockIdx.x] = t;
      }
      if (!fs_barrier(a)) return;
      // ||r||^2: every CTA adds the partials in the same order
      {
        double v = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += kFsThreads) v += __ldcg(a.partials + b);
        v = fs_warp_sum(v);
        if (lane == 0) red[w] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
          double t = 0.0;
          for (int k = 0; k < kFsWarps; ++k) t += red[k];
          s_rr = t;
        }
        __syncthreads();
      }
      rr = s_rr;
    }
    const bool finite = isfinite(rr);
    const bool conv = finite && rr <= target;
    if (conv && a.phase == 1) {  // provisional: the resuming launch decides with the final rule
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.col_rr[0] = rr;
        a.col_iters[0] = it;
        a.st->iters = it;
        a.col_done[0] = 2;
      }
      return;
    }
    if (!finite || conv || it >= max_outer) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.col_done[0] = 1;
        a.col_rr[0] = rr;
        a.col_iters[0] = it;
        if (!finite) atomicCAS(&a.st->status, 0, (int32_t)ILS_ERR_NONFINITE);
        else if (!conv) atomicCAS(&a.st->status, 0, (int32_t)ILS_ERR_NO_CONVERGENCE);
        a.st->iters = it;
        a.st->done = 1;  // the answer is in x (buffer 0)
      }
      return;
    }
    ++it;
    // d_1 = P r; d_{s+1} = B d_s + d_1; the last sweep adds d to x
    const bool one = a.sweeps == 1;
    if (R > 0) fs_sweep_reg<RR>(n, row, pr, (const double*)a.r, (const float*)nullptr, a.c32, one ? a.x : nullptr, vs);
    else fs_sweep(n, a.P32, (const double*)a.r, (const float*)nullptr, a.c32, one ? a.x : nullptr, vs);
    if (!fs_barrier(a)) return;
    const float* dcur = a.c32;
    for (int sw = 1; sw < a.sweeps; ++sw) {
      float* dn = a.d32[sw & 1];
      double* xu = sw + 1 == a.sweeps ? a.x : nullptr;
      if (R > 0) fs_sweep_reg<RR>(n, row, br, dcur, a.c32, dn, xu, vs);
      else if (a.bf16) fs_sweep(n, a.Bt16, dcur, a.c32, dn, xu, vs);
      else fs_sweep(n, a.Bt32, dcur, a.c32, dn, xu, vs);
      if (!fs_barrier(a)) return;
      dcur = dn;
    }
  }
}

// ---------------------------------------------------------------------------------------
// The same refinement on one thread-block cluster (n <= 512): CTA c of CS = ceil(n / 32)
// keeps rows 32 c .. 32 c + 31, their H entries in registers (FP64; warp w holds rows
// 4 w .. 4 w + 3, lane l columns l + 32 u) and their P and B entries in shared memory.
// After every product each CTA writes its 32 results into every CTA's copy of the vector
// (distributed shared memory) and the cluster meets at its hardware barrier: no grid
// barrier, no round trip through L2.  The squared residual is the sum of the CTAs'
// partials in rank order, the same in every CTA, so all take the same decision.  Nothing
// here spins: the barrier is the hardware's, and every CTA reaches each one.
constexpr int kClRows = 32;       // rows per CTA
constexpr int kClRowsPerWarp = 4;
constexpr int kClMaxCtas = 16;

__device__ __forceinline__ void cl_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Store v at the same shared-memory address of CTA `rank` of the cluster.
__device__ __forceinline__ void cl_put(const float* local, uint32_t rank, float v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(cl_smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(remote), "f"(v) : "memory");
}
__device__ __forceinline__ void cl_put(const double* local, uint32_t rank, double v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(cl_smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(v) : "memory");
}

// Lane 0 holds the warp's result v for row i: lanes 0 .. CS-1 write it to every CTA.
template <typename T>
__device__ __forceinline__ void cl_broadcast(T* vec, int64_t i, T v, int cs) {
  const int lane = threadIdx.x & 31;
  v = __shfl_sync(0xffffffffu, v, 0);
  if (lane < cs) cl_put(vec + i, (uint32_t)lane, v);
}

// One FP32 product row block from shared memory: out_q = sum_j M(r_q, j) v_j for the warp's
// rows r_q (M row-major with stride 32 R, zero past n, as is v); results in every lane.
template <int R>
__device__ __forceinline__ void cl_rows_f32(const float* M, const float* v, int w, float (&out)[kClRowsPerWarp]) {
  const int lane = threadIdx.x & 31;
  float acc[kClRowsPerWarp];
#pragma unroll
  for (int q = 0; q < kClRowsPerWarp; ++q) acc[q] = 0.f;
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int j = lane + 32 * u;
    const float vj = v[j];
#pragma unroll
    for (int q = 0; q < kClRowsPerWarp; ++q) acc[q] = fmaf(M[(w * kClRowsPerWarp + q) * 32 * R + j], vj, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < kClRowsPerWarp; ++q) out[q] = fs_warp_sum(acc[q]);
}

// The refinement's stop decision (shared by both kernels' exits): 0 go on, 1 stop, 2
// provisional stop (phase 1: the resuming launch decides with the final rule).
__device__ __forceinline__ int cl_decide(const FusedArgs& a, double rr, double target, int64_t it,
                                         int64_t max_outer) {
  const bool finite = isfinite(rr);
  const bool conv = finite && rr <= target;
  if (conv && a.phase == 1) return 2;
  return (!finite || conv || it >= max_outer) ? 1 : 0;
}

// Rank 0 records the end of the solve (or the provisional stop); every CTA has written its
// rows of x.
__device__ __forceinline__ void cl_finish(const FusedArgs& a, int how, double rr, double target, int64_t it) {
  a.col_rr[0] = rr;
  a.col_iters[0] = it;
  a.st->iters = it;
  if (how == 2) {
    a.col_done[0] = 2;
    return;
  }
  const bool finite = isfinite(rr);
  const bool conv = finite && rr <= target;
  a.col_done[0] = 1;
  if (!finite) atomicCAS(&a.st->status, 0, (int32_t)ILS_ERR_NONFINITE);
  else if (!conv) atomicCAS(&a.st->status, 0, (int32_t)ILS_ERR_NO_CONVERGENCE);
  a.st->done = 1;  // the answer is in x (buffer 0)
}

// (sh, sl) += p + e, with the rounding error of sh + p kept in sl (a double-FP32 sum)
__device__ __forceinline__ void df_add(float& sh, float& sl, float p, float e) {
  const float t = sh + p;
  const float bp = t - sh;
  const float err = (sh - (t - bp)) + (p - bp);
  sh = t;
  sl += err + e;
}

// v 2^k, by one multiplication where 2^k is a normal double (exact unless v 2^k is
// subnormal), else by ldexp.
__device__ __forceinline__ double times_pow2(double v, int k) {
  if (k >= -1022 && k <= 1023) return v * __longlong_as_double((long long)(k + 1023) << 52);
  return ldexp(v, k);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(cl_smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(cl_smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}

// Rows row0 .. row0 + 31 of the n x n row-major FP32 matrix M into S (stride LD, zero past n
// and past the last row), by asynchronous copies (16 bytes where n is a multiple of 4).
template <int LD>
__device__ __forceinline__ void cl_stage_rows(float* S, const float* M, int64_t n, int64_t row0) {
  if ((n & 3) == 0 && ((reinterpret_cast<uintptr_t>(M) & 15) == 0)) {
    for (int e = threadIdx.x; e < kClRows * LD / 4; e += kFsThreads) {
      const int j = 4 * (e % (LD / 4));
      const int64_t i = row0 + e / (LD / 4);
      const int64_t have = (i < n && j < n) ? (n - j < 4 ? n - j : 4) : 0;
      cp_async16(S + 4 * e, have ? M + i * n + j : M, (int)(4 * have));
    }
  } else {
    for (int e = threadIdx.x; e < kClRows * LD; e += kFsThreads) {
      const int j = e % LD;
      const int64_t i = row0 + e / LD;
      const bool ok = i < n && j < n;
      cp_async4(S + e, ok ? M + i * n + j : M, ok ? 4 : 0);
    }
  }
}

// v 2^k in FP32, exact while v 2^k stays normal (in two steps where 2^k itself is not).
__device__ __forceinline__ float times_pow2f(float v, int k) {
  if (k >= -126 && k <= 127) return v * __int_as_float((k + 127) << 23);
  const int k1 = k / 2;
  return (v * __int_as_float((k1 + 127) << 23)) * __int_as_float((k - k1 + 127) << 23);
}

template <int R>
__global__ void __launch_bounds__(kFsThreads, 1) mixed_solve_cluster_kernel(FusedArgs a) {
  constexpr int LD = 32 * R;  // padded length of every vector and matrix row (zero past n)
  const int64_t n = a.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t rank = cl_rank();
  const int cs = (int)gridDim.x;  // the grid is one cluster
  const int64_t row0 = (int64_t)rank * kClRows;
  extern __shared__ __align__(16) double cl_smem[];
  double* part = cl_smem;                                   // kClMaxCtas partial sums
  float* vA = reinterpret_cast<float*>(part + kClMaxCtas);  // LD
  float* vB = vA + LD;                                      // LD
  float* xh = vB + LD;                                      // LD: x 2^-f, leading FP32 part
  float* xl = xh + LD;                                      // LD: and the rest (x during the launch)
  float* Ps = xl + LD;                                      // kClRows x LD
  float* Bs = Ps + kClRows * LD;                            // kClRows x LD
  __shared__ int redi[kFsWarps];
  __shared__ float th[kClRows], tl[kClRows];  // the CTA's row results, for warp 0's FP64 tail
  __shared__ double s_rr;
  __shared__ int s_how, s_f;

  if (*((volatile int32_t*)&a.st->done)) return;  // read before any barrier: the same in every CTA
  int64_t it = *((volatile int64_t*)&a.st->iters);
  const int64_t max_outer = a.st->max_outer;
  const double target = a.tol2 * (a.tol_scale && a.phase != 1 ? *a.tol_scale : 1.0) * a.bnorm2[0];
  bool resume = a.phase == 2 && *((volatile int32_t*)a.col_done) == 2;
  // Warp 0 finishes the CTA's rows in FP64, lane l taking row row0 + l: one FP64
  // instruction for all 32 rows (GB300's FP64 unit is narrow).
  const int64_t my_row = row0 + lane;
  const bool my_ok = w == 0 && my_row < n;
  const double my_b = my_ok ? a.bbar[my_row] : 0.0;
  const int my_e = my_ok ? a.He[my_row] : 0;
  if (resume) {  // decide on the kept residual before loading anything
    const double rr = *((volatile double*)a.col_rr);
    const int how = cl_decide(a, rr, target, it, max_outer);
    if (how != 0) {
      if (rank == 0 && threadIdx.x == 0) cl_finish(a, how, rr, target, it);
      return;
    }
  }

  // this CTA's rows: P and B to shared memory (asynchronous), H (double-FP32) to registers
  cl_stage_rows<LD>(Ps, a.P32, n, row0);
  if (a.A2_32) cl_stage_rows<LD>(Bs, a.A2_32, n, row0);  // Bs holds Abar2's rows in this mode
  else if (!a.bf16) cl_stage_rows<LD>(Bs, a.Bt32, n, row0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (a.bf16 && !a.A2_32) {
    for (int e = threadIdx.x; e < kClRows * LD; e += kFsThreads) {
      const int64_t j = e % LD, i = row0 + e / LD;
      Bs[e] = (i < n && j < n) ? __bfloat162float(a.Bt16[i * n + j]) : 0.f;
    }
  }
  float hh[kClRowsPerWarp][R], hl[kClRowsPerWarp][R];
#pragma unroll
  for (int q = 0; q < kClRowsPerWarp; ++q) {
    const int64_t i = row0 + w * kClRowsPerWarp + q;
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int64_t j = lane + 32 * u;
      const bool ok = i < n && j < n;
      hh[q][u] = ok ? __ldg(a.Hh + i * n + j) : 0.f;
      hl[q][u] = ok ? __ldg(a.Hl + i * n + j) : 0.f;
    }
  }
  // x = 2^f (xh + xl), |x 2^-f| < 1 at the start (f from the largest exponent field of x)
  {
    int m = 0;
    for (int j = threadIdx.x; j < n; j += kFsThreads) m = max(m, (int)((__double_as_longlong(__ldcg(a.x + j)) >> 52) & 0x7FF));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) redi[w] = m;
    __syncthreads();
    m = 0;
#pragma unroll
    for (int k = 0; k < kFsWarps; ++k) m = max(m, redi[k]);
    if (threadIdx.x == 0) s_f = (m == 0 || m == 0x7FF) ? 0 : m - 1022;
    __syncthreads();
  }
  int f = s_f;
  for (int j = threadIdx.x; j < LD; j += kFsThreads) {
    const double xi = j < n ? times_pow2(__ldcg(a.x + j), -f) : 0.0;
    const float hi = __double2float_rn(xi);
    xh[j] = hi;
    xl[j] = __double2float_rn(xi - (double)hi);
    vA[j] = (resume && j < n) ? (float)__ldcg(a.r + j) : 0.f;
    vB[j] = 0.f;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  cl_barrier();  // every CTA is running and initialized before any remote store

  for (;;) {
    double rr;
    if (resume) {  // r (in vA) and ||r||^2 of this x were left by the provisional launch
      resume = false;
      rr = *((volatile double*)a.col_rr);
    } else {
      // Keep x 2^-f within [2^-40, 2^40]: rescale by a power of two (exact) when it drifts
      // (the same decision in every CTA: each holds the whole vector).
      {
        int m = 0;
        for (int j = threadIdx.x; j < n; j += kFsThreads) m = max(m, (__float_as_int(xh[j]) >> 23) & 0xFF);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) redi[w] = m;
        __syncthreads();
        m = 0;
#pragma unroll
        for (int k = 0; k < kFsWarps; ++k) m = max(m, redi[k]);
        if (m != 0 && (m > 127 + 40 || m < 127 - 40)) {
          const int k = m - 126;  // the largest |x 2^-f| becomes < 1
          for (int j = threadIdx.x; j < LD; j += kFsThreads) {
            xh[j] = times_pow2f(xh[j], -k);
            xl[j] = times_pow2f(xl[j], -k);
          }
          f += k;
          __syncthreads();
        }
      }
      // r = bbar - H x for this CTA's rows, H x in double-FP32 (products split exactly by
      // an FMA, cross terms in FP32, sums with their rounding errors carried); r to every
      // CTA's vA, the partial ||r||^2 to part
#pragma unroll
      for (int q = 0; q < kClRowsPerWarp; ++q) {
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const int j = lane + 32 * u;
          const float bh = xh[j], bl = xl[j];
          const float p = hh[q][u] * bh;
          const float e = fmaf(hh[q][u], bl, fmaf(hl[q][u], bh, fmaf(hh[q][u], bh, -p)));
          df_add(sh, sl, p, e);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
          df_add(sh, sl, oh, ol);
        }
        if (lane == 0) {
          th[w * kClRowsPerWarp + q] = sh;
          tl[w * kClRowsPerWarp + q] = sl;
        }
      }
      __syncthreads();
      if (w == 0) {
        double r = 0.0;
        if (my_ok) {
          r = my_b - times_pow2((double)th[lane] + (double)tl[lane], my_e + f);
          a.r[my_row] = r;
          const float r32 = (float)r;
          for (int k = 0; k < cs; ++k) cl_put(vA + my_row, (uint32_t)k, r32);
        }
        double rp = r * r;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rp += __shfl_xor_sync(0xffffffffu, rp, o);
        rp = __shfl_sync(0xffffffffu, rp, 0);  // one value, the same in every CTA
        if (lane < cs) cl_put(part + rank, (uint32_t)lane, rp);
      }
      cl_barrier();
      if (w == 0) {  // the same tree over the same partials in every CTA
        double t = lane < cs ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_rr = t;
      }
      __syncthreads();
      rr = s_rr;
    }
    if (threadIdx.x == 0) s_how = cl_decide(a, rr, target, it, max_outer);
    __syncthreads();
    const int how = s_how;
    if (how != 0) {
      if (my_ok) a.x[my_row] = times_pow2((double)xh[my_row] + (double)xl[my_row], f);
      if (rank == 0 && threadIdx.x == 0) cl_finish(a, how, rr, target, it);
      return;
    }
    ++it;
    // c = d_1 = P r; d_{s+1} = B d_s + c; the last sweep adds d to x and broadcasts x
    float c[kClRowsPerWarp], o[kClRowsPerWarp];
    cl_rows_f32<R>(Ps, vA, w, c);
    const float* vin = vB;
    for (int sw = 0; sw < a.sweeps; ++sw) {
      float* vout = (vin == vB) ? vA : vB;  // vA (r) is free once P r is formed
      if (sw > 0 && a.A2_32) {
        // t = Abar2 d_s to every CTA's vA (free: P r is formed), then d_{s+1} = P t + c
        cl_rows_f32<R>(Bs, vB, w, o);
#pragma unroll
        for (int q = 0; q < kClRowsPerWarp; ++q) {
          const int64_t i = row0 + w * kClRowsPerWarp + q;
          if (i < n) cl_broadcast(vA, i, o[q], cs);
        }
        cl_barrier();
        cl_rows_f32<R>(Ps, vA, w, o);
        vout = vB;  // d_{s+1} goes back to vB (its readers, the product above, are past the barrier)
      } else if (sw > 0) {
        cl_rows_f32<R>(Bs, vin, w, o);
      }
      const bool last = sw + 1 == a.sweeps;
#pragma unroll
      for (int q = 0; q < kClRowsPerWarp; ++q) {
        const int64_t i = row0 + w * kClRowsPerWarp + q;
        const float d = sw > 0 ? o[q] + c[q] : c[q];
        if (last) {
          if (lane == 0) th[w * kClRowsPerWarp + q] = d;
        } else if (i < n) {
          cl_broadcast(sw == 0 ? vB : vout, i, d, cs);
        }
      }
      if (last) {  // x += d in double-FP32 (warp 0, one row per lane), x to every CTA
        __syncthreads();
        if (my_ok) {
          float ph = xh[my_row], pl = xl[my_row];
          df_add(ph, pl, times_pow2f(th[lane], -f), 0.f);
          const float t = ph + pl;
          pl = pl - (t - ph);
          ph = t;
          for (int k = 0; k < cs; ++k) {
            cl_put(xh + my_row, (uint32_t)k, ph);
            cl_put(xl + my_row, (uint32_t)k, pl);
          }
        }
      }
      cl_barrier();
      if (sw > 0) vin = vout;
    }
  }
}

// H(i, j) = 2^e_i (hh + hl): one CTA per row; e_i from the largest exponent field of row i
// (integer work), each scaled entry split into its FP32 rounding and the FP32 rounding of
// the remainder.
__global__ void split_rows_df_kernel(int64_t n, const double* __restrict__ H, float* __restrict__ Hh,
                                     float* __restrict__ Hl, int32_t* __restrict__ He) {
  __shared__ int red[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double* row = H + i * n;
    int m = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
      m = max(m, (int)((__double_as_longlong(row[j]) >> 52) & 0x7FF));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[w] = m;
    __syncthreads();
    m = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = max(m, red[k]);
    const int e = (m == 0 || m == 0x7FF) ? 0 : m - 1022;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double v = times_pow2(row[j], -e);
      const float hi = __double2float_rn(v);
      Hh[i * n + j] = hi;
      Hl[i * n + j] = __double2float_rn(v - (double)hi);
    }
    if (threadIdx.x == 0) He[i] = e;
    __syncthreads();  // red is reused by the next row
  }
}

template <int R>
cudaError_t launch_cluster_solve_r(const FusedArgs& a, int cs, cudaStream_t s) {
  constexpr int LD = 32 * R;
  const size_t smem = sizeof(double) * kClMaxCtas + sizeof(float) * (4 * LD + 2 * kClRows * LD);
  static int checked = 0;  // 1: the cluster fits, -1: it does not (per process)
  if (checked == 0) {
    cudaError_t e = cudaFuncSetAttribute(mixed_solve_cluster_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mixed_solve_cluster_kernel<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      checked = -1;
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kClMaxCtas, 1, 1);
      cfg.blockDim = dim3(kFsThreads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kClMaxCtas;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, mixed_solve_cluster_kernel<R>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        clusters = 0;
      }
      checked = clusters >= 1 ? 1 : -1;
    }
  }
  if (checked < 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cs, 1, 1);
  cfg.blockDim = dim3(kFsThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, mixed_solve_cluster_kernel<R>, a);
  note_launch();
  return e;
}

// One cluster of ceil(n / 32) CTAs (n <= 512), or cudaErrorNotSupported (nothing enqueued).
cudaError_t launch_cluster_solve(const FusedArgs& a, cudaStream_t s) {
  const int cs = (int)((a.n + kClRows - 1) / kClRows);
  if (a.n <= 128) return launch_cluster_solve_r<4>(a, cs, s);
  if (a.n <= 256) return launch_cluster_solve_r<8>(a, cs, s);
  return launch_cluster_solve_r<16>(a, cs, s);
}

}  // namespace

cudaError_t mixed_solve_fused(const SpIterArgs& sa, const MixedArgs& ma, int precision, uint32_t* sync,
                              cudaStream_t s, int phase, BReady b_ready) {
  auto wait_b = [&]() -> cudaError_t {
    if (!b_ready.fn) return cudaSuccess;
    cudaEvent_t ev = nullptr;
    cudaError_t e = b_ready.fn(b_ready.ctx, &ev);
    if (e == cudaSuccess && ev) e = cudaStreamWaitEvent(s, ev, 0);
    return e;
  };
  // the phase input vector is staged in shared memory: n doubles, at most 32 KB
  if (sa.k != 1 || ma.k != 1 || ma.sweeps < 1 || sa.n > 4096) return cudaErrorNotSupported;
  static int max_grid = 0;  // at most one CTA per SM: every CTA is resident with room to spare
  if (max_grid == 0) {
    int dev = 0, sms = 0, coop = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    for (auto k : {mixed_solve_fused_kernel<0>, mixed_solve_fused_kernel<4>, mixed_solve_fused_kernel<8>,
                   mixed_solve_fused_kernel<16>}) {
      int o = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, kFsThreads, sizeof(double) * 4096);
      occ = occ == 0 ? o : std::min(occ, o);
    }
    if (e != cudaSuccess) return e;
    if (!coop || occ < 1) return cudaErrorNotSupported;
    max_grid = sms;
  }
  // a warp per row where n allows: fewer CTAs make each grid barrier cheaper
  const int grid = (int)std::min<int64_t>(max_grid, std::max<int64_t>(1, (sa.n + kFsWarps - 1) / kFsWarps));
  // rows in registers when every warp has at most one row of at most 512 entries
  const bool one_row = (int64_t)grid * kFsWarps >= sa.n;
  const int R = !one_row ? 0 : (sa.n <= 128 ? 4 : (sa.n <= 256 ? 8 : (sa.n <= 512 ? 16 : 0)));
  FusedArgs a;
  a.n = sa.n;
  a.sweeps = ma.sweeps;
  a.bf16 = precision == ILS_BF16_REFINE ? 1 : 0;
  a.H = sa.H;
  a.bbar = sa.bbar;
  a.bnorm2 = sa.bnorm2;
  a.tol2 = sa.tol2;
  a.tol_scale = sa.tol_scale;
  a.x = sa.X0;
  a.r = sa.bhat_out;
  a.c32 = ma.c32;
  a.d32[0] = ma.d32[0];
  a.d32[1] = ma.d32[1];
  a.P32 = ma.P32;
  a.Bt32 = ma.Bt32;
  a.Bt16 = static_cast<const __nv_bfloat16*>(ma.Bt16);
  a.partials = sa.partials;
  a.col_done = sa.col_done;
  a.col_rr = sa.col_rr;
  a.col_iters = sa.col_iters;
  a.st = sa.st;
  a.sync = sync;
  a.wait_ns = sa.wait_ns > 0 ? (uint64_t)sa.wait_ns : 1000000000ull;
  a.phase = phase;
  // n <= 512 and no wait limit of the caller's (a limit asks for the bounded grid barrier):
  // the cluster-resident kernel
  a.Hh = ma.Hh;
  a.Hl = ma.Hl;
  a.He = ma.He;
  a.A2_32 = precision == ILS_FP32_REFINE ? ma.A2_32 : nullptr;
  if (sa.n <= (int64_t)kClRows * kClMaxCtas && sa.wait_ns <= 0 && ma.Hh && ma.Hl && ma.He) {
    if (!a.A2_32) {
      const cudaError_t ew = wait_b();
      if (ew != cudaSuccess) return ew;
    }
    const cudaError_t ec = launch_cluster_solve(a, s);
    if (ec != cudaErrorNotSupported) return ec;
  }
  {  // the grid kernel reads B
    const cudaError_t ew = wait_b();
    if (ew != cudaSuccess) return ew;
  }
  cudaError_t e = cudaMemsetAsync(sync, 0, 4 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kFsThreads, 1, 1);
  cfg.dynamicSmemBytes = sizeof(double) * (size_t)std::max<int64_t>(sa.n, 32 * R);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (R) {
    case 4: e = cudaLaunchKernelEx(&cfg, mixed_solve_fused_kernel<4>, a); break;
    case 8: e = cudaLaunchKernelEx(&cfg, mixed_solve_fused_kernel<8>, a); break;
    case 16: e = cudaLaunchKernelEx(&cfg, mixed_solve_fused_kernel<16>, a); break;
    default: e = cudaLaunchKernelEx(&cfg, mixed_solve_fused_kernel<0>, a); break;
  }
  note_launch();
  return e;
}

cudaError_t split_rows_df(int64_t n, const double* H, float* Hh, float* Hl, int32_t* He, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  split_rows_df_kernel<<<(unsigned)std::min<int64_t>(n, 4096), 256, 0, s>>>(n, H, Hh, Hl, He);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
