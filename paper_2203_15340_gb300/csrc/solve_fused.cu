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

}  // namespace

cudaError_t mixed_solve_fused(const SpIterArgs& sa, const MixedArgs& ma, int precision, uint32_t* sync,
                              cudaStream_t s, int phase) {
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

}  // namespace ils
