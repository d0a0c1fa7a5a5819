// Mixed-precision SP with FP64 refinement for many right-hand sides at once (k >= 32).
//
// With a block of right-hand sides every product of the refinement is a dense GEMM:
//   bbar = A^T J B             (m x n x k, once)          FP64-accurate split digit products
//   R    = bbar - H X          (n x n x k, each step)     on the tcgen05 tensor cores
//   C    = P R,  D <- B D + C  (n x n x k, s sweeps)      FP32 (Alg. 1 step 6 on the correction)
//   X   += D                                               FP64
// so the FP64-accurate parts (the right-hand side and the residual, which decide the
// accuracy) run as exact BF16 digit products on the tensor cores instead of on the narrow
// FP64 pipe, and the sweeps need only FP32 accuracy.  Each column stops on its own test
// (before each correction, as in Sec. 5); a finished column's residual is replaced by zero
// so its correction is exactly zero and its iterate stays.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ils_internal.h"

namespace ils {
namespace {

constexpr int kWmThreads = 256;

__device__ __forceinline__ double wm_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ||bbar(:, c)||^2 for each column (one CTA per column).
__global__ void __launch_bounds__(kWmThreads) wm_norms_kernel(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                              double* __restrict__ out) {
  const int64_t c = blockIdx.x;
  double part = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = V[i + c * ldv];
    part = fma(v, v, part);
  }
  __shared__ double red[kWmThreads / 32];
  part = wm_warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWmThreads / 32; ++w) t += red[w];
    out[c] = t;
  }
}

// Column c of the residual R = bbar - H X_k: its norm decides whether the column is done
// (relres^2 <= tol2 * scale, scale = 1 / kappa_est^2 for the error-bound rule); an active
// column's residual goes to FP32 for the sweeps, a finished one's is zeroed.  state:
// [0] active columns left (counted down), [1] status.
__global__ void __launch_bounds__(kWmThreads)
wm_check_kernel(int64_t n, const double* __restrict__ R, int64_t ldr, float* __restrict__ R32, const double* __restrict__ bn,
                int32_t* __restrict__ done, double* __restrict__ rr_out, int64_t* __restrict__ iters, int64_t it,
                int64_t max_outer, double tol2, const double* __restrict__ tol_scale, int32_t* __restrict__ state) {
  const int64_t c = blockIdx.x;
  __shared__ double red[kWmThreads / 32];
  __shared__ int finish;
  const bool was_done = done[c] != 0;
  double part = 0.0;
  if (!was_done)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = R[i + c * ldr];
      part = fma(v, v, part);
    }
  part = wm_warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    finish = 1;
    if (!was_done) {
      double rr = 0.0;
      for (int w = 0; w < kWmThreads / 32; ++w) rr += red[w];
      const bool finite = isfinite(rr);
      const bool conv = finite && rr <= tol2 * (tol_scale ? *tol_scale : 1.0) * bn[c];
      finish = (!finite || conv || it >= max_outer) ? 1 : 0;
      rr_out[c] = rr;
      iters[c] = it;
      if (finish) {
        done[c] = 1;
        atomicSub(state, 1);
        if (!finite) atomicCAS(state + 1, 0, ILS_ERR_NONFINITE);
        else if (!conv) atomicCAS(state + 1, 0, ILS_ERR_NO_CONVERGENCE);
      }
    }
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) R32[i + c * n] = finish ? 0.f : (float)R[i + c * ldr];
}

// X(:, c) += D(:, c) in FP64 (D is zero for finished columns).
__global__ void wm_update_kernel(int64_t n, int64_t k, const float* __restrict__ D, double* __restrict__ X, int64_t ldx) {
  const int64_t total = n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, c = e / n;
    X[i + c * ldx] += (double)D[e];
  }
}

__global__ void wm_init_kernel(int64_t k, int32_t* done, int32_t* state) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x)
    done[c] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    state[0] = (int32_t)k;
    state[1] = 0;
  }
}

}  // namespace

cudaError_t wide_mixed_solve(const WideMixedArgs& a, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                             int x0_zero, WideMixedResult* res, int32_t* h_state, cudaStream_t s) {
  const int64_t m = a.m, n = a.n, p = a.p;
  const int64_t kb_max = std::min<int64_t>(k, kWideMixedBlock);
  res->relres = 0.0;
  res->refinements = 0;
  res->status = 0;
  if (k <= 0) return cudaSuccess;
  // one device allocation, carved into aligned pieces
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t o_slA = take(2 * digit_slice_elems(m, n)), o_exA = take(4 * n);
  const size_t o_slB = take(2 * digit_slice_elems(m, kb_max)), o_exB = take(4 * kb_max);
  const size_t o_slH = take(2 * digit_slice_elems(n, n)), o_exH = take(4 * n);
  const size_t o_slX = take(2 * digit_slice_elems(n, kb_max)), o_exX = take(4 * kb_max);
  const size_t o_part = take(8 * std::max(gemm_partial_elems(m, n, kb_max), gemm_partial_elems(n, n, kb_max)));
  const size_t o_bbar = take(8 * n * kb_max), o_R = take(8 * n * kb_max);
  const size_t o_bn = take(8 * kb_max), o_rr = take(8 * kb_max), o_it = take(8 * kb_max);
  const size_t o_done = take(4 * kb_max), o_state = take(8), o_err = take(4);
  const size_t o_R32 = take(4 * n * kb_max), o_C32 = take(4 * n * kb_max), o_Da = take(4 * n * kb_max),
               o_Db = take(4 * n * kb_max);
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, off, s);
  if (e != cudaSuccess) return e;
  void* slA = base + o_slA;
  int* exA = (int*)(base + o_exA);
  void* slB = base + o_slB;
  int* exB = (int*)(base + o_exB);
  void* slH = base + o_slH;
  int* exH = (int*)(base + o_exH);
  void* slX = base + o_slX;
  int* exX = (int*)(base + o_exX);
  double* part = (double*)(base + o_part);
  double* bbar = (double*)(base + o_bbar);
  double* R = (double*)(base + o_R);
  double* bn = (double*)(base + o_bn);
  double* rr = (double*)(base + o_rr);
  int64_t* its = (int64_t*)(base + o_it);
  int32_t* done = (int32_t*)(base + o_done);
  int32_t* state = (int32_t*)(base + o_state);
  int32_t* err = (int32_t*)(base + o_err);
  float* R32 = (float*)(base + o_R32);
  float* C32 = (float*)(base + o_C32);
  float* Da = (float*)(base + o_Da);
  float* Db = (float*)(base + o_Db);
  std::vector<double> hrr(kb_max), hbn(kb_max);
  std::vector<int64_t> hit(kb_max);
  auto run = [&]() -> cudaError_t {
    cudaError_t e2;
    if ((e2 = cudaMemsetAsync(err, 0, 4, s)) != cudaSuccess) return e2;
    // digits of A (no sign: J goes with B) and of H, once per call
    if ((e2 = split_digits(m, n, a.A, m, m, slA, exA, err, s)) != cudaSuccess) return e2;
    if ((e2 = split_digits(n, n, a.H, n, n, slH, exH, err, s)) != cudaSuccess) return e2;
    for (int64_t c0 = 0; c0 < k; c0 += kb_max) {
      const int64_t kb = std::min<int64_t>(kb_max, k - c0);
      const double* Bc = B + c0 * ldb;
      double* Xc = X + c0 * ldx;
      // bbar = A^T J B (Alg. 1 step 4): rows >= p of B split negated
      if ((e2 = split_digits(m, kb, Bc, ldb, p, slB, exB, err, s)) != cudaSuccess) return e2;
      if ((e2 = gemm_split_tc(m, n, kb, slA, exA, slB, exB, bbar, n, nullptr, 0, part, err, s)) != cudaSuccess)
        return e2;
      wm_norms_kernel<<<(unsigned)kb, kWmThreads, 0, s>>>(n, bbar, n, bn);
      note_launch();
      if (x0_zero && (e2 = cudaMemset2DAsync(Xc, sizeof(double) * ldx, 0, sizeof(double) * n, kb, s)) != cudaSuccess)
        return e2;
      wm_init_kernel<<<(unsigned)std::min<int64_t>((kb + 255) / 256, 64), 256, 0, s>>>(kb, done, state);
      note_launch();
      if ((e2 = cudaGetLastError()) != cudaSuccess) return e2;
      for (int64_t it = 0;; ++it) {
        // R = bbar - H X_k in FP64 accuracy; the test of Sec. 5 before the update
        if ((e2 = split_digits(n, kb, Xc, ldx, n, slX, exX, err, s)) != cudaSuccess) return e2;
        if ((e2 = gemm_split_tc(n, n, kb, slH, exH, slX, exX, R, n, bbar, n, part, err, s)) != cudaSuccess) return e2;
        wm_check_kernel<<<(unsigned)kb, kWmThreads, 0, s>>>(n, R, n, R32, bn, done, rr, its, it, a.max_outer, a.tol2,
                                                            a.tol_scale, state);
        note_launch();
        if ((e2 = cudaGetLastError()) != cudaSuccess) return e2;
        if ((e2 = cudaMemcpyAsync(h_state, state, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e2;
        if ((e2 = cudaStreamSynchronize(s)) != cudaSuccess) return e2;
        if (h_state[0] <= 0) break;
        // correction: s SP sweeps on H d = r from d = 0 (d_1 = P r, d_{j+1} = B d_j + P r), FP32
        GemmF32 g{};
        g.M = n; g.N = kb; g.K = n; g.lda = n; g.ldb = n; g.ldc = n;
        g.A = a.P32; g.B = R32; g.C = C32; g.alpha = 1.f; g.beta = 0.f;
        if ((e2 = gemm_f32(false, false, g, 1, s)) != cudaSuccess) return e2;  // C = P r (P symmetric)
        float* d = C32;
        for (int sw = 1; sw < a.sweeps; ++sw) {
          float* nd = (d == Da) ? Db : Da;
          if ((e2 = cudaMemcpyAsync(nd, C32, sizeof(float) * n * kb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e2;
          GemmF32 gs{};
          gs.M = n; gs.N = kb; gs.K = n; gs.lda = n; gs.ldb = n; gs.ldc = n;
          gs.A = a.Bt32; gs.B = d; gs.C = nd; gs.alpha = 1.f; gs.beta = 1.f;
          if ((e2 = gemm_f32(true, false, gs, 1, s)) != cudaSuccess) return e2;  // nd = B d + c (B = Bt32^T)
          d = nd;
        }
        wm_update_kernel<<<(unsigned)std::min<int64_t>((n * kb + 255) / 256, 4096), 256, 0, s>>>(n, kb, d, Xc, ldx);
        note_launch();
        if ((e2 = cudaGetLastError()) != cudaSuccess) return e2;
      }
      if ((e2 = cudaMemcpyAsync(hrr.data(), rr, 8 * kb, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e2;
      if ((e2 = cudaMemcpyAsync(hbn.data(), bn, 8 * kb, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e2;
      if ((e2 = cudaMemcpyAsync(hit.data(), its, 8 * kb, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e2;
      if ((e2 = cudaMemcpyAsync(h_state + 2, err, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e2;
      if ((e2 = cudaStreamSynchronize(s)) != cudaSuccess) return e2;
      for (int64_t c = 0; c < kb; ++c) {
        const double rel = hbn[c] > 0.0 ? std::sqrt(hrr[c] / hbn[c]) : std::sqrt(hrr[c]);
        res->relres = (rel != rel) ? rel : std::max(res->relres, rel);
        res->refinements = std::max<int64_t>(res->refinements, hit[c]);
      }
      if (h_state[1] != 0 && res->status == 0) res->status = h_state[1];
      if (h_state[2] != 0 && res->status == 0) res->status = h_state[2] == 2 ? ILS_ERR_NONFINITE : ILS_ERR_TIMEOUT;
    }
    return cudaSuccess;
  };
  e = run();
  cudaFreeAsync(base, s);
  return e;
}

}  // namespace ils
