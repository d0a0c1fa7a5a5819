// Explicit inverse of symmetric positive definite matrices by block Gauss-Jordan
// elimination (the sweep operator), FP32, one cooperative launch.
//
// P = Abar1^{-1} of Alg. 1 step 2, formed without a separate triangular factor and
// inverse.  Sweeping the 32 x 32 pivot block k of a symmetric A (D = A_kk) replaces
//   A_kk <- -D^{-1},  A_ik <- A_ik D^{-1},  A_kj <- D^{-1} A_kj,  A_ij <- A_ij - A_ik D^{-1} A_kj
// (i, j != k); after every block has been swept, A holds -A^{-1}.  The pivot blocks D are
// the Schur complements that a Cholesky factorization meets, so the scalar sweep of D
// (which yields -D^{-1}) also tests condition (1.3): a pivot that is not positive and
// finite is reported as NOT_SPD / NONFINITE, like a failed Cholesky pivot.
//
// Work split: the lower 32 x 32 tiles of every matrix are spread over the CTAs and stay in
// their shared memory for the whole launch.  Step k of a tile needs D_k^{-1} and the old
// blocks k of its block rows i and j (block column k before step k); their producers
// post them to global memory once and raise a flag for each, so every tile waits only
// for what it reads (data-driven, no grid barrier).  The critical path is the chain of
// pivot blocks: the owner of tile (k+1,k+1) updates it with D_k^{-1}, sweeps it and posts
// D_{k+1}^{-1}.  Posts are fenced before their flag is raised; waits read through L2.
// Every wait is bounded: past about 1 s the CTA records TIMEOUT, raises the abort word
// (which releases every other waiter) and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ils_internal.h"

namespace ils {
namespace {

constexpr int kGjThreads = 256;
constexpr int kGjMaxOwn = 4;  // tiles a CTA keeps in shared memory
constexpr int kGjPad = 36;    // row stride of a tile in shared memory (16-byte rows)
constexpr int kGjTile = 32 * kGjPad;

struct GjArgs {
  const float* A[2];  // n x n column-major, symmetric, both triangles stored
  float* P[2];        // the inverse, full (nullptr: status only)
  float* C[2];        // nb x nb blocks of 32 x 32: C(k, i) = block (i, k) before step k, row-major
  float* D[2];        // nb blocks of 32 x 32: D_k^{-1}, row-major
  uint32_t* flag[2];  // [k * nb + i]: C(k, i) posted; [nb * nb + k]: D_k^{-1} posted
  int32_t* status[2];
  uint32_t* abort_word;
  int64_t n;
  int nb;     // 32-row blocks
  int count;  // matrices (1 or 2)
  int tiles;  // lower tiles per matrix
};

__device__ __forceinline__ uint32_t gj_ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t gj_ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *flag != 0 (relaxed polls; an acquire fence once it is seen), then
// the CTA goes on.  False on abort or after about 1 s, recorded as TIMEOUT.
__device__ bool gj_wait(const uint32_t* flag, uint32_t* abort_word, int32_t* status) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int res = 1;
    uint64_t t0 = 0;
    for (uint32_t spin = 0;; ++spin) {
      if (gj_ld_relaxed(flag) != 0u) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        break;
      }
      if ((spin & 15u) == 15u) {
        if (gj_ld_acquire(abort_word) != 0u) {
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
    ok = res;
  }
  __syncthreads();
  return ok != 0;
}

// After the CTA's stores of a post: order them before the flag (CTA barrier, then a
// release store by thread 0).
__device__ __forceinline__ void gj_raise(uint32_t* flag) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(1u) : "memory");
}

// Lower tile t of an nb-block matrix, row-major over the lower triangle: (i, j), i >= j.
__device__ __forceinline__ void gj_tile_ij(int t, int* i, int* j) {
  int r = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  *i = r;
  *j = t - r * (r + 1) / 2;
}

__device__ __forceinline__ int gj_pivot_code(float d) {
  if (!isfinite(d)) return ILS_ERR_NONFINITE;
  if (!(d > 0.f)) return ILS_ERR_NOT_SPD;
  return 0;
}

// kSweepWarps warps: sweeps of all 32 pivots of the tile T (in place), leaving -D^{-1};
// lane = row, warp w holding its kSweepCols columns of it in registers.  The pivots are swept two at
// a time (a 2 x 2 block pivot, which equals two successive scalar sweeps): with the block
// M = [a b; b d] of pivots c, c+1,
//   rows i off the pivots:  [t0 t1] = [a_ic a_i,c+1] M^{-1},  a_iq -= t0 a_cq + t1 a_c+1,q,
//   pivot rows:             a_Pq <- M^{-1} a_Pq,  the block itself <- -M^{-1}.
// A sweep keeps the matrix symmetric, so pivot rows c, c+1 are columns c, c+1: the warp
// holding them posts both to `prow` (4 x 32 floats, alternating halves), a barrier of the
// sweeping warps follows, and every lane reads its two entries and the rows' entries of its
// warp's columns.  Every lane applies the same multiply and two multiply-adds per entry.
// The block's scalar pivots are a and det / a; one that is not positive and finite is
// recorded (a is replaced by 1 and det by a, so that the launch runs to its end).
constexpr int kSweepWarps = 4;
constexpr int kSweepCols = 32 / kSweepWarps;

__device__ void gj_sweep_pivot(float* T, float* prow, int32_t* status) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // w < kSweepWarps
  const int q0 = kSweepCols * w;
  float v[kSweepCols];
#pragma unroll
  for (int q = 0; q < kSweepCols; ++q) v[q] = T[lane * kGjPad + q0 + q];
#pragma unroll
  for (int c = 0; c < 32; c += 2) {
    float* pr = prow + ((c >> 1) & 1) * 64;
    const bool owner = w == c / kSweepCols;
    if (owner) {
      pr[lane] = v[c % kSweepCols];
      pr[32 + lane] = v[(c + 1) % kSweepCols];
    }
    asm volatile("bar.sync 1, %0;" ::"r"(32 * kSweepWarps) : "memory");
    const float ai0 = pr[lane], ai1 = pr[32 + lane];  // a_ic, a_i,c+1
    float r0[kSweepCols], r1[kSweepCols];            // a_cq, a_c+1,q of this warp's columns
#pragma unroll
    for (int h = 0; h < kSweepCols / 4; ++h) {
      const float4 w0 = reinterpret_cast<const float4*>(pr + q0)[h];
      const float4 w1 = reinterpret_cast<const float4*>(pr + 32 + q0)[h];
      r0[4 * h] = w0.x;
      r0[4 * h + 1] = w0.y;
      r0[4 * h + 2] = w0.z;
      r0[4 * h + 3] = w0.w;
      r1[4 * h] = w1.x;
      r1[4 * h + 1] = w1.y;
      r1[4 * h + 2] = w1.z;
      r1[4 * h + 3] = w1.w;
    }
    float a = pr[c], b = pr[c + 1], d = pr[32 + c + 1];
    const int code = gj_pivot_code(a);
    if (code != 0) a = 1.f;
    float det = fmaf(a, d, -b * b);
    const int code2 = gj_pivot_code(det);
    if (code2 != 0) det = a;
    if ((code != 0 || code2 != 0) && threadIdx.x == 0) atomicCAS(status, 0, code != 0 ? code : code2);
    const float rdet = __fdividef(1.f, det);
    const float m00 = d * rdet, m01 = -b * rdet, m11 = a * rdet;  // M^{-1}
    const bool p0 = lane == c, p1 = lane == c + 1;
    const float t0 = fmaf(ai0, m00, ai1 * m01), t1 = fmaf(ai0, m01, ai1 * m11);
    const float alpha = (p0 || p1) ? 0.f : 1.f;
    const float beta0 = p0 ? m00 : (p1 ? m01 : -t0);
    const float beta1 = p0 ? m01 : (p1 ? m11 : -t1);
#pragma unroll
    for (int q = 0; q < kSweepCols; ++q) v[q] = fmaf(beta1, r1[q], fmaf(beta0, r0[q], alpha * v[q]));
    if (owner) {  // the pivot columns themselves
      v[c % kSweepCols] = p0 ? -m00 : (p1 ? -m01 : t0);
      v[(c + 1) % kSweepCols] = p0 ? -m01 : (p1 ? -m11 : t1);
    }
  }
#pragma unroll
  for (int q = 0; q < kSweepCols; ++q) T[lane * kGjPad + q0 + q] = v[q];
}

// acc[q] += sum_m L(r, m) R(m, c0 + q) for the thread's outputs r = tid / 8,
// c0 = 4 (tid % 8), q < 4 (R read four columns at a time).
__device__ __forceinline__ void gj_mm4(const float* L, const float* R, float acc[4]) {
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
#pragma unroll 8
  for (int m = 0; m < 32; ++m) {
    const float a = L[r * kGjPad + m];
    const float4 b = *reinterpret_cast<const float4*>(R + m * kGjPad + c0);
    acc[0] = fmaf(a, b.x, acc[0]);
    acc[1] = fmaf(a, b.y, acc[1]);
    acc[2] = fmaf(a, b.z, acc[2]);
    acc[3] = fmaf(a, b.w, acc[3]);
  }
}

// Stage a 32 x 32 row-major global block (16-byte aligned) into a padded shared tile, or
// its transpose.
__device__ __forceinline__ void gj_stage(float* dst, const float* src, bool transpose = false) {
  for (int e = threadIdx.x; e < 256; e += kGjThreads) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(src) + e);
    const int r = e >> 3, c = (e & 7) * 4;
    if (transpose) {
      dst[c * kGjPad + r] = v.x;
      dst[(c + 1) * kGjPad + r] = v.y;
      dst[(c + 2) * kGjPad + r] = v.z;
      dst[(c + 3) * kGjPad + r] = v.w;
    } else {
      *reinterpret_cast<float4*>(dst + r * kGjPad + c) = v;
    }
  }
}

// Post sign * (a padded shared tile, or its transpose) as a 32 x 32 row-major global block.
__device__ __forceinline__ void gj_post(float* dst, const float* T, bool transpose, float sign) {
  for (int e = threadIdx.x; e < 1024; e += kGjThreads) {
    const int r = e >> 5, c = e & 31;
    dst[e] = sign * (transpose ? T[c * kGjPad + r] : T[r * kGjPad + c]);
  }
}

// After tile (i, j) of matrix m is final for the steps before k1: post what step k1 needs
// from it and raise its flag.
__device__ void gj_post_for(const GjArgs& a, int m, int i, int j, int k1, float* T, float* prow) {
  const int nb = a.nb;
  if (i == k1 && j == k1) {
    if (threadIdx.x < 32 * kSweepWarps) gj_sweep_pivot(T, prow, a.status[m]);  // T := -D^{-1}
    __syncthreads();
    gj_post(a.D[m] + (size_t)k1 * 1024, T, false, -1.f);
    gj_raise(a.flag[m] + (size_t)nb * nb + k1);
  } else if (j == k1) {
    gj_post(a.C[m] + ((size_t)k1 * nb + i) * 1024, T, false, 1.f);  // A(block i, block k1)
    gj_raise(a.flag[m] + (size_t)k1 * nb + i);
  } else if (i == k1) {
    gj_post(a.C[m] + ((size_t)k1 * nb + j) * 1024, T, true, 1.f);   // A(block j, block k1) = A(k1, j)^T
    gj_raise(a.flag[m] + (size_t)k1 * nb + j);
  }
}

__global__ void __launch_bounds__(kGjThreads) spd_gj_kernel(GjArgs a) {
  extern __shared__ __align__(16) float gj_smem[];
  float* own = gj_smem;                 // kGjMaxOwn tiles
  float* Ci = own + kGjMaxOwn * kGjTile;  // C_k(i)
  float* Cj = Ci + kGjTile;             // C_k(j)
  float* Dm = Cj + kGjTile;             // D^{-1}
  float* X = Dm + kGjTile;              // C_k(i) D^{-1}
  float* prow = X + kGjTile;            // 4 x 32: pivot rows of the block sweeps
  const int64_t n = a.n;
  const int total = a.count * a.tiles;
  const int tid = threadIdx.x;
  const int r = tid >> 3, c0 = (tid & 7) * 4;

  int om[kGjMaxOwn], oi[kGjMaxOwn], oj[kGjMaxOwn];
#pragma unroll
  for (int s = 0; s < kGjMaxOwn; ++s) {
    const int task = blockIdx.x + s * gridDim.x;
    om[s] = task < total ? task / a.tiles : -1;
    if (task < total) gj_tile_ij(task % a.tiles, &oi[s], &oj[s]);
    else oi[s] = oj[s] = 0;
  }
  // Own tiles; indices past n act as an identity block.
#pragma unroll
  for (int s = 0; s < kGjMaxOwn; ++s) {
    if (om[s] < 0) continue;
    float* T = own + s * kGjTile;
    const float* A = a.A[om[s]];
    for (int e = tid; e < 1024; e += kGjThreads) {
      const int rr = e & 31, cc = e >> 5;
      const int64_t gi = 32 * (int64_t)oi[s] + rr, gj = 32 * (int64_t)oj[s] + cc;
      T[rr * kGjPad + cc] = (gi < n && gj < n) ? A[gi + gj * n] : (gi == gj ? 1.f : 0.f);
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < kGjMaxOwn; ++s) {
    if (om[s] < 0) continue;
    gj_post_for(a, om[s], oi[s], oj[s], 0, own + s * kGjTile, prow);
    __syncthreads();
  }

  const int nb = a.nb;
  for (int k = 0; k < nb; ++k) {
#pragma unroll
    for (int s = 0; s < kGjMaxOwn; ++s) {
      if (om[s] < 0) continue;
      const int m = om[s], i = oi[s], j = oj[s];
      float* T = own + s * kGjTile;
      if (!(i == k && j == k)) {  // the pivot tile was swept when it was posted
        const uint32_t* fl = a.flag[m];
        // The blocks of column k are posted a step before D_k^{-1}: stage them first.
        if (j != k && i != k) {
          if (!gj_wait(fl + (size_t)k * nb + i, a.abort_word, a.status[m])) return;
          if (j != i && !gj_wait(fl + (size_t)k * nb + j, a.abort_word, a.status[m])) return;
          gj_stage(Ci, a.C[m] + ((size_t)k * nb + i) * 1024);
          gj_stage(Cj, a.C[m] + ((size_t)k * nb + j) * 1024, true);  // C_k(j)^T = A_kj
        }
        if (!gj_wait(fl + (size_t)nb * nb + k, a.abort_word, a.status[m])) return;
        gj_stage(Dm, a.D[m] + (size_t)k * 1024);
        __syncthreads();
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (j == k || i == k) {
          if (j == k) gj_mm4(T, Dm, acc);  // A_ik D^{-1}
          else gj_mm4(Dm, T, acc);         // D^{-1} A_kj
          __syncthreads();                 // T is an operand: all reads before the write
        } else {
          gj_mm4(Ci, Dm, acc);  // X = A_ik D^{-1}
          *reinterpret_cast<float4*>(X + r * kGjPad + c0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = 0.f;
          gj_mm4(X, Cj, acc);  // X A_kj
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = T[r * kGjPad + c0 + q] - acc[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) T[r * kGjPad + c0 + q] = acc[q];
        __syncthreads();
      }
      if (k + 1 < nb) {
        gj_post_for(a, m, i, j, k + 1, T, prow);
        __syncthreads();
      }
    }
  }
  // Every tile now holds -(A^{-1}); write the inverse, both triangles.
#pragma unroll
  for (int s = 0; s < kGjMaxOwn; ++s) {
    if (om[s] < 0 || !a.P[om[s]]) continue;
    float* P = a.P[om[s]];
    const float* T = own + s * kGjTile;
    for (int e = tid; e < 1024; e += kGjThreads) {
      const int rr = e & 31, cc = e >> 5;
      const int64_t gi = 32 * (int64_t)oi[s] + rr, gj = 32 * (int64_t)oj[s] + cc;
      // a diagonal tile writes its lower half twice, so each element has one writer
      if (gi < n && gj < n && (oi[s] != oj[s] || rr >= cc)) {
        const float v = -T[rr * kGjPad + cc];
        P[gi + gj * n] = v;
        P[gj + gi * n] = v;
      }
    }
  }
}

size_t gj_smem_bytes() { return sizeof(float) * ((size_t)(kGjMaxOwn + 4) * kGjTile + 128); }

}  // namespace

size_t spd_inverse_scratch_floats(int64_t n) {
  const size_t nb = (size_t)((n + 31) / 32);
  // per matrix: C (nb^2 blocks), D (nb blocks), flags (nb^2 + nb words, padded to 16 bytes);
  // then the abort word
  const size_t blocks = nb * nb + nb;
  return 2 * (blocks * 1024 + ((blocks + 3) & ~(size_t)3)) + 64;
}

cudaError_t spd_inverse_f32(int64_t n, int count, const float* const* A, float* const* P, float* scratch,
                            int32_t* const* status, cudaStream_t s) {
  if (n <= 0 || count < 1 || count > 2) return cudaErrorInvalidValue;
  const int nb = (int)((n + 31) / 32);
  const int tiles = nb * (nb + 1) / 2;
  const int total = count * tiles;
  int dev = 0, sms = 0, coop = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spd_gj_kernel, kGjThreads, gj_smem_bytes());
  if (e != cudaSuccess) return e;
  const int64_t grid_max = (int64_t)occ * sms;
  const int grid = (int)std::min<int64_t>(total, grid_max);
  if (!coop || grid < 1 || (int64_t)grid * kGjMaxOwn < total) return cudaErrorNotSupported;
  GjArgs a;
  const size_t blocks = (size_t)nb * nb + nb;
  const size_t per = blocks * 1024 + ((blocks + 3) & ~(size_t)3);  // floats, then flag words (16-byte steps)
  for (int i = 0; i < 2; ++i) {
    const int src = i < count ? i : 0;
    float* base = scratch + (size_t)src * per;
    a.A[i] = A[src];
    a.P[i] = P[src];
    a.C[i] = base;
    a.D[i] = base + (size_t)nb * nb * 1024;
    a.flag[i] = reinterpret_cast<uint32_t*>(base + blocks * 1024);
    a.status[i] = status[src];
  }
  a.abort_word = reinterpret_cast<uint32_t*>(scratch + 2 * per);
  a.n = n;
  a.nb = nb;
  a.count = count;
  a.tiles = tiles;
  for (int i = 0; i < count; ++i)
    if ((e = cudaMemsetAsync(a.flag[i], 0, sizeof(uint32_t) * blocks, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.abort_word, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
  // Cooperative launch: every CTA is resident, so a CTA waiting on a flag never holds the
  // SM its producer needs.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kGjThreads, 1, 1);
  cfg.dynamicSmemBytes = gj_smem_bytes();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, spd_gj_kernel, a);
  note_launch();
  return e;
}

}  // namespace ils
