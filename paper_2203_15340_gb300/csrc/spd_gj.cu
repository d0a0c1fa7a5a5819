// Explicit inverse of symmetric positive definite matrices by block Gauss-Jordan
// elimination (the sweep operator), FP32, one cooperative launch.
//
// P = Abar1^{-1} of Alg. 1 step 2, formed without a separate triangular factor and
// inverse.  Sweeping the TS x TS pivot block k of a symmetric A (D = A_kk) replaces
//   A_kk <- -D^{-1},  A_ik <- A_ik D^{-1},  A_kj <- D^{-1} A_kj,  A_ij <- A_ij - A_ik D^{-1} A_kj
// (i, j != k); after every block has been swept, A holds -A^{-1}.  The pivot blocks D are
// the Schur complements that a Cholesky factorization meets, so the scalar sweep of D
// (which yields -D^{-1}) also tests condition (1.3): a pivot that is not positive and
// finite is reported as NOT_SPD / NONFINITE, like a failed Cholesky pivot.
//
// Work split: the lower TS x TS tiles of every matrix (TS = 32 where each tile gets a CTA
// of its own, else 64) are spread over the CTAs and stay in their shared memory for the
// whole launch.  Step k of a tile needs D_k^{-1} and the old blocks
// k of its block rows i and j (block column k before step k); their producers post them to
// global memory once and raise a flag for each, so every tile waits only for what it reads
// (data-driven, no grid barrier).  The critical path is the chain of pivot blocks: the
// owner of tile (k+1,k+1) updates it with D_k^{-1}, sweeps it and posts D_{k+1}^{-1}.  Each
// link of that chain pays a handoff (post, fence, flag, poll, staging) besides its sweep
// and products; the wider blocks halve the number of links for the same pivot order, at
// four times the products per link.  Posts are fenced before their
// flag is raised; waits read through L2.  Every wait is bounded: past about 1 s the CTA
// records TIMEOUT, raises the abort word (which releases every other waiter) and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ils_internal.h"

namespace ils {
namespace {

constexpr int kGjThreads = 256;

// Shapes of a TS x TS tile: shared-memory row stride (16-byte rows), tiles a CTA keeps,
// warps of the pivot sweep and their column share, rows per lane in the sweep, rows per
// thread in the tile products (each thread forms kMR x 4 outputs).
template <int TS>
struct GjShape {
  static_assert(TS == 32 || TS == 64, "tile sizes 32 and 64");
  static constexpr int kPad = TS + 4;
  static constexpr int kTile = TS * kPad;
  static constexpr int kElems = TS * TS;
  static constexpr int kMaxOwn = TS == 32 ? 4 : 2;
  static constexpr int kSweepWarps = TS == 32 ? 4 : 8;
  static constexpr int kCols = TS / kSweepWarps;
  static constexpr int kRows = TS / 32;
  static constexpr int kColGroups = TS / 4;
  static constexpr int kMR = TS * TS / (4 * kGjThreads);
  static constexpr int kSweepUnroll = TS == 32 ? 16 : 4;  // fully unrolled where it fits in registers
  static_assert(kSweepWarps * 32 <= kGjThreads && kCols % 4 == 0, "sweep shape");
  static_assert(kMR * (kGjThreads / kColGroups) == TS, "product shape");
  static size_t smem_bytes() { return sizeof(float) * ((size_t)(kMaxOwn + 4) * kTile + 4 * TS); }
};

struct GjArgs {
  const float* A[2];  // n x n column-major, symmetric, both triangles stored
  float* P[2];        // the inverse, full (nullptr: status only)
  float* C[2];        // nb x nb blocks of TS x TS: C(k, i) = block (i, k) before step k, row-major
  float* D[2];        // nb blocks of TS x TS: D_k^{-1}, row-major
  uint32_t* flag[2];  // [k * nb + i]: C(k, i) posted; [nb * nb + k]: D_k^{-1} posted
  int32_t* status[2];
  uint32_t* abort_word;
  int64_t n;
  int nb;     // TS-row blocks
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

// G::kSweepWarps warps: sweeps of all TS pivots of the tile T (in place), leaving -D^{-1};
// lane l holds rows l, l + 32, ... and warp w its G::kCols columns, in registers.  The
// pivots are swept two at a time (a 2 x 2 block pivot, which equals two successive scalar
// sweeps): with the block M = [a b; b d] of pivots c, c+1,
//   rows i off the pivots:  [t0 t1] = [a_ic a_i,c+1] M^{-1},  a_iq -= t0 a_cq + t1 a_c+1,q,
//   pivot rows:             a_Pq <- M^{-1} a_Pq,  the block itself <- -M^{-1}.
// A sweep keeps the matrix symmetric, so pivot rows c, c+1 are columns c, c+1: the warp
// holding them posts both to `prow` (4 x TS floats, alternating halves), a barrier of the
// sweeping warps follows, and every lane reads its rows' two entries and the pivot rows'
// entries of its warp's columns.  Every lane applies the same multiply and two
// multiply-adds per entry.  The block's scalar pivots are a and det / a; one that is not
// positive and finite is recorded (a is replaced by 1 and det by a, so that the launch
// runs to its end).
template <int TS>
__device__ void gj_sweep_pivot(float* T, float* prow, int32_t* status) {
  using G = GjShape<TS>;
  constexpr int NC = G::kCols, NR = G::kRows;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // w < G::kSweepWarps
  const int q0 = NC * w;
  float v[NR][NC];
#pragma unroll
  for (int rr = 0; rr < NR; ++rr)
#pragma unroll
    for (int q = 0; q < NC; ++q) v[rr][q] = T[(lane + 32 * rr) * G::kPad + q0 + q];
#pragma unroll(G::kSweepUnroll)
  for (int c = 0; c < TS; c += 2) {
    float* pr = prow + ((c >> 1) & 1) * (2 * TS);
    const bool owner = w == c / NC;
    const int qc = c % NC;  // even, so qc + 1 < NC
    if (owner) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) {
#pragma unroll
        for (int q = 0; q < NC; q += 2) {
          if (q == qc) {
            pr[lane + 32 * rr] = v[rr][q];
            pr[TS + lane + 32 * rr] = v[rr][q + 1];
          }
        }
      }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(32 * G::kSweepWarps) : "memory");
    float r0[NC], r1[NC];  // a_cq, a_c+1,q of this warp's columns
#pragma unroll
    for (int h = 0; h < NC / 4; ++h) {
      const float4 w0 = reinterpret_cast<const float4*>(pr + q0)[h];
      const float4 w1 = reinterpret_cast<const float4*>(pr + TS + q0)[h];
      r0[4 * h] = w0.x;
      r0[4 * h + 1] = w0.y;
      r0[4 * h + 2] = w0.z;
      r0[4 * h + 3] = w0.w;
      r1[4 * h] = w1.x;
      r1[4 * h + 1] = w1.y;
      r1[4 * h + 2] = w1.z;
      r1[4 * h + 3] = w1.w;
    }
    float a = pr[c], b = pr[c + 1], d = pr[TS + c + 1];
    const int code = gj_pivot_code(a);
    if (code != 0) a = 1.f;
    float det = fmaf(a, d, -b * b);
    const int code2 = gj_pivot_code(det);
    if (code2 != 0) det = a;
    if ((code != 0 || code2 != 0) && threadIdx.x == 0) atomicCAS(status, 0, code != 0 ? code : code2);
    const float rdet = __fdividef(1.f, det);
    const float m00 = d * rdet, m01 = -b * rdet, m11 = a * rdet;  // M^{-1}
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
      const int row = lane + 32 * rr;
      const float ai0 = pr[row], ai1 = pr[TS + row];  // a_ic, a_i,c+1
      const bool p0 = row == c, p1 = row == c + 1;
      const float t0 = fmaf(ai0, m00, ai1 * m01), t1 = fmaf(ai0, m01, ai1 * m11);
      const float alpha = (p0 || p1) ? 0.f : 1.f;
      const float beta0 = p0 ? m00 : (p1 ? m01 : -t0);
      const float beta1 = p0 ? m01 : (p1 ? m11 : -t1);
#pragma unroll
      for (int q = 0; q < NC; ++q) v[rr][q] = fmaf(beta1, r1[q], fmaf(beta0, r0[q], alpha * v[rr][q]));
      if (owner) {  // the pivot columns themselves
#pragma unroll
        for (int q = 0; q < NC; q += 2) {
          if (q == qc) {
            v[rr][q] = p0 ? -m00 : (p1 ? -m01 : t0);
            v[rr][q + 1] = p0 ? -m01 : (p1 ? -m11 : t1);
          }
        }
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < NR; ++rr)
#pragma unroll
    for (int q = 0; q < NC; ++q) T[(lane + 32 * rr) * G::kPad + q0 + q] = v[rr][q];
}

// acc[i][q] += sum_m L(r_i, m) R(m, c0 + q) for the thread's outputs: rows
// r_i = G::kMR (tid / G::kColGroups) + i, columns c0 = 4 (tid % G::kColGroups), q < 4.
// With 32-wide tiles (one output row per thread) the thread's row of L is read into
// registers, a quarter of the row at a time by 16-byte loads, so each step of the product
// reads only R's float4 from shared memory; the sums run in the same order.
template <int TS>
__device__ __forceinline__ void gj_mm(const float* L, const float* R, float (&acc)[GjShape<TS>::kMR][4]) {
  using G = GjShape<TS>;
  const int r0 = (threadIdx.x / G::kColGroups) * G::kMR, c0 = (threadIdx.x % G::kColGroups) * 4;
  if constexpr (G::kMR == 1) {
#pragma unroll
    for (int part = 0; part < 4; ++part) {  // 8 entries of the row at a time
      float lr[TS / 4];
#pragma unroll
      for (int h = 0; h < TS / 16; ++h) {
        const float4 v = reinterpret_cast<const float4*>(L + r0 * G::kPad + part * (TS / 4))[h];
        lr[4 * h] = v.x;
        lr[4 * h + 1] = v.y;
        lr[4 * h + 2] = v.z;
        lr[4 * h + 3] = v.w;
      }
#pragma unroll
      for (int mm = 0; mm < TS / 4; ++mm) {
        const int m = part * (TS / 4) + mm;
        const float4 b = *reinterpret_cast<const float4*>(R + m * G::kPad + c0);
        acc[0][0] = fmaf(lr[mm], b.x, acc[0][0]);
        acc[0][1] = fmaf(lr[mm], b.y, acc[0][1]);
        acc[0][2] = fmaf(lr[mm], b.z, acc[0][2]);
        acc[0][3] = fmaf(lr[mm], b.w, acc[0][3]);
      }
    }
  } else {
#pragma unroll 8
    for (int m = 0; m < TS; ++m) {
      const float4 b = *reinterpret_cast<const float4*>(R + m * G::kPad + c0);
#pragma unroll
      for (int i = 0; i < G::kMR; ++i) {
        const float a = L[(r0 + i) * G::kPad + m];
        acc[i][0] = fmaf(a, b.x, acc[i][0]);
        acc[i][1] = fmaf(a, b.y, acc[i][1]);
        acc[i][2] = fmaf(a, b.z, acc[i][2]);
        acc[i][3] = fmaf(a, b.w, acc[i][3]);
      }
    }
  }
}

// Stage a TS x TS row-major global block (16-byte aligned) into a padded shared tile, or
// its transpose.
template <int TS>
__device__ __forceinline__ void gj_stage(float* dst, const float* src, bool transpose = false) {
  using G = GjShape<TS>;
  for (int e = threadIdx.x; e < G::kElems / 4; e += kGjThreads) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(src) + e);
    const int r = e / G::kColGroups, c = (e % G::kColGroups) * 4;
    if (transpose) {
      dst[c * G::kPad + r] = v.x;
      dst[(c + 1) * G::kPad + r] = v.y;
      dst[(c + 2) * G::kPad + r] = v.z;
      dst[(c + 3) * G::kPad + r] = v.w;
    } else {
      *reinterpret_cast<float4*>(dst + r * G::kPad + c) = v;
    }
  }
}

// Post sign * (a padded shared tile, or its transpose) as a TS x TS row-major global block.
template <int TS>
__device__ __forceinline__ void gj_post(float* dst, const float* T, bool transpose, float sign) {
  using G = GjShape<TS>;
  for (int e = threadIdx.x; e < G::kElems; e += kGjThreads) {
    const int r = e / TS, c = e % TS;
    dst[e] = sign * (transpose ? T[c * G::kPad + r] : T[r * G::kPad + c]);
  }
}

// After tile (i, j) of matrix m is final for the steps before k1: post what step k1 needs
// from it and raise its flag.
template <int TS>
__device__ void gj_post_for(const GjArgs& a, int m, int i, int j, int k1, float* T, float* prow) {
  using G = GjShape<TS>;
  const int nb = a.nb;
  if (i == k1 && j == k1) {
    if (threadIdx.x < 32 * G::kSweepWarps) gj_sweep_pivot<TS>(T, prow, a.status[m]);  // T := -D^{-1}
    __syncthreads();
    gj_post<TS>(a.D[m] + (size_t)k1 * G::kElems, T, false, -1.f);
    gj_raise(a.flag[m] + (size_t)nb * nb + k1);
  } else if (j == k1) {
    gj_post<TS>(a.C[m] + ((size_t)k1 * nb + i) * G::kElems, T, false, 1.f);  // A(block i, block k1)
    gj_raise(a.flag[m] + (size_t)k1 * nb + i);
  } else if (i == k1) {
    gj_post<TS>(a.C[m] + ((size_t)k1 * nb + j) * G::kElems, T, true, 1.f);  // A(block j, block k1) = A(k1, j)^T
    gj_raise(a.flag[m] + (size_t)k1 * nb + j);
  }
}

template <int TS>
__global__ void __launch_bounds__(kGjThreads) spd_gj_kernel(GjArgs a) {
  using G = GjShape<TS>;
  constexpr int MR = G::kMR;
  extern __shared__ __align__(16) float gj_smem[];
  float* own = gj_smem;                  // G::kMaxOwn tiles
  float* Ci = own + G::kMaxOwn * G::kTile;  // C_k(i)
  float* Cj = Ci + G::kTile;             // C_k(j)
  float* Dm = Cj + G::kTile;             // D^{-1}
  float* X = Dm + G::kTile;              // C_k(i) D^{-1}
  float* prow = X + G::kTile;            // 4 x TS: pivot rows of the block sweeps
  const int64_t n = a.n;
  const int total = a.count * a.tiles;
  const int tid = threadIdx.x;
  const int r0 = (tid / G::kColGroups) * MR, c0 = (tid % G::kColGroups) * 4;

  int om[G::kMaxOwn], oi[G::kMaxOwn], oj[G::kMaxOwn];
#pragma unroll
  for (int s = 0; s < G::kMaxOwn; ++s) {
    const int task = blockIdx.x + s * gridDim.x;
    om[s] = task < total ? task / a.tiles : -1;
    if (task < total) gj_tile_ij(task % a.tiles, &oi[s], &oj[s]);
    else oi[s] = oj[s] = 0;
  }
  // Own tiles; indices past n act as an identity block.
#pragma unroll
  for (int s = 0; s < G::kMaxOwn; ++s) {
    if (om[s] < 0) continue;
    float* T = own + s * G::kTile;
    const float* A = a.A[om[s]];
    for (int e = tid; e < G::kElems; e += kGjThreads) {
      const int rr = e % TS, cc = e / TS;
      const int64_t gi = TS * (int64_t)oi[s] + rr, gj = TS * (int64_t)oj[s] + cc;
      T[rr * G::kPad + cc] = (gi < n && gj < n) ? A[gi + gj * n] : (gi == gj ? 1.f : 0.f);
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < G::kMaxOwn; ++s) {
    if (om[s] < 0) continue;
    gj_post_for<TS>(a, om[s], oi[s], oj[s], 0, own + s * G::kTile, prow);
    __syncthreads();
  }

  const int nb = a.nb;
  for (int k = 0; k < nb; ++k) {
#pragma unroll
    for (int s = 0; s < G::kMaxOwn; ++s) {
      if (om[s] < 0) continue;
      const int m = om[s], i = oi[s], j = oj[s];
      float* T = own + s * G::kTile;
      if (!(i == k && j == k)) {  // the pivot tile was swept when it was posted
        const uint32_t* fl = a.flag[m];
        // The blocks of column k are posted a step before D_k^{-1}: stage them first.
        if (j != k && i != k) {
          if (!gj_wait(fl + (size_t)k * nb + i, a.abort_word, a.status[m])) return;
          if (j != i && !gj_wait(fl + (size_t)k * nb + j, a.abort_word, a.status[m])) return;
          gj_stage<TS>(Ci, a.C[m] + ((size_t)k * nb + i) * G::kElems);
          gj_stage<TS>(Cj, a.C[m] + ((size_t)k * nb + j) * G::kElems, true);  // C_k(j)^T = A_kj
        }
        if (!gj_wait(fl + (size_t)nb * nb + k, a.abort_word, a.status[m])) return;
        gj_stage<TS>(Dm, a.D[m] + (size_t)k * G::kElems);
        __syncthreads();
        float acc[MR][4];
#pragma unroll
        for (int x = 0; x < MR; ++x) acc[x][0] = acc[x][1] = acc[x][2] = acc[x][3] = 0.f;
        if (j == k || i == k) {
          if (j == k) gj_mm<TS>(T, Dm, acc);  // A_ik D^{-1}
          else gj_mm<TS>(Dm, T, acc);         // D^{-1} A_kj
          __syncthreads();                    // T is an operand: all reads before the write
        } else {
          gj_mm<TS>(Ci, Dm, acc);  // X = A_ik D^{-1}
#pragma unroll
          for (int x = 0; x < MR; ++x) {
            *reinterpret_cast<float4*>(X + (r0 + x) * G::kPad + c0) = make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
            acc[x][0] = acc[x][1] = acc[x][2] = acc[x][3] = 0.f;
          }
          __syncthreads();
          gj_mm<TS>(X, Cj, acc);  // X A_kj
#pragma unroll
          for (int x = 0; x < MR; ++x)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[x][q] = T[(r0 + x) * G::kPad + c0 + q] - acc[x][q];
        }
#pragma unroll
        for (int x = 0; x < MR; ++x)
          *reinterpret_cast<float4*>(T + (r0 + x) * G::kPad + c0) = make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
        __syncthreads();
      }
      if (k + 1 < nb) {
        gj_post_for<TS>(a, m, i, j, k + 1, T, prow);
        __syncthreads();
      }
    }
  }
  // Every tile now holds -(A^{-1}); write the inverse, both triangles.
#pragma unroll
  for (int s = 0; s < G::kMaxOwn; ++s) {
    if (om[s] < 0 || !a.P[om[s]]) continue;
    float* P = a.P[om[s]];
    const float* T = own + s * G::kTile;
    for (int e = tid; e < G::kElems; e += kGjThreads) {
      const int rr = e % TS, cc = e / TS;
      const int64_t gi = TS * (int64_t)oi[s] + rr, gj = TS * (int64_t)oj[s] + cc;
      // a diagonal tile writes its lower half twice, so each element has one writer
      if (gi < n && gj < n && (oi[s] != oj[s] || rr >= cc)) {
        const float v = -T[rr * G::kPad + cc];
        P[gi + gj * n] = v;
        P[gj + gi * n] = v;
      }
    }
  }
}

// Scratch floats of one launch with TS x TS tiles: per matrix C (nb^2 blocks), D (nb
// blocks) and flags (nb^2 + nb words, padded to 16 bytes); then the abort word.
size_t gj_scratch_floats(int64_t n, int ts) {
  const size_t nb = (size_t)((n + ts - 1) / ts);
  const size_t blocks = nb * nb + nb;
  return 2 * (blocks * ts * ts + ((blocks + 3) & ~(size_t)3)) + 64;
}

// Launch with TS x TS tiles, at most max_own of them per CTA, or cudaErrorNotSupported
// (nothing enqueued) where they do not fit one cooperative wave that way.
template <int TS>
cudaError_t gj_launch(int64_t n, int count, const float* const* A, float* const* P, float* scratch,
                      int32_t* const* status, int max_own, cudaStream_t s) {
  using G = GjShape<TS>;
  const int nb = (int)((n + TS - 1) / TS);
  const int tiles = nb * (nb + 1) / 2;
  const int total = count * tiles;
  int dev = 0, sms = 0, coop = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess && G::smem_bytes() > 48 * 1024)
    e = cudaFuncSetAttribute(spd_gj_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes());
  // SMs running it keep the largest shared-memory carveout, so that the other cooperative
  // inverse (the test of H) and the setup's cluster kernels can be placed beside its CTAs
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spd_gj_kernel<TS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spd_gj_kernel<TS>, kGjThreads, G::smem_bytes());
  if (e != cudaSuccess) return e;
  const int64_t grid_max = (int64_t)occ * sms;
  const int grid = (int)std::min<int64_t>(total, grid_max);
  if (!coop || grid < 1 || (int64_t)grid * std::min(max_own, G::kMaxOwn) < total) return cudaErrorNotSupported;
  GjArgs a;
  const size_t blocks = (size_t)nb * nb + nb;
  const size_t per = blocks * G::kElems + ((blocks + 3) & ~(size_t)3);  // floats, then flag words (16-byte steps)
  for (int i = 0; i < 2; ++i) {
    const int src = i < count ? i : 0;
    float* base = scratch + (size_t)src * per;
    a.A[i] = A[src];
    a.P[i] = P[src];
    a.C[i] = base;
    a.D[i] = base + (size_t)nb * nb * G::kElems;
    a.flag[i] = reinterpret_cast<uint32_t*>(base + blocks * G::kElems);
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
  cfg.dynamicSmemBytes = G::smem_bytes();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, spd_gj_kernel<TS>, a);
  note_launch();
  return e;
}

}  // namespace

size_t spd_inverse_scratch_floats(int64_t n) { return std::max(gj_scratch_floats(n, 32), gj_scratch_floats(n, 64)); }

cudaError_t spd_inverse_f32(int64_t n, int count, const float* const* A, float* const* P, float* scratch,
                            int32_t* const* status, cudaStream_t s, bool wide_first) {
  if (n <= 0 || count < 1 || count > 2) return cudaErrorInvalidValue;
  // The chain's links are shortest with 32-wide blocks and one tile per CTA; where 32-wide
  // tiles would have to share CTAs, 64-wide blocks (half the links, each longer) are faster
  // (measured: n = 1024, 265 us against 344 us).  wide_first takes the 64-wide blocks
  // wherever they fit: a quarter of the CTAs, for a launch that runs beside other work.
  cudaError_t e = wide_first ? cudaErrorNotSupported : gj_launch<32>(n, count, A, P, scratch, status, 1, s);
  if (e != cudaErrorNotSupported) return e;
  e = gj_launch<64>(n, count, A, P, scratch, status, GjShape<64>::kMaxOwn, s);
  if (e != cudaErrorNotSupported) return e;
  return gj_launch<32>(n, count, A, P, scratch, status, GjShape<32>::kMaxOwn, s);
}

}  // namespace ils
