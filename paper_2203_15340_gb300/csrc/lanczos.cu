// Lanczos estimates of the quantities that certify a solve (Theorem 2.1's setting):
//   kappa_2(H), H = A^T J A:  x - x* = -H^{-1} r gives ||x - x*|| / ||x*|| <= kappa_2(H) relres;
//   rho(Abar1^{-1} Abar2):    the SP contraction factor of Theorem 2.1 (rho < 1 iff (1.3)).
//
// Standard Lanczos on H gives its extreme eigenvalues.  For rho, C = Abar2 P (P = Abar1^{-1})
// is self-adjoint in the inner product <x, y>_P = x^T P y and has the eigenvalues of
// B = P Abar2, so Lanczos on C in that inner product needs one product with Abar2 and one
// with P per step.  In general: operator C = M2 M1, inner product M1 (M1 = I: standard).
//
// GB300 design: one thread-block cluster per operator.  Each CTA keeps its slice of rows
// of M2 (and M1) in shared memory as FP32 for all steps, so a step reads no global memory;
// vectors are exchanged through distributed shared memory and every reduction adds the
// CTAs' partials in rank order (all CTAs hold identical scalars).  The extreme eigenvalues
// of the k x k tridiagonal matrix come from Sturm-sequence bisection in FP64.  Ritz values
// lie inside the spectrum, so the estimates approach the extremes from inside.
#include <cmath>
#include <utility>

#include "ils_internal.h"

namespace ils {
namespace {

constexpr int kLzThreads = 256;
constexpr int kLzWarps = kLzThreads / 32;
constexpr int kLzMaxCs = 16;
constexpr int kLzMaxSteps = 256;

__device__ __forceinline__ uint32_t lz_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Store v into the same shared-memory location of cluster CTA `rank`.
__device__ __forceinline__ void st_remote(const float* local, uint32_t rank, float v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(lz_smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(remote), "f"(v) : "memory");
}

// Store four consecutive floats (16-byte aligned) into the same location of CTA `rank`.
__device__ __forceinline__ void st_remote4(const float* local, uint32_t rank, const float (&v)[4]) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(lz_smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(remote), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3])
               : "memory");
}

// All threads of all CTAs of the cluster; release/acquire orders the DSMEM stores.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ float lz_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Number of eigenvalues below x of the symmetric tridiagonal T_m (diagonal al, squared
// off-diagonal be2), already shifted and scaled so that its Gershgorin interval is [-1, 1]:
// the sign changes of the Sturm sequence p_0 = 1, p_1 = al_0 - x, p_i = (al_{i-1} - x)
// p_{i-1} - be_{i-2}^2 p_{i-2}.  FP32 (the estimates need a few digits, and this GPU's FP64
// pipe is narrow), division-free; a zero term takes the sign opposite to its predecessor's,
// and the pair is rescaled by 2^-60 (exact) whenever it grows past 2^60.
__device__ int sturm_count_scaled(const float* al, const float* be2, int m, float x) {
  float pm2 = 1.0f, pm1 = al[0] - x;
  int cnt = 0;
  bool neg_prev = false;  // sign of p_0 = 1
  bool neg = pm1 < 0.0f || (pm1 == 0.0f && !neg_prev);
  cnt += neg != neg_prev;
  neg_prev = neg;
#pragma unroll 4
  for (int i = 1; i < m; ++i) {
    const float p = fmaf(al[i] - x, pm1, -be2[i - 1] * pm2);
    neg = p < 0.0f || (p == 0.0f && !neg_prev);
    cnt += neg != neg_prev;
    neg_prev = neg;
    pm2 = pm1;
    pm1 = p;
    if (fabsf(pm1) > 0x1p60f) {
      pm1 *= 0x1p-60f;
      pm2 *= 0x1p-60f;
    }
  }
  return cnt;
}

struct TridiagSmem {
  float al[kLzMaxSteps];
  float be2[kLzMaxSteps];
  float lo[2], hi[2];
  float wlo[32], whi[32];  // per-warp Gershgorin bounds
  int wfirst[32];          // per-warp first point past the target count
};

// Smallest and largest eigenvalues of T_m by multisection with every thread of the block:
// half the threads bracket the smallest, half the largest, each round evaluating one Sturm
// count per thread at evenly spaced points and keeping the sub-interval where the count
// first reaches 1 (smallest) or m (largest); four rounds of 128 points narrow [-1, 1] to
// about 1e-8 of the spectrum's width.  The Gershgorin interval that is mapped to [-1, 1]
// is formed in FP32 by all threads at once (a thread per row, then a block min / max) and
// widened by 2^-16 of its half-width, which covers the roundings of the discs.  Called by
// all threads; results in thread 0.
__device__ void tridiag_extremes_block(const double* al, const double* be, int m, TridiagSmem& ts,
                                       double* lo_out, double* hi_out) {
  const int half = blockDim.x / 2;
  const int grp = threadIdx.x < half ? 0 : 1;
  const int t = threadIdx.x - grp * half;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  float glo = INFINITY, ghi = -INFINITY;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const float a = (float)al[i];
    const float b = (float)be[i];
    const float rad = (i > 0 ? fabsf((float)be[i - 1]) : 0.f) + (i + 1 < m ? fabsf(b) : 0.f);
    glo = fminf(glo, a - rad);
    ghi = fmaxf(ghi, a + rad);
    ts.al[i] = a;
    ts.be2[i] = b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  if (lane == 0) {
    ts.wlo[wid] = glo;
    ts.whi[wid] = ghi;
  }
  if (threadIdx.x < 2) {
    ts.lo[threadIdx.x] = -1.0f;
    ts.hi[threadIdx.x] = 1.0f;
  }
  __syncthreads();
  glo = ts.wlo[0];
  ghi = ts.whi[0];
  for (int w = 1; w < nw; ++w) {
    glo = fminf(glo, ts.wlo[w]);
    ghi = fmaxf(ghi, ts.whi[w]);
  }
  const float c = 0.5f * (glo + ghi);
  const float scale = fmaxf(0.5f * (ghi - glo) * (1.0f + 0x1p-16f), 0x1p-100f);
  const float inv = 1.0f / scale;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    ts.al[i] = (ts.al[i] - c) * inv;
    const float b = ts.be2[i] * inv;
    ts.be2[i] = b * b;
  }
  __syncthreads();
  // A group is a whole number of warps (blockDim a multiple of 64): each warp posts its
  // first point past the target (a ballot), and the group's first thread takes the least.
  const int wpg = (half + 31) >> 5;
  for (int round = 0; round < 4; ++round) {
    const float a = ts.lo[grp], b = ts.hi[grp];
    const float x = a + (b - a) * (float)(t + 1) / (float)(half + 1);
    const int cnt = sturm_count_scaled(ts.al, ts.be2, m, x);
    const unsigned hit = __ballot_sync(0xffffffffu, cnt >= (grp == 0 ? 1 : m));
    if (lane == 0) ts.wfirst[wid] = hit ? (t - lane) + __ffs((int)hit) - 1 : half;
    __syncthreads();
    if (t == 0) {
      int f = half;
      for (int k = 0; k < wpg; ++k) f = min(f, ts.wfirst[grp * wpg + k]);
      const float w = (b - a) / (float)(half + 1);
      ts.lo[grp] = a + w * (float)f;
      ts.hi[grp] = f < half ? a + w * (float)(f + 1) : b;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *lo_out = (double)c + (double)scale * 0.5 * ((double)ts.lo[0] + (double)ts.hi[0]);
    *hi_out = (double)c + (double)scale * 0.5 * ((double)ts.lo[1] + (double)ts.hi[1]);
  }
}

struct LzSmem {
  float part_a[kLzMaxCs * kLzWarps];  // per (CTA, warp) partials, written remotely by every CTA
  float part_b[kLzMaxCs * kLzWarps];
  double alpha[kLzMaxSteps];
  double beta[kLzMaxSteps];
};

// Rows r0 .. r0 + R - 1 of an n x n symmetric matrix (column-major source, column i = row i)
// times the full vector x; y[r - r0] receives the products.  src rows come from shared
// memory (ROWS_IN_SMEM, FP32) or straight from the FP64/FP32 source.  Each warp keeps four
// rows in flight (four independent FMA chains over the same x entries), since one row at a
// time leaves a warp waiting on a single dependent chain.
template <bool ROWS_IN_SMEM>
__device__ __forceinline__ float row_entry(const float* srows, const void* src, int f64, int n, int r0, int rr, int j) {
  if (ROWS_IN_SMEM) return srows[(size_t)rr * n + j];
  if (f64) return (float)__ldg(static_cast<const double*>(src) + (size_t)(r0 + rr) * n + j);
  return __ldg(static_cast<const float*>(src) + (size_t)(r0 + rr) * n + j);
}

template <bool ROWS_IN_SMEM>
__device__ void slice_matvec(int n, int r0, int R, const float* srows, const void* src, int f64, const float* x,
                             float* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int rr = 4 * w; rr < R; rr += 4 * kLzWarps) {
    const int nrow = min(4, R - rr);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int j = lane; j < n; j += 32) {
      const float xv = x[j];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nrow) acc[q] = fmaf(row_entry<ROWS_IN_SMEM>(srows, src, f64, n, r0, rr + q, j), xv, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float v = lz_warp_sum(acc[q]);
      if (lane == 0 && q < nrow) y[rr + q] = v;
    }
  }
}

// As slice_matvec, but each warp stores its rows of y straight into y's copy in every CTA
// of the cluster (lane l < cs writes CTA l; four rows as one 16-byte store where aligned),
// so the product needs no block barrier before the exchange.
template <bool ROWS_IN_SMEM>
__device__ void slice_matvec_push(int n, int r0, int R, const float* srows, const void* src, int f64, const float* x,
                                  float* yfull, int cs) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int rr = 4 * w; rr < R; rr += 4 * kLzWarps) {
    const int nrow = min(4, R - rr);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int j = lane; j < n; j += 32) {
      const float xv = x[j];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nrow) acc[q] = fmaf(row_entry<ROWS_IN_SMEM>(srows, src, f64, n, r0, rr + q, j), xv, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = lz_warp_sum(acc[q]);  // every lane holds the sums
    if (lane < cs) {
      float* dst = yfull + r0 + rr;
      if (nrow == 4 && (lz_smem_u32(dst) & 15u) == 0u) {
        st_remote4(dst, (uint32_t)lane, acc);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nrow) st_remote(dst + q, (uint32_t)lane, acc[q]);
      }
    }
  }
}

// Warp w of CTA `rank` publishes its partial v into slot rank * kLzWarps + w of every CTA.
__device__ __forceinline__ void publish_partial(float* slots, float v, int rank, int cs) {
  v = lz_warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane < cs) st_remote(&slots[rank * kLzWarps + w], (uint32_t)lane, v);
}

// Sum of the cs * kLzWarps published partials, formed by every warp in the same order (so
// every thread of every CTA holds the same value).
__device__ __forceinline__ float gather_partials(const float* slots, int cs) {
  const int lane = threadIdx.x & 31;
  float v = 0.f;
  for (int i = lane; i < cs * kLzWarps; i += 32) v += slots[i];
  return lz_warp_sum(v);
}

// dst[0 .. cnt) = FP32 copy of src[off .. off + cnt).  An FP32 source whose slice and
// destination are 16-byte aligned moves as float4, eight loads in flight per thread (the
// slice is read once per launch, so its latency is paid up front); otherwise entry by entry.
__device__ void load_rows(float* dst, const void* src, int f64, size_t off, size_t cnt) {
  const float* s32 = static_cast<const float*>(src) + off;
  if (!f64 && ((reinterpret_cast<uintptr_t>(s32) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    constexpr int kB = 8;
    const size_t c4 = cnt / 4;
    const float4* s4 = reinterpret_cast<const float4*>(s32);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (size_t base = threadIdx.x; base < c4; base += (size_t)kB * blockDim.x) {
      float4 v[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const size_t e = base + (size_t)u * blockDim.x;
        if (e < c4) v[u] = __ldg(s4 + e);
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const size_t e = base + (size_t)u * blockDim.x;
        if (e < c4) d4[e] = v[u];
      }
    }
    for (size_t e = 4 * c4 + threadIdx.x; e < cnt; e += blockDim.x) dst[e] = __ldg(s32 + e);
    return;
  }
  for (size_t e = threadIdx.x; e < cnt; e += blockDim.x)
    dst[e] = f64 ? (float)__ldg(static_cast<const double*>(src) + off + e) : __ldg(s32 + e);
}

// Rows held in registers (standard Lanczos, n <= 512, at most 32 rows a CTA): warp w keeps
// rows 4w .. 4w + 3 of the slice and lane l their columns l + 32k (k < 16), zero past the
// ends, so a step reads only x from shared memory.  The sums run in the same order as
// slice_matvec's (k ascending, the zero padding adds nothing), so the products are the same.
constexpr int kRegCols = 16;
constexpr int kRegRowsPerCta = 4 * kLzWarps;

__device__ __forceinline__ void load_rows_reg(float (&rv)[4][kRegCols], const void* src, int f64, int n, int r0,
                                              int nr) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // one branch on the source type, outside the loops, so all 64 loads issue before the
  // first is used
  if (f64) {
    const double* s64 = static_cast<const double*>(src);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < kRegCols; ++k) {
        const int rr = 4 * w + q, j = lane + 32 * k;
        rv[q][k] = rr < nr && j < n ? (float)__ldg(s64 + (size_t)(r0 + rr) * n + j) : 0.f;
      }
  } else {
    const float* s32 = static_cast<const float*>(src);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < kRegCols; ++k) {
        const int rr = 4 * w + q, j = lane + 32 * k;
        rv[q][k] = rr < nr && j < n ? __ldg(s32 + (size_t)(r0 + rr) * n + j) : 0.f;
      }
  }
}

__device__ __forceinline__ void matvec_push_reg(const float (&rv)[4][kRegCols], int n, int r0, int nr, const float* x,
                                                float* yfull, int cs) {
  const int lane = threadIdx.x & 31, rr = 4 * (threadIdx.x >> 5);
  if (rr >= nr) return;  // warp-uniform
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kRegCols; ++k) {
    const int j = lane + 32 * k;
    const float xv = j < n ? x[j] : 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fmaf(rv[q][k], xv, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = lz_warp_sum(acc[q]);
  if (lane < cs) {
    const int nrow = min(4, nr - rr);
    float* dst = yfull + r0 + rr;
    if (nrow == 4 && (lz_smem_u32(dst) & 15u) == 0u) {
      st_remote4(dst, (uint32_t)lane, acc);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nrow) st_remote(dst + q, (uint32_t)lane, acc[q]);
    }
  }
}

struct LzArgs {
  LanczosProblem prob[4];
  int count;
  int cs;
};

// ROWS: where a CTA's rows live for all steps: 0 read from L2 each step, 1 shared memory,
// 2 registers (standard Lanczos only).
template <int ROWS>
__global__ void __launch_bounds__(kLzThreads, 1) lanczos_cluster_kernel(LzArgs args) {
  constexpr bool SMEM = ROWS == 1;
  const int cs = args.cs;
  const LanczosProblem P = args.prob[blockIdx.x / cs];
  const int rank = (int)cluster_rank();
  const int n = (int)P.n;
  const bool gen = P.M1 != nullptr;
  const int R = (n + cs - 1) / cs;
  const int r0 = min(n, rank * R);
  const int nr = max(0, min(n, r0 + R) - r0);
  const int steps = min(P.steps, kLzMaxSteps);
  extern __shared__ __align__(16) float lsm[];
  float* rows2 = lsm;
  float* rows1 = rows2 + (SMEM ? (size_t)R * n : 0);
  float* tF = rows1 + (SMEM && args.prob[0].M1 != nullptr ? (size_t)R * n : 0);
  const int n4 = (n + 3) & ~3;
  float* uF = tF + n4;
  float* sF = uF + n4;
  float* wF = sF + n4;  // the second copy of y (standard Lanczos)
  float* yS = wF + n4;  // this CTA's rows of M2 t
  float* sS = yS + R;  // and of M1 u
  __shared__ LzSmem sm;
  float rv[4][kRegCols];
  if (ROWS == 2) load_rows_reg(rv, P.M2, P.m2_f64, n, r0, nr);
  if (SMEM) {
    load_rows(rows2, P.M2, P.m2_f64, (size_t)r0 * n, (size_t)nr * n);
    if (gen) load_rows(rows1, P.M1, P.m1_f64, (size_t)r0 * n, (size_t)nr * n);
  }
  // Start vector: a fixed deterministic pattern with components along every eigenvector.
  for (int s = threadIdx.x; s < n; s += blockDim.x) uF[s] = 1.0f + 0.5f * __cosf(0.7f * (float)s + 0.3f);
  cluster_sync();  // every CTA of the cluster runs before any shared memory is addressed remotely
  // v_0 = e / ||e||_M1 and t_0 = M1 v_0 (thread i of each CTA owns entry r0 + i of the slices)
  float nrm2;
  if (gen) {
    slice_matvec<SMEM>(n, r0, nr, rows1, P.M1, P.m1_f64, uF, sS);
    __syncthreads();
    const int i = threadIdx.x;
    float part = 0.f;
    if (i < nr) {
      part = uF[r0 + i] * sS[i];
      for (int rk = 0; rk < cs; ++rk) st_remote(&tF[r0 + i], (uint32_t)rk, sS[i]);
    }
    publish_partial(sm.part_b, part, rank, cs);
    cluster_sync();
    nrm2 = gather_partials(sm.part_b, cs);
  } else {
    float part = 0.f;
    for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) part = fmaf(uF[s2], uF[s2], part);
    part = lz_warp_sum(part);  // every CTA holds all of e: its own sum, no exchange
    if ((threadIdx.x & 31) == 0) sm.part_b[threadIdx.x >> 5] = part;
    __syncthreads();
    nrm2 = gather_partials(sm.part_b, 1);
    for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) tF[s2] = uF[s2];
  }
  const float inv0 = rsqrtf(nrm2);
  __syncthreads();
  for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) tF[s2] *= inv0;
  int m = 0;
  if (!gen) {
    // Standard Lanczos (M1 = I), one cluster barrier per step: every warp pushes its rows of
    // y = M2 v_j into every CTA's copy of y (two copies, alternating by step: a CTA one step
    // ahead writes the other), and after the barrier each CTA forms alpha_j = y^T v_j,
    // u = y - alpha_j v_j - beta_{j-1} v_{j-1}, beta_j = ||u|| and v_{j+1} = u / beta_j over
    // the whole vector itself: the same vectors and the same order of sums in every CTA,
    // so every CTA holds the same values.  Each thread updates the entries it sums, so the
    // two reductions take one block barrier each and the step three in all.
    float* vF = tF;                                   // v_j (full)
    float* vpF = sF;                                  // v_{j-1}
    // y: two copies, wF at even steps (uF holds the start vector until every CTA has passed
    // step 0's barrier), uF at odd steps
    __shared__ float red2[2][kLzWarps];               // alternating: a call reuses its buffer two calls later
    auto block_sum = [&](float v, int buf) {
      v = lz_warp_sum(v);
      if ((threadIdx.x & 31) == 0) red2[buf][threadIdx.x >> 5] = v;
      __syncthreads();
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < kLzWarps; ++w) t += red2[buf][w];
      return t;
    };
    for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) vpF[s2] = 0.f;
    float beta_prev = 0.f;
    __syncthreads();
    for (int j = 0; j < steps; ++j) {
      float* yF = (j & 1) ? uF : wF;
      if (ROWS == 2) {
        matvec_push_reg(rv, n, r0, nr, vF, yF, cs);  // this CTA's rows of M2 v_j
      } else {
        slice_matvec_push<SMEM>(n, r0, nr, rows2, P.M2, P.m2_f64, vF, yF, cs);
      }
      cluster_sync();
      float pa = 0.f;
      for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) pa = fmaf(yF[s2], vF[s2], pa);
      const float alpha = block_sum(pa, 0);
      float pb = 0.f;
      for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) {
        const float u = fmaf(-beta_prev, vpF[s2], fmaf(-alpha, vF[s2], yF[s2]));
        yF[s2] = u;
        pb = fmaf(u, u, pb);
      }
      const float beta = sqrtf(fmaxf(block_sum(pb, 1), 0.f));
      if (threadIdx.x == 0) {
        sm.alpha[j] = (double)alpha;
        sm.beta[j] = (double)beta;
      }
      m = j + 1;
      if (!(beta > 1e-6f * fabsf(alpha)) || !isfinite(beta)) break;  // invariant subspace (same in every CTA)
      const float ib = 1.0f / beta;
      for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) {
        vpF[s2] = vF[s2];
        vF[s2] = yF[s2] * ib;
      }
      beta_prev = beta;
      __syncthreads();
    }
  }
  float vcur = 0.f, vprev = 0.f;  // thread i: v_j and v_{j-1} at entry r0 + i
  if (threadIdx.x < nr) vcur = uF[r0 + threadIdx.x] * inv0;
  __syncthreads();
  float beta_prev = 0.f;
  for (int j = 0; gen && j < steps; ++j) {
    slice_matvec<SMEM>(n, r0, nr, rows2, P.M2, P.m2_f64, tF, yS);  // y = C v_j = M2 t_j
    __syncthreads();
    const int i = threadIdx.x;
    const bool mine = i < nr;
    const float y = mine ? yS[i] : 0.f;
    publish_partial(sm.part_a, mine ? y * tF[r0 + i] : 0.f, rank, cs);
    cluster_sync();
    const float alpha = gather_partials(sm.part_a, cs);  // <C v_j, v_j>_M1 = y^T t_j
    const float u = mine ? fmaf(-beta_prev, vprev, fmaf(-alpha, vcur, y)) : 0.f;
    float b2part;
    if (gen) {
      if (mine)
        for (int rk = 0; rk < cs; ++rk) st_remote(&uF[r0 + i], (uint32_t)rk, u);
      cluster_sync();
      slice_matvec<SMEM>(n, r0, nr, rows1, P.M1, P.m1_f64, uF, sS);  // s = M1 u
      __syncthreads();
      const float sv = mine ? sS[i] : 0.f;
      if (mine)
        for (int rk = 0; rk < cs; ++rk) st_remote(&sF[r0 + i], (uint32_t)rk, sv);
      b2part = u * sv;
    } else {
      if (mine)
        for (int rk = 0; rk < cs; ++rk) st_remote(&uF[r0 + i], (uint32_t)rk, u);
      b2part = u * u;
    }
    publish_partial(sm.part_b, b2part, rank, cs);
    cluster_sync();
    const float beta = sqrtf(fmaxf(gather_partials(sm.part_b, cs), 0.f));
    if (threadIdx.x == 0) {
      sm.alpha[j] = (double)alpha;
      sm.beta[j] = (double)beta;
    }
    m = j + 1;
    if (!(beta > 1e-6f * fabsf(alpha)) || !isfinite(beta)) break;  // invariant subspace (same in every thread)
    const float ib = 1.0f / beta;
    vprev = vcur;
    vcur = u * ib;
    const float* next_t = gen ? sF : uF;
    for (int s2 = threadIdx.x; s2 < n; s2 += blockDim.x) tF[s2] = next_t[s2] * ib;
    beta_prev = beta;
    __syncthreads();
  }
  __syncthreads();
  if (rank == 0) {
    __shared__ TridiagSmem ts;
    double lo = 0.0, hi = 0.0;
    if (m > 0) tridiag_extremes_block(sm.alpha, sm.beta, m, ts, &lo, &hi);
    if (threadIdx.x == 0) {
      P.out[0] = lo;
      P.out[1] = hi;
      P.out[2] = (double)m;
    }
  }
  cluster_sync();  // no CTA leaves while another may still store into its shared memory
}

size_t lz_smem(int64_t n, int cs, bool rows, bool any_gen) {
  const int64_t R = (n + cs - 1) / cs;
  return sizeof(float) * (size_t)((rows ? R * n * (any_gen ? 2 : 1) : 0) + 4 * ((n + 3) & ~3) + 2 * R + 4);
}

template <int ROWS>
cudaError_t lz_launch(const LzArgs& a, size_t smem, cudaStream_t s) {
  auto kern = lanczos_cluster_kernel<ROWS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)  // placed beside the cooperative inverses: keep the SMs' carveout at its largest
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (a.cs > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.count * a.cs), 1, 1);
  cfg.blockDim = dim3(kLzThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  note_launch();
  return e;
}

// est[0..2] = lambda_min(H), lambda_max(H), rho from the problems' outputs; est[3] = kappa,
// est[4] = 1 / kappa^2.  A non-positive lambda_min(H) or a rho >= 1 raises est[7] to
// ILS_ERR_NOT_SPD (condition (1.3) fails).  gram_bound (matrix-free route, where H is never
// formed): kap_out holds Abar1's extremes and kappa is the bound kappa(Abar1) / (1 - rho),
// from lambda_max(H) <= lambda_max(Abar1) and lambda_min(H) >= lambda_min(Abar1) (1 - rho)
// (H = Abar1^{1/2} (I - M) Abar1^{1/2} with the eigenvalues of M in [0, rho]).
__global__ void estimates_finish_kernel(const double* kap_out, const double* rho_out, double* est, int gram_bound) {
  if (threadIdx.x != 0) return;
  double status = est[7];
  if (rho_out) {
    est[2] = rho_out[1];
    est[6] = rho_out[2];
    if (!(rho_out[1] < 1.0)) status = (double)ILS_ERR_NOT_SPD;
  }
  if (kap_out) {
    double lo = kap_out[0], hi = kap_out[1];
    if (gram_bound) lo = (rho_out && rho_out[1] < 1.0) ? lo * (1.0 - rho_out[1]) : 0.0;
    est[0] = lo;
    est[1] = hi;
    est[5] = kap_out[2];
    const double kappa = lo > 0.0 ? hi / lo : INFINITY;
    est[3] = kappa;
    est[4] = isfinite(kappa) && kappa > 0.0 ? 1.0 / (kappa * kappa) : 0.0;
    if (!(lo > 0.0)) status = (double)ILS_ERR_NOT_SPD;
  }
  est[7] = status;
}

// ---- matrix-free route: rho by Lanczos on C = (A_2^T A_2) P in the P inner product, one step
// per launch pair (the A_2 stream of stream.cu, then this CTA), state in `w`:
//   w[0 .. n)    v_j (float)      w[n .. 2n)   v_{j-1}       w[2n .. 3n) u
//   w[3n .. 4n)  s = P u          then, as doubles from an aligned offset: t_j (n, the
//   stream's input), alpha and beta (kLzMaxSteps each), beta_{j-1}, steps taken, stopped.
// P is FP32 (n <= 512).
constexpr int kMfThreads = 512;

// Block sum of FP32 shares, accumulated in FP64 by thread 0 alone and broadcast (as FP64)
// through shared memory.
__device__ double mf_block_sum(float v, float* red, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = lz_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kMfThreads / 32; ++i) s += (double)red[i];
    *out = s;
  }
  __syncthreads();
  return *out;
}

// y := M x for the n x n FP32 matrix M (column i = row i): a warp per row.
__device__ void mf_matvec(int n, const float* M, const float* x, float* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = w; r < n; r += kMfThreads / 32) {
    float acc = 0.f;
    for (int j = lane; j < n; j += 32) acc = fmaf(__ldg(M + (size_t)r * n + j), x[j], acc);
    acc = lz_warp_sum(acc);
    if (lane == 0) y[r] = acc;
  }
}

struct MfState {
  float* v;
  float* vp;
  float* u;
  float* s;
  double* t;
  double* alpha;
  double* beta;
  double* scal;  // [0] beta_{j-1}, [1] steps taken, [2] stopped
};

__device__ MfState mf_state(int n, float* w) {
  MfState st;
  st.v = w;
  st.vp = w + n;
  st.u = w + 2 * n;
  st.s = w + 3 * n;
  double* d = reinterpret_cast<double*>(w + ((4 * n + 3) & ~3));
  st.t = d;
  st.alpha = d + n;
  st.beta = st.alpha + kLzMaxSteps;
  st.scal = st.beta + kLzMaxSteps;
  return st;
}

__global__ void __launch_bounds__(kMfThreads) lz_mf_init_kernel(int n, const float* P, float* w) {
  __shared__ float red[kMfThreads / 32];
  __shared__ double sum;
  __shared__ float inv;
  MfState st = mf_state(n, w);
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    st.u[s] = 1.0f + 0.5f * __cosf(0.7f * (float)s + 0.3f);
    st.vp[s] = 0.f;
  }
  __syncthreads();
  mf_matvec(n, P, st.u, st.s);
  __syncthreads();
  float part = 0.f;
  for (int s = threadIdx.x; s < n; s += blockDim.x) part = fmaf(st.u[s], st.s[s], part);
  mf_block_sum(part, red, &sum);
  if (threadIdx.x == 0) inv = (float)(1.0 / sqrt(sum));
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    st.v[s] = st.u[s] * inv;
    st.t[s] = (double)(st.s[s] * inv);
  }
  if (threadIdx.x == 0) {
    st.scal[0] = 0.0;
    st.scal[1] = 0.0;
    st.scal[2] = 0.0;
  }
}

// One step after y = A_2^T (A_2 t_j) (FP64, from the stream).  Scalars in thread 0.
__global__ void __launch_bounds__(kMfThreads) lz_mf_step_kernel(int n, const float* P, const double* y, float* w,
                                                                int j) {
  __shared__ float red[kMfThreads / 32];
  __shared__ double sum;
  __shared__ float sc[3];
  __shared__ int stopped;
  MfState st = mf_state(n, w);
  if (threadIdx.x == 0) stopped = st.scal[2] != 0.0;
  __syncthreads();
  if (stopped) return;  // stopped at an invariant subspace
  float part = 0.f;
  for (int s = threadIdx.x; s < n; s += blockDim.x) part = fmaf((float)y[s], (float)st.t[s], part);
  const double alpha = mf_block_sum(part, red, &sum);
  if (threadIdx.x == 0) {
    sc[0] = (float)alpha;
    sc[1] = (float)st.scal[0];
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x)
    st.u[s] = fmaf(-sc[1], st.vp[s], fmaf(-sc[0], st.v[s], (float)y[s]));
  __syncthreads();
  mf_matvec(n, P, st.u, st.s);
  __syncthreads();
  part = 0.f;
  for (int s = threadIdx.x; s < n; s += blockDim.x) part = fmaf(st.u[s], st.s[s], part);
  const double b2 = mf_block_sum(part, red, &sum);
  if (threadIdx.x == 0) {
    const double beta = sqrt(fmax(b2, 0.0));
    const bool stop = !(beta > 1e-10 * fabs(alpha)) || !isfinite(beta);
    sc[2] = stop ? 0.f : (float)(1.0 / beta);
    st.alpha[j] = alpha;
    st.beta[j] = beta;
    st.scal[0] = beta;
    st.scal[1] = (double)(j + 1);
    if (stop) st.scal[2] = 1.0;
  }
  __syncthreads();
  const float ib = sc[2];
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    st.vp[s] = st.v[s];
    st.v[s] = st.u[s] * ib;
    st.t[s] = (double)(st.s[s] * ib);
  }
}

__global__ void lz_mf_finish_kernel(int n, float* w, double* out) {
  __shared__ TridiagSmem ts;
  MfState st = mf_state(n, w);
  const int m = (int)st.scal[1];
  double lo = 0.0, hi = 0.0;
  if (m > 0) tridiag_extremes_block(st.alpha, st.beta, m, ts, &lo, &hi);
  if (threadIdx.x == 0) {
    out[0] = lo;
    out[1] = hi;
    out[2] = (double)m;
  }
}

}  // namespace

cudaError_t lanczos_extremes(int count, const LanczosProblem* probs, cudaStream_t s) {
  if (count < 1 || count > 4) return cudaErrorInvalidValue;
  LzArgs a;
  bool any_gen = false;
  for (int i = 0; i < count; ++i) {
    if (probs[i].n != probs[0].n || probs[i].n < 1) return cudaErrorInvalidValue;
    a.prob[i] = probs[i];
    any_gen = any_gen || probs[i].M1 != nullptr;
  }
  // the problem with M1 goes first: the shared-memory layout is sized from problem 0
  for (int i = 1; i < count && a.prob[0].M1 == nullptr; ++i)
    if (a.prob[i].M1) std::swap(a.prob[0], a.prob[i]);
  a.count = count;
  const int64_t n = probs[0].n;
  const size_t limit = 220 * 1024;
  // A thread of each CTA owns one row of the CTA's slice, so a slice holds at most kLzThreads
  // rows: 8 CTAs up to n = 2048, 16 up to n = 4096.  The rows stay in shared memory where
  // they fit, else each step reads them from L2.
  // Standard Lanczos takes 16 CTAs first: its step is one barrier after the product, so
  // half the rows per CTA shorten the step (and half the shared memory lets the cluster
  // share SMs with the setup's other kernels).
  const int order[2] = {any_gen ? 8 : 16, any_gen ? 16 : 8};
  // Rows in registers first (standard Lanczos, n <= 512), then in shared memory, then from L2.
  for (int pass = 0; pass < 3; ++pass) {
    for (int cs : order) {
      if ((n + cs - 1) / cs > kLzThreads) continue;
      a.cs = cs;
      cudaError_t e;
      if (pass == 0) {
        if (any_gen || n > 32 * kRegCols || (n + cs - 1) / cs > kRegRowsPerCta) continue;
        e = lz_launch<2>(a, lz_smem(n, cs, false, false), s);
      } else if (pass == 1) {
        const size_t sm_rows = lz_smem(n, cs, true, any_gen);
        if (sm_rows > limit) continue;
        e = lz_launch<1>(a, sm_rows, s);
      } else {
        e = lz_launch<0>(a, lz_smem(n, cs, false, any_gen), s);
      }
      if (e == cudaSuccess) return e;
      cudaGetLastError();  // this cluster size is not available: try the next
    }
  }
  return cudaErrorNotSupported;
}

size_t lz_mf_work_floats(int64_t n) { return (size_t)((4 * n + 3) & ~3) + 2 * ((size_t)n + 2 * kLzMaxSteps + 4); }

cudaError_t lz_mf_init(int64_t n, const float* P, float* w, cudaStream_t s) {
  lz_mf_init_kernel<<<1, kMfThreads, 0, s>>>((int)n, P, w);
  note_launch();
  return cudaGetLastError();
}

double* lz_mf_vector(int64_t n, float* w) { return reinterpret_cast<double*>(w + ((4 * n + 3) & ~3)); }

cudaError_t lz_mf_step(int64_t n, const float* P, const double* y, float* w, int j, cudaStream_t s) {
  lz_mf_step_kernel<<<1, kMfThreads, 0, s>>>((int)n, P, y, w, j);
  note_launch();
  return cudaGetLastError();
}

cudaError_t lz_mf_finish(int64_t n, float* w, double* out, cudaStream_t s) {
  lz_mf_finish_kernel<<<1, 256, 0, s>>>((int)n, w, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t estimates_finish(const double* kap_out, const double* rho_out, double* est, cudaStream_t s,
                             bool gram_bound) {
  estimates_finish_kernel<<<1, 32, 0, s>>>(kap_out, rho_out, est, gram_bound ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
