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
__device__ __forceinline__ void st_remote_d(const double* local, uint32_t rank, double v) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(lz_smem_u32(local)), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(v) : "memory");
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

// Number of eigenvalues of the symmetric tridiagonal (alpha, beta) below x (Sturm count).
__device__ int sturm_count(const double* al, const double* be, int m, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
    d = (al[i] - x) - (i > 0 ? b2 / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Smallest and largest eigenvalues of T_m by bisection inside the Gershgorin interval.
__device__ void tridiag_extremes(const double* al, const double* be, int m, double* lo_out, double* hi_out) {
  double glo = 1e300, ghi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double rad = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
    glo = fmin(glo, al[i] - rad);
    ghi = fmax(ghi, al[i] + rad);
  }
  for (int which = 0; which < 2; ++which) {
    double a = glo, b = ghi;
    for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
      const double mid = 0.5 * (a + b);
      const int c = sturm_count(al, be, m, mid);
      // which 0: the smallest eigenvalue is below mid iff c >= 1; which 1: the largest iff c >= m
      if (which == 0 ? (c >= 1) : (c >= m)) b = mid;
      else a = mid;
    }
    (which == 0 ? *lo_out : *hi_out) = 0.5 * (a + b);
  }
}

struct LzSmem {
  double part_a[kLzMaxCs];
  double part_b[kLzMaxCs];
  double alpha[kLzMaxSteps];
  double beta[kLzMaxSteps];
  double warp_part[kLzWarps];
};

// Rows r0 .. r0 + R - 1 of an n x n symmetric matrix (column-major source, column i = row i)
// times the full vector x; y[r - r0] receives the products.  src rows come from shared
// memory (ROWS_IN_SMEM, FP32) or straight from the FP64/FP32 source.
template <bool ROWS_IN_SMEM>
__device__ void slice_matvec(int n, int r0, int R, const float* srows, const void* src, int f64, const float* x,
                             float* y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int rr = w; rr < R; rr += kLzWarps) {
    float acc = 0.f;
    if (ROWS_IN_SMEM) {
      const float* row = srows + (size_t)rr * n;
      for (int j = lane; j < n; j += 32) acc = fmaf(row[j], x[j], acc);
    } else if (f64) {
      const double* row = static_cast<const double*>(src) + (size_t)(r0 + rr) * n;
      for (int j = lane; j < n; j += 32) acc = fmaf((float)__ldg(row + j), x[j], acc);
    } else {
      const float* row = static_cast<const float*>(src) + (size_t)(r0 + rr) * n;
      for (int j = lane; j < n; j += 32) acc = fmaf(__ldg(row + j), x[j], acc);
    }
    acc = lz_warp_sum(acc);
    if (lane == 0) y[rr] = acc;
  }
}

// Sum over the CTA of v (every thread passes its share); the result is valid in thread 0.
__device__ double cta_sum(double v, LzSmem& sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sm.warp_part[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kLzWarps; ++i) s += sm.warp_part[i];
  return s;
}

struct LzArgs {
  LanczosProblem prob[4];
  int count;
  int cs;
};

template <bool SMEM>
__global__ void __launch_bounds__(kLzThreads, 1) lanczos_cluster_kernel(LzArgs args) {
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
  float* uF = tF + n;
  float* sF = uF + n;
  float* vS = sF + n;
  float* vpS = vS + R;
  float* yS = vpS + R;
  float* uS = yS + R;
  float* sS = uS + R;
  __shared__ LzSmem sm;
  if (SMEM) {
    for (size_t e = threadIdx.x; e < (size_t)nr * n; e += blockDim.x) {
      const size_t src = (size_t)r0 * n + e;
      rows2[e] = P.m2_f64 ? (float)__ldg(static_cast<const double*>(P.M2) + src) : __ldg(static_cast<const float*>(P.M2) + src);
      if (gen) rows1[e] = P.m1_f64 ? (float)__ldg(static_cast<const double*>(P.M1) + src) : __ldg(static_cast<const float*>(P.M1) + src);
    }
  }
  // Start vector: a fixed deterministic pattern with components along every eigenvector.
  for (int s = threadIdx.x; s < n; s += blockDim.x) uF[s] = 1.0f + 0.5f * __cosf(0.7f * (float)s + 0.3f);
  cluster_sync();  // every CTA of the cluster runs before any shared memory is addressed remotely
  double nrm2;
  if (gen) {
    slice_matvec<SMEM>(n, r0, nr, rows1, P.M1, P.m1_f64, uF, sS);
    __syncthreads();
    double part = 0.0;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) part += (double)uF[r0 + i] * (double)sS[i];
    part = cta_sum(part, sm);
    if (threadIdx.x == 0)
      for (int rk = 0; rk < cs; ++rk) st_remote_d(&sm.part_b[rank], (uint32_t)rk, part);
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
      for (int rk = 0; rk < cs; ++rk) st_remote(&tF[r0 + i], (uint32_t)rk, sS[i]);
    cluster_sync();
    nrm2 = 0.0;
    for (int rk = 0; rk < cs; ++rk) nrm2 += sm.part_b[rk];
  } else {
    double part = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) part += (double)uF[s] * (double)uF[s];
    part = cta_sum(part, sm);
    if (threadIdx.x == 0) sm.part_b[0] = part;
    __syncthreads();
    nrm2 = sm.part_b[0];
    for (int s = threadIdx.x; s < n; s += blockDim.x) tF[s] = uF[s];
  }
  const float inv0 = (float)(1.0 / sqrt(nrm2));
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) tF[s] *= inv0;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    vS[i] = uF[r0 + i] * inv0;
    vpS[i] = 0.f;
  }
  __syncthreads();
  double beta_prev = 0.0;
  int m = 0;
  for (int j = 0; j < steps; ++j) {
    slice_matvec<SMEM>(n, r0, nr, rows2, P.M2, P.m2_f64, tF, yS);  // y = C v_j = M2 t_j
    __syncthreads();
    double part = 0.0;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) part += (double)yS[i] * (double)tF[r0 + i];
    part = cta_sum(part, sm);
    if (threadIdx.x == 0)
      for (int rk = 0; rk < cs; ++rk) st_remote_d(&sm.part_a[rank], (uint32_t)rk, part);
    cluster_sync();
    double alpha = 0.0;
    for (int rk = 0; rk < cs; ++rk) alpha += sm.part_a[rk];  // <C v_j, v_j>_M1 = y^T t_j
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
      uS[i] = (float)((double)yS[i] - alpha * (double)vS[i] - beta_prev * (double)vpS[i]);
    __syncthreads();
    if (gen) {
      for (int i = threadIdx.x; i < nr; i += blockDim.x)
        for (int rk = 0; rk < cs; ++rk) st_remote(&uF[r0 + i], (uint32_t)rk, uS[i]);
      cluster_sync();
      slice_matvec<SMEM>(n, r0, nr, rows1, P.M1, P.m1_f64, uF, sS);  // s = M1 u
      __syncthreads();
      part = 0.0;
      for (int i = threadIdx.x; i < nr; i += blockDim.x) part += (double)uS[i] * (double)sS[i];
      part = cta_sum(part, sm);
      if (threadIdx.x == 0)
        for (int rk = 0; rk < cs; ++rk) st_remote_d(&sm.part_b[rank], (uint32_t)rk, part);
      for (int i = threadIdx.x; i < nr; i += blockDim.x)
        for (int rk = 0; rk < cs; ++rk) st_remote(&sF[r0 + i], (uint32_t)rk, sS[i]);
      cluster_sync();
    } else {
      part = 0.0;
      for (int i = threadIdx.x; i < nr; i += blockDim.x) part += (double)uS[i] * (double)uS[i];
      part = cta_sum(part, sm);
      if (threadIdx.x == 0)
        for (int rk = 0; rk < cs; ++rk) st_remote_d(&sm.part_b[rank], (uint32_t)rk, part);
      for (int i = threadIdx.x; i < nr; i += blockDim.x)
        for (int rk = 0; rk < cs; ++rk) st_remote(&uF[r0 + i], (uint32_t)rk, uS[i]);
      cluster_sync();
    }
    double b2 = 0.0;
    for (int rk = 0; rk < cs; ++rk) b2 += sm.part_b[rk];
    const double beta = sqrt(fmax(b2, 0.0));
    if (threadIdx.x == 0) {
      sm.alpha[j] = alpha;
      sm.beta[j] = beta;
    }
    m = j + 1;
    if (!(beta > 1e-10 * fabs(alpha)) || !isfinite(beta)) break;  // invariant subspace (or breakdown)
    const float ib = (float)(1.0 / beta);
    const float* next_t = gen ? sF : uF;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      vpS[i] = vS[i];
      vS[i] = uS[i] * ib;
    }
    for (int s = threadIdx.x; s < n; s += blockDim.x) tF[s] = next_t[s] * ib;
    beta_prev = beta;
    __syncthreads();
  }
  __syncthreads();
  if (rank == 0 && threadIdx.x == 0) {
    double lo = 0.0, hi = 0.0;
    if (m > 0) tridiag_extremes(sm.alpha, sm.beta, m, &lo, &hi);
    P.out[0] = lo;
    P.out[1] = hi;
    P.out[2] = (double)m;
  }
  cluster_sync();  // no CTA leaves while another may still store into its shared memory
}

size_t lz_smem(int64_t n, int cs, bool rows, bool any_gen) {
  const int64_t R = (n + cs - 1) / cs;
  return sizeof(float) * (size_t)((rows ? R * n * (any_gen ? 2 : 1) : 0) + 3 * n + 5 * R + 4);
}

template <bool SMEM>
cudaError_t lz_launch(const LzArgs& a, size_t smem, cudaStream_t s) {
  auto kern = lanczos_cluster_kernel<SMEM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

__device__ __forceinline__ double mf_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < kMfThreads / 32; ++i) s += red[i];
  return s;
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
  __shared__ double red[kMfThreads / 32];
  MfState st = mf_state(n, w);
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    st.u[s] = 1.0f + 0.5f * __cosf(0.7f * (float)s + 0.3f);
    st.vp[s] = 0.f;
  }
  __syncthreads();
  mf_matvec(n, P, st.u, st.s);
  __syncthreads();
  double part = 0.0;
  for (int s = threadIdx.x; s < n; s += blockDim.x) part += (double)st.u[s] * (double)st.s[s];
  const double inv = 1.0 / sqrt(mf_block_sum(part, red));
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    st.v[s] = (float)(st.u[s] * inv);
    st.t[s] = st.s[s] * inv;
  }
  if (threadIdx.x == 0) {
    st.scal[0] = 0.0;
    st.scal[1] = 0.0;
    st.scal[2] = 0.0;
  }
}

// One step after y = A_2^T (A_2 t_j) (FP64, from the stream).
__global__ void __launch_bounds__(kMfThreads) lz_mf_step_kernel(int n, const float* P, const double* y, float* w,
                                                                int j) {
  __shared__ double red[kMfThreads / 32];
  MfState st = mf_state(n, w);
  if (st.scal[2] != 0.0) return;  // stopped at an invariant subspace
  double part = 0.0;
  for (int s = threadIdx.x; s < n; s += blockDim.x) part += y[s] * st.t[s];
  const double alpha = mf_block_sum(part, red);
  const double bprev = st.scal[0];
  for (int s = threadIdx.x; s < n; s += blockDim.x)
    st.u[s] = (float)(y[s] - alpha * (double)st.v[s] - bprev * (double)st.vp[s]);
  __syncthreads();
  mf_matvec(n, P, st.u, st.s);
  __syncthreads();
  part = 0.0;
  for (int s = threadIdx.x; s < n; s += blockDim.x) part += (double)st.u[s] * (double)st.s[s];
  const double beta = sqrt(fmax(mf_block_sum(part, red), 0.0));
  const bool stop = !(beta > 1e-10 * fabs(alpha)) || !isfinite(beta);
  const double ib = stop ? 0.0 : 1.0 / beta;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    st.vp[s] = st.v[s];
    st.v[s] = (float)(st.u[s] * ib);
    st.t[s] = st.s[s] * ib;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st.alpha[j] = alpha;
    st.beta[j] = beta;
    st.scal[0] = beta;
    st.scal[1] = (double)(j + 1);
    if (stop) st.scal[2] = 1.0;
  }
}

__global__ void lz_mf_finish_kernel(int n, float* w, double* out) {
  if (threadIdx.x != 0) return;
  MfState st = mf_state(n, w);
  const int m = (int)st.scal[1];
  double lo = 0.0, hi = 0.0;
  if (m > 0) tridiag_extremes(st.alpha, st.beta, m, &lo, &hi);
  out[0] = lo;
  out[1] = hi;
  out[2] = (double)m;
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
  for (int cs : {16, 8}) {
    a.cs = cs;
    const size_t sm_rows = lz_smem(n, cs, true, any_gen);
    cudaError_t e;
    if (sm_rows <= limit) e = lz_launch<true>(a, sm_rows, s);
    else e = lz_launch<false>(a, lz_smem(n, cs, false, any_gen), s);
    if (e == cudaSuccess) return e;
    cudaGetLastError();  // cluster size not available: try the portable size
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
  lz_mf_finish_kernel<<<1, 32, 0, s>>>((int)n, w, out);
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
