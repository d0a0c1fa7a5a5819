// Sparse A in CSR: the setup products and the parts of the solve that touch A.
//
// The setup transposes A to CSC (columns of A_1 are what the RK and RGS steps of Alg. 2
// read), sorts every column by row so that A_1's entries are a prefix of each column, and
// forms the dense n x n Gram matrices A_1^T A_1 and A_2^T A_2 from the rows' outer
// products.  Everything after that (Cholesky, P, B, H, the outer steps and SP-SCD) works on
// those dense n x n products exactly as for dense A.
#include <algorithm>

#include <cooperative_groups.h>

#include "ils_internal.h"
#include "philox.cuh"

namespace ils {
namespace {

// Structure checks of the CSR input: rowptr[0] = 0, rowptr[m] = nnz, nondecreasing, and
// 0 <= colind < n.  Every later kernel also clips its ranges, so bad input only sets err.
__global__ void csr_check_kernel(int64_t m, int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind, int32_t* __restrict__ err) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  if (tid == 0 && (rowptr[0] != 0 || rowptr[m] != nnz)) atomicExch(err, ILS_ERR_INVALID_ARG);
  for (int64_t r = tid; r < m; r += stride)
    if (rowptr[r] > rowptr[r + 1]) atomicExch(err, ILS_ERR_INVALID_ARG);
  for (int64_t e = tid; e < nnz; e += stride)
    if (colind[e] < 0 || colind[e] >= n) atomicExch(err, ILS_ERR_INVALID_ARG);
}

__global__ void csc_count_kernel(int64_t nnz, int64_t n, const int32_t* __restrict__ colind, int32_t* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = colind[e];
    if (c >= 0 && c < n) atomicAdd(&cnt[c], 1);
  }
}

__device__ __forceinline__ void row_range(const int32_t* rowptr, int64_t r, int64_t nnz, int32_t& e0, int32_t& e1) {
  e0 = max(rowptr[r], 0);
  e1 = (int32_t)((int64_t)rowptr[r + 1] < nnz ? (int64_t)rowptr[r + 1] : nnz);
}

// colptr[j] = sum_{i<j} cnt[i] (single CTA, chunks of blockDim with a shared carry).
__global__ void exclusive_scan_kernel(int64_t n, const int32_t* __restrict__ cnt, int32_t* __restrict__ colptr) {
  __shared__ int32_t buf[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t j = base + threadIdx.x;
    buf[threadIdx.x] = j < n ? cnt[j] : 0;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const int32_t v = threadIdx.x >= (unsigned)off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += v;
      __syncthreads();
    }
    if (j < n) colptr[j] = carry + buf[threadIdx.x] - (j < n ? cnt[j] : 0);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) colptr[n] = carry;
}

__global__ void csc_fill_kernel(int64_t m, int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colind, const double* __restrict__ val,
                                const int32_t* __restrict__ colptr, const int32_t* __restrict__ cnt,
                                int32_t* __restrict__ fill, int32_t* __restrict__ rowind, double* __restrict__ cval,
                                int32_t* __restrict__ err) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    int32_t e0, e1;
    row_range(rowptr, r, nnz, e0, e1);
    for (int32_t e = e0; e < e1; ++e) {
      const int32_t c = colind[e];
      if (c < 0 || c >= n) continue;
      const int32_t slot = atomicAdd(&fill[c], 1);
      if (slot >= cnt[c]) {  // an entry reached twice: rowptr ranges overlap
        atomicExch(err, ILS_ERR_INVALID_ARG);
        continue;
      }
      const int32_t pos = colptr[c] + slot;
      rowind[pos] = (int32_t)r;
      const double v = val[e];
      if (!isfinite(v)) atomicExch(err, ILS_ERR_NONFINITE);
      cval[pos] = v;
    }
  }
}

// Sort each column's (row, value) pairs by row: one CTA per column, bitonic sort in shared
// memory (columns of up to 4096 entries), then count the rows below p.
__global__ void __launch_bounds__(512) csc_sort_kernel(int64_t n, int64_t p, const int32_t* __restrict__ colptr,
                                                        int32_t* __restrict__ rowind, double* __restrict__ cval,
                                                        int32_t* __restrict__ split, int32_t* __restrict__ err) {
  __shared__ int32_t kr[4096];
  __shared__ double kv[4096];
  const int64_t j = blockIdx.x;
  const int32_t b = colptr[j], cnt = colptr[j + 1] - b;
  if (cnt > 4096) {
    if (threadIdx.x == 0) atomicExch(err, ILS_ERR_INVALID_ARG);
    return;
  }
  int size = 1;
  while (size < cnt) size <<= 1;
  for (int i = threadIdx.x; i < size; i += blockDim.x) {
    kr[i] = i < cnt ? rowind[b + i] : 0x7FFFFFFF;
    kv[i] = i < cnt ? cval[b + i] : 0.0;
  }
  __syncthreads();
  for (int k = 2; k <= size; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < size; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const bool up = (i & k) == 0;
          if ((kr[i] > kr[l]) == up) {
            const int32_t tr = kr[i];
            kr[i] = kr[l];
            kr[l] = tr;
            const double tv = kv[i];
            kv[i] = kv[l];
            kv[l] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    if (i + 1 < cnt && kr[i] == kr[i + 1]) atomicExch(err, ILS_ERR_INVALID_ARG);  // duplicate (row, column)
    rowind[b + i] = kr[i];
    cval[b + i] = kv[i];
    // the first entry at or past row p marks the end of A_1's part of the column
    const bool below = kr[i] < p;
    const bool next_not = (i + 1 == cnt) || kr[i + 1] >= p;
    if (below && next_not) split[j] = i + 1;
  }
  if (threadIdx.x == 0 && (cnt == 0 || kr[0] >= p)) split[j] = 0;
}

// Upper triangles of A_1^T A_1 (rows < p) and A_2^T A_2 (rows >= p) from each row's outer
// product (FP64 atomics; the order of the additions is not fixed).
__global__ void sparse_gram_kernel(int64_t m, int64_t n, int64_t p, int64_t nnz, const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ colind, const double* __restrict__ val,
                                   double* __restrict__ G1, double* __restrict__ G2) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double* G = r < p ? G1 : G2;
    int32_t e0, e1;
    row_range(rowptr, r, nnz, e0, e1);
    for (int32_t a = e0; a < e1; ++a) {
      const int32_t ca = colind[a];
      const double va = val[a];
      for (int32_t bb = e0; bb < e1; ++bb) {
        const int32_t cb = colind[bb];
        if (ca <= cb && ca >= 0 && cb < n) atomicAdd(&G[ca + (int64_t)cb * n], va * val[bb]);
      }
    }
  }
}

__global__ void mirror_upper_kernel(int64_t n, double* __restrict__ G) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (uint32_t)e % (uint32_t)n, j = (uint32_t)e / (uint32_t)n;
    if (i > j) G[e] = G[j + i * n];
  }
}

// out(j, c) = sum over column j of A of sign(row) a_rj b(row, c); sign = -1 for rows >= p.
template <int KR>
__global__ void __launch_bounds__(128) csc_rhs_kernel(int64_t n, int64_t p, const int32_t* __restrict__ colptr,
                                                      const int32_t* __restrict__ rowind,
                                                      const double* __restrict__ cval, const double* __restrict__ B,
                                                      int64_t ldb, double* __restrict__ out, int64_t ldo) {
  const int64_t j = blockIdx.x;
  double acc[KR];
#pragma unroll
  for (int c = 0; c < KR; ++c) acc[c] = 0.0;
  for (int32_t e = colptr[j] + threadIdx.x; e < colptr[j + 1]; e += blockDim.x) {
    const int32_t r = rowind[e];
    const double a = r < p ? cval[e] : -cval[e];
#pragma unroll
    for (int c = 0; c < KR; ++c) acc[c] = fma(a, B[r + c * ldb], acc[c]);
  }
  __shared__ double red[4][KR];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < KR; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < KR) out[j + threadIdx.x * ldo] = (red[0][threadIdx.x] + red[1][threadIdx.x]) +
                                                     (red[2][threadIdx.x] + red[3][threadIdx.x]);
}

constexpr int kChainThreads = 512;
constexpr int kChainWarps = kChainThreads / 32;

template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum, broadcast to every thread (red: kChainWarps + 1 slots).
template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum_t(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // red may still be read from the previous call
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    T t = lane < kChainWarps ? red[lane] : T(0);
    t = warp_sum_t(t);
    if (lane == 0) red[kChainWarps] = t;
  }
  __syncthreads();
  return red[kChainWarps];
}

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

template <class T>
__device__ __forceinline__ const T* values(const SparseCols& sc);
template <>
__device__ __forceinline__ const double* values<double>(const SparseCols& sc) { return sc.val; }
template <>
__device__ __forceinline__ const float* values<float>(const SparseCols& sc) { return sc.val32; }

// SP-RK-RGS inner chain (Alg. 2 steps 6-12) on the sparse columns of A_1, one CTA per
// right-hand side.  The RK step touches the rows of column j1, the RGS step those of
// column j2; w and e = w - A_1 z (length p each) live in a global slice of the chain,
// z and the running column norms in shared memory.  The inner stop test uses
// A_1 z = w - e, so ||bhat - Abar1 z|| = ||bhat - A_1^T (w - e)|| costs one pass over
// A_1's entries instead of an n x n product.
// T = double: the paper's chain (z = w = 0 at the start, x_{k+1} = z).
// T = float (a.correction): bhat holds the FP64 residual r = bbar - H x_k; the chain
// solves Abar1 d = r from d = 0 in FP32 and x_k += d in FP64, so the fixed point and the
// stopping test stay FP64.
template <class T>
__global__ void __launch_bounds__(kChainThreads) rkrgs_sparse_chain_kernel(RandArgs a, SparseCols sc) {
  const int c = blockIdx.x;
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done) || a.col_done[c]) return;
  const int n = (int)a.n;
  const int64_t p = a.p;
  const int cur = *((volatile int32_t*)&st->cur);
  double* xout = (cur ? a.X1 : a.X0) + (size_t)c * n;
  const uint32_t k = (uint32_t)(st->iters - 1);
  extern __shared__ double smem[];
  double* cum = smem;
  T* z = reinterpret_cast<T*>(smem + n);
  T* w = reinterpret_cast<T*>(a.vec_scratch) + (size_t)c * 2 * p;
  T* e = w + p;
  __shared__ T red[kChainWarps + 1];
  const double* bhat = a.bhat + (size_t)c * n;
  const T* val = values<T>(sc);
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    z[s] = T(0);
    cum[s] = a.cum[s];
  }
  for (int64_t r = threadIdx.x; r < p; r += blockDim.x) {
    w[r] = T(0);
    e[r] = T(0);
  }
  __syncthreads();
  const double target2 = a.col_target2[c];
  int64_t t = 0;
  bool stop = false;
  for (; t < a.max_inner && !stop; ++t) {
    double u0, u1;
    step_uniforms(a.seed, (uint32_t)(a.chain0 + c), k, (uint64_t)t, &u0, &u1);
    const int j1 = invcdf_pick(cum, n, u0);
    const int j2 = a.same_index ? j1 : invcdf_pick(cum, n, u1);
    // RK step on A_1^T w = bhat (step 9)
    const int32_t b1 = sc.colptr[j1], n1 = sc.split[j1];
    T part = T(0);
    for (int32_t q = threadIdx.x; q < n1; q += blockDim.x) part = fma(val[b1 + q], w[sc.rowind[b1 + q]], part);
    const T delta = (T(bhat[j1]) - block_sum(part, red)) / T(a.norms2[j1]);
    for (int32_t q = threadIdx.x; q < n1; q += blockDim.x) {
      const int32_t r = sc.rowind[b1 + q];
      const T av = val[b1 + q];
      w[r] = fma(delta, av, w[r]);
      e[r] = fma(delta, av, e[r]);
    }
    __syncthreads();  // the RGS dot reads rows the RK update may have written
    // RGS step on A_1 z = w with the updated w (step 11)
    const int32_t b2 = sc.colptr[j2], n2 = sc.split[j2];
    part = T(0);
    for (int32_t q = threadIdx.x; q < n2; q += blockDim.x) part = fma(val[b2 + q], e[sc.rowind[b2 + q]], part);
    const T eps = block_sum(part, red) / T(a.norms2[j2]);
    if (threadIdx.x == 0) z[j2] += eps;
    for (int32_t q = threadIdx.x; q < n2; q += blockDim.x) {
      const int32_t r = sc.rowind[b2 + q];
      e[r] = fma(-eps, val[b2 + q], e[r]);
    }
    __syncthreads();  // the next RK dot reads rows this update may have written
    if ((t + 1) % a.check_every == 0) {
      // ||bhat - A_1^T (w - e)||^2, one warp per column of A_1
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      T acc2 = T(0);
      for (int j = wid; j < n; j += kChainWarps) {
        const int32_t bj = sc.colptr[j], nj = sc.split[j];
        T d = T(0);
        for (int32_t q = lane; q < nj; q += 32) {
          const int32_t r = sc.rowind[bj + q];
          d = fma(val[bj + q], w[r] - e[r], d);
        }
        d = warp_sum_t(d);
        const T rv = T(bhat[j]) - d;
        acc2 = fma(rv, rv, acc2);
      }
      if ((double)block_sum(lane == 0 ? acc2 : T(0), red) <= target2) stop = true;
    }
  }
  __syncthreads();
  if (a.correction) {
    for (int s = threadIdx.x; s < n; s += blockDim.x) xout[s] += (double)z[s];
  } else {
    for (int s = threadIdx.x; s < n; s += blockDim.x) xout[s] = (double)z[s];  // x_{k+1} = z (step 13)
  }
  if (threadIdx.x == 0) a.col_inner[c] += t;
}

// ---------------------------------------------------------------------------------------
// The same chain on a thread-block cluster of CS CTAs of one warp each.
//
// Only e = w - A_1 z is stored, split by rows over the cluster's shared memory (CTA r
// owns rows [r S, (r+1) S) of A_1), with the residual s = bhat - Abar1 z split by
// entries (CTA r owns n/CS of them).  w itself is never formed: since w = e + A_1 z,
//   A_1(:,j1)^T w = A_1(:,j1)^T e + (Abar1 z)_j1 = A_1(:,j1)^T e + bhat_j1 - s_j1,
// so the RK step of Alg. 2 is delta = (s_j1 - A_1(:,j1)^T e) / ||A_1(:,j1)||^2, and the
// RGS step that follows reads e after e += delta A_1(:,j1):
//   A_1(:,j2)^T e' = A_1(:,j2)^T e + delta Abar1(j2, j1).
// Both dot products therefore come from the same e, and one exchange per step (the two
// partial dots and the owner's s_j1, through distributed shared memory and a cluster
// barrier) gives every CTA delta and eps; then e += delta A_1(:,j1), e -= eps A_1(:,j2),
// z_j2 += eps and s -= eps Abar1(:,j2) on the local rows.  In exact arithmetic these are
// the steps of Alg. 2.  The index draws do not depend on the data, so the columns of a
// step (segments, values, Abar1 entries, 1/||A_1(:,j)||^2) are fetched a step ahead.
// Every CTA adds the same numbers in the same order, so all take the same branch at
// every barrier.
// ---------------------------------------------------------------------------------------
constexpr int kMaxE = 4;  // column-segment entries per lane held in registers

// 16-byte vectors of T for the residual update: VecT<float> = float4, VecT<double> = double2.
template <class T>
struct VecT;
template <>
struct VecT<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct VecT<double> {
  using type = double2;
  static constexpr int width = 2;
};
// Vectors of Abar1(:, j2) per lane: 512 entries of the CTA's share of s in registers.
template <class T>
constexpr int kVecPerLane = 512 / (32 * VecT<T>::width);

// Columns of one step, as raw loads: nothing consumes a fetched value until the step
// that uses it, so the warp never waits on these loads while it works on another step.
template <class T>
struct StepCols {
  int32_t r1[kMaxE], r2[kMaxE];  // absolute row, or -1 past the segment
  T v1[kMaxE], v2[kMaxE];
  typename VecT<T>::type g[kVecPerLane<T>];  // Abar1(i0 + width (lane + 32 i) + 0.., j2)
};

// Per-step scalars of the next 64 steps (two blocks of 32), in shared memory.
struct PickRing {
  int32_t j1[64], j2[64], b1[64], e1[64], b2[64], e2[64];
  double inv1[64], inv2[64], c12[64];
};

struct StepPick {
  int j1, j2;
  int32_t b1, e1, b2, e2;
  double inv1, inv2, c12;
};

// Draws of steps 32 blk .. 32 blk + 31 (one per lane) and everything about them that does
// not depend on the data: this CTA's segments of both columns, 1/||A_1(:,j)||^2 and
// Abar1(j1, j2).  The warp waits for these loads once per 32 steps.
template <int CS>
__device__ __forceinline__ void draw_block(const RandArgs& a, const SparseCols& sc, const double* cum, int c,
                                           uint32_t k, int rank, int64_t blk, PickRing& ring) {
  double u0, u1;
  const int64_t t = 32 * blk + threadIdx.x;
  step_uniforms(a.seed, (uint32_t)(a.chain0 + c), k, (uint64_t)t, &u0, &u1);
  const int n = (int)a.n;
  const int j1 = invcdf_pick(cum, n, u0);
  const int j2 = a.same_index ? j1 : invcdf_pick(cum, n, u1);
  const int q = (int)(blk & 1) * 32 + threadIdx.x;
  ring.j1[q] = j1;
  ring.j2[q] = j2;
  ring.b1[q] = sc.seg[j1 * (CS + 1) + rank];
  ring.e1[q] = sc.seg[j1 * (CS + 1) + rank + 1];
  ring.b2[q] = sc.seg[j2 * (CS + 1) + rank];
  ring.e2[q] = sc.seg[j2 * (CS + 1) + rank + 1];
  ring.inv1[q] = sc.inv_norms2[j1];
  ring.inv2[q] = sc.inv_norms2[j2];
  ring.c12[q] = a.G1[(int64_t)j2 * n + j1];
}

__device__ __forceinline__ StepPick read_pick(const PickRing& ring, int64_t t) {
  const int q = (int)((t >> 5) & 1) * 32 + (int)(t & 31);
  StepPick sp;
  sp.j1 = ring.j1[q];
  sp.j2 = ring.j2[q];
  sp.b1 = ring.b1[q];
  sp.e1 = ring.e1[q];
  sp.b2 = ring.b2[q];
  sp.e2 = ring.e2[q];
  sp.inv1 = ring.inv1[q];
  sp.inv2 = ring.inv2[q];
  sp.c12 = ring.c12[q];
  return sp;
}

template <class T>
__device__ __forceinline__ void load_cols(StepCols<T>& out, const StepPick& sp, const SparseCols& sc, const T* val,
                                          int i0, int ni) {
  using V = typename VecT<T>::type;
  constexpr int W = VecT<T>::width;
  const int lane = threadIdx.x;
#pragma unroll
  for (int i = 0; i < kMaxE; ++i) {
    const int32_t q1 = sp.b1 + lane + 32 * i, q2 = sp.b2 + lane + 32 * i;
    out.r1[i] = -1;
    out.v1[i] = T(0);
    out.r2[i] = -1;
    out.v2[i] = T(0);
    if (q1 < sp.e1) {
      out.r1[i] = __ldg(sc.rowind + q1);
      out.v1[i] = __ldg(val + q1);
    }
    if (q2 < sp.e2) {
      out.r2[i] = __ldg(sc.rowind + q2);
      out.v2[i] = __ldg(val + q2);
    }
  }
  const V* gcol = reinterpret_cast<const V*>(reinterpret_cast<const T*>(sc.G1c) + (int64_t)sp.j2 * sc.ldg + i0);
#pragma unroll
  for (int i = 0; i < kVecPerLane<T>; ++i) {
    const int v = lane + 32 * i;
    if (W * v < ni) out.g[i] = __ldg(gcol + v);
  }
}

// Distributed-shared-memory exchange.  Lane r of every CTA writes this CTA's triple into
// slot `rank` of CTA r with st.async, which also counts the bytes on CTA r's mbarrier for
// that buffer; each CTA waits for its own mbarrier (CS triples), so no cluster-wide
// barrier (and no release fence) sits on the chain.  Buffers alternate by round: a peer
// can only write round R + 2 after this CTA has sent round R + 1, i.e. after it has read
// round R.  Waits are bounded by the global timer (2 s); on a timeout the chain records
// ILS_ERR_TIMEOUT and stops.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void xbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
}
__device__ __forceinline__ void xbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool xbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_addr(bar);
  uint64_t t0 = 0;
  for (uint32_t spin = 0;; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((spin & 63) == 0) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (spin == 0) t0 = t;
      else if (t - t0 > 2000000000ull) return false;
    }
  }
}
__device__ __forceinline__ void st_async_triple(uint32_t raddr, uint32_t rbar, float v0, float v1, float v2) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               ::"r"(raddr), "f"(v0), "f"(v1), "f"(v2), "f"(0.f), "r"(rbar) : "memory");
}
__device__ __forceinline__ void st_async_triple(uint32_t raddr, uint32_t rbar, double v0, double v1, double v2) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
               ::"r"(raddr), "d"(v0), "d"(v1), "r"(rbar) : "memory");
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
               ::"r"(raddr + 16u), "d"(v2), "d"(0.0), "r"(rbar) : "memory");
}

// Sum over the cluster of (v0, v1, v2), added in rank order (the same in every CTA).
// Returns false on a timed-out wait.
template <class T, int CS>
__device__ __forceinline__ bool cluster_sum3(T& v0, T& v1, T& v2, T* slots, uint64_t* xbar, int& round, int rank) {
  const int b = round & 1;
  T* buf = slots + b * 4 * CS;  // [CS][4]
  uint64_t* bar = xbar + b;
  if (threadIdx.x == 0) xbar_expect(bar, (uint32_t)(CS * 4 * sizeof(T)));
  if (threadIdx.x < CS) {
    const uint32_t r = threadIdx.x;
    st_async_triple(map_rank(smem_addr(buf + 4 * rank), r), map_rank(smem_addr(bar), r), v0, v1, v2);
  }
  const bool ok = xbar_wait(bar, (uint32_t)((round >> 1) & 1));
  T s0 = buf[0], s1 = buf[1], s2 = buf[2];
#pragma unroll
  for (int r = 1; r < CS; ++r) {
    s0 += buf[4 * r];
    s1 += buf[4 * r + 1];
    s2 += buf[4 * r + 2];
  }
  v0 = s0;
  v1 = s1;
  v2 = s2;
  ++round;
  return ok;
}

template <class T, int CS>
struct ChainCtx {
  RandArgs a;
  SparseCols sc;
  const T* val;
  const double* cum;
  T* z;
  T* res;
  T* slots;
  uint64_t* xbar;
  T* e;
  PickRing* ring;
  int c, rank, n, i0, ni;
  int32_t r0;
  uint32_t k;
  double target2;
  int round;
  int64_t next_check;
  bool stop;
};

// One inner step t of the chain with the columns in cc; fetches step t+1's into cn.
template <class T, int CS>
__device__ __forceinline__ void chain_step(ChainCtx<T, CS>& x, int64_t t, const StepCols<T>& cc, StepCols<T>& cn,
                                           cooperative_groups::cluster_group& cl) {
  using V = typename VecT<T>::type;
  constexpr int W = VecT<T>::width;
  const int lane = threadIdx.x;
  if ((t & 31) == 0 && t > 0) {  // the block after next (the next one is in place)
    __syncwarp();
    draw_block<CS>(x.a, x.sc, x.cum, x.c, x.k, x.rank, (t >> 5) + 1, *x.ring);
    __syncwarp();
  }
  load_cols<T>(cn, read_pick(*x.ring, t + 1), x.sc, x.val, x.i0, x.ni);
  const StepPick p0 = read_pick(*x.ring, t);
  T* e = x.e;
  const int32_t r0 = x.r0;
  // local parts of A_1(:,j1)^T e and A_1(:,j2)^T e, and s_j1 from its owner
  T d1 = T(0), d2 = T(0);
#pragma unroll
  for (int i = 0; i < kMaxE; ++i) {
    d1 = fma(cc.v1[i], e[max(cc.r1[i] - r0, 0)], d1);
    d2 = fma(cc.v2[i], e[max(cc.r2[i] - r0, 0)], d2);
  }
  for (int32_t q = p0.b1 + 32 * kMaxE + lane; q < p0.e1; q += 32) d1 = fma(x.val[q], e[x.sc.rowind[q] - r0], d1);
  for (int32_t q = p0.b2 + 32 * kMaxE + lane; q < p0.e2; q += 32) d2 = fma(x.val[q], e[x.sc.rowind[q] - r0], d2);
  d1 = warp_sum_t(d1);
  d2 = warp_sum_t(d2);
  const int own = p0.j1 - x.i0;
  T s1 = (own >= 0 && own < x.ni) ? x.res[own] : T(0);
  if (!cluster_sum3<T, CS>(d1, d2, s1, x.slots, x.xbar, x.round, x.rank)) {
    atomicCAS(&x.a.st->status, 0, ILS_ERR_TIMEOUT);
    x.stop = true;
    return;
  }
  // RK step on A_1^T w = bhat (step 9), RGS step on A_1 z = w (step 11)
  const T delta = (s1 - d1) * T(p0.inv1);
  const T eps = fma(delta, T(p0.c12), d2) * T(p0.inv2);
#pragma unroll
  for (int i = 0; i < kMaxE; ++i)
    if (cc.r1[i] >= 0) e[cc.r1[i] - r0] = fma(delta, cc.v1[i], e[cc.r1[i] - r0]);
  for (int32_t q = p0.b1 + 32 * kMaxE + lane; q < p0.e1; q += 32) {
    const int32_t r = x.sc.rowind[q] - r0;
    e[r] = fma(delta, x.val[q], e[r]);
  }
  __syncwarp();  // a row of both columns takes the RK update before the RGS update
#pragma unroll
  for (int i = 0; i < kMaxE; ++i)
    if (cc.r2[i] >= 0) e[cc.r2[i] - r0] = fma(-eps, cc.v2[i], e[cc.r2[i] - r0]);
  for (int32_t q = p0.b2 + 32 * kMaxE + lane; q < p0.e2; q += 32) {
    const int32_t r = x.sc.rowind[q] - r0;
    e[r] = fma(-eps, x.val[q], e[r]);
  }
  if (lane == 0) x.z[p0.j2] += eps;
  // s -= eps Abar1(:, j2) on this CTA's entries
  V* rv = reinterpret_cast<V*>(x.res);
#pragma unroll
  for (int i = 0; i < kVecPerLane<T>; ++i) {
    const int v = lane + 32 * i;
    if (W * v < x.ni) {
      V r = rv[v];
      const V g = cc.g[i];
      if constexpr (W == 4) {
        r.x = fma(-eps, g.x, r.x);
        r.y = fma(-eps, g.y, r.y);
        r.z = fma(-eps, g.z, r.z);
        r.w = fma(-eps, g.w, r.w);
      } else {
        r.x = fma(-eps, g.x, r.x);
        r.y = fma(-eps, g.y, r.y);
      }
      rv[v] = r;
    }
  }
  const T* gcol = reinterpret_cast<const T*>(x.sc.G1c) + (int64_t)p0.j2 * x.sc.ldg + x.i0;
  for (int ii = W * (lane + 32 * kVecPerLane<T>); ii < x.ni; ii += W * 32)
    for (int u = 0; u < W; ++u) x.res[ii + u] = fma(-eps, gcol[ii + u], x.res[ii + u]);
  __syncwarp();
  if (t + 1 == x.next_check) {  // inner stop test: ||s||^2 <= target2
    x.next_check += x.a.check_every;
    T acc = T(0);
    for (int i = lane; i < x.ni; i += 32) acc = fma(x.res[i], x.res[i], acc);
    acc = warp_sum_t(acc);
    T u1 = T(0), u2 = T(0);
    if (!cluster_sum3<T, CS>(acc, u1, u2, x.slots, x.xbar, x.round, x.rank)) {
      atomicCAS(&x.a.st->status, 0, ILS_ERR_TIMEOUT);
      x.stop = true;
      return;
    }
    if ((double)acc <= x.target2) x.stop = true;
  }
}

template <class T, int CS>
__global__ void __launch_bounds__(32) rkrgs_cluster_kernel(RandArgs a, SparseCols sc) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  ChainCtx<T, CS> x;
  x.a = a;
  x.sc = sc;
  x.rank = (int)cl.block_rank();
  x.c = blockIdx.x / CS;
  SolveState* st = a.st;
  // the same c for every CTA of the cluster, so the whole cluster returns or none does
  if (*((volatile int32_t*)&st->done) || a.col_done[x.c]) return;
  const int n = (int)a.n, lane = threadIdx.x;
  x.n = n;
  const int32_t S = sc.slice;
  x.r0 = x.rank * S;
  const int nres = sc.nres;  // a multiple of the vector width
  x.i0 = x.rank * nres;
  x.ni = max(0, min(nres, n - x.i0));
  const int cur = *((volatile int32_t*)&st->cur);
  x.k = (uint32_t)(st->iters - 1);
  const double* bhat = a.bhat + (size_t)x.c * n;
  x.val = values<T>(sc);
  extern __shared__ double smem[];
  double* cum = smem;                                 // n
  x.res = reinterpret_cast<T*>(cum + ((n + 1) & ~1));  // nres (16-byte aligned): s = bhat - Abar1 z
  x.slots = x.res + nres;                             // 2 x CS x 4 (16-byte aligned: st.async targets)
  x.z = x.slots + 8 * CS;                             // n
  x.e = x.z + n;                                      // S: e = w - A_1 z on rows r0 .. r0+S-1
  x.cum = cum;
  __shared__ PickRing ring;
  __shared__ __align__(8) uint64_t xbar[2];
  x.ring = &ring;
  x.xbar = xbar;
  if (lane == 0) {
    xbar_init(&xbar[0]);
    xbar_init(&xbar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int s = lane; s < n; s += 32) {
    cum[s] = a.cum[s];
    x.z[s] = T(0);
  }
  for (int i = lane; i < nres; i += 32) x.res[i] = i < x.ni ? T(bhat[x.i0 + i]) : T(0);
  for (int32_t r = lane; r < S; r += 32) x.e[r] = T(0);  // the whole slice: padding lanes read e[0]
  __syncwarp();
  draw_block<CS>(a, sc, cum, x.c, x.k, x.rank, 0, ring);
  draw_block<CS>(a, sc, cum, x.c, x.k, x.rank, 1, ring);
  __syncwarp();
  cl.sync();  // every CTA of the cluster is running and initialized before any remote store
  x.target2 = a.col_target2[x.c];
  x.round = 0;
  x.next_check = a.check_every;
  x.stop = false;
  StepCols<T> ca, cb;
  load_cols<T>(ca, read_pick(ring, 0), sc, x.val, x.i0, x.ni);
  int64_t t = 0;
  // two steps per trip so that the two column buffers swap roles without copies
  for (;;) {
    if (t >= a.max_inner || x.stop) break;
    chain_step<T, CS>(x, t, ca, cb, cl);
    ++t;
    if (t >= a.max_inner || x.stop) break;
    chain_step<T, CS>(x, t, cb, ca, cl);
    ++t;
  }
  cl.sync();  // no CTA leaves while another may still address its shared memory
  if (x.rank == 0) {
    double* xout = (cur ? a.X1 : a.X0) + (size_t)x.c * n;
    if (a.correction) {
      for (int s = lane; s < n; s += 32) xout[s] += (double)x.z[s];
    } else {
      for (int s = lane; s < n; s += 32) xout[s] = (double)x.z[s];  // x_{k+1} = z (step 13)
    }
    if (lane == 0) a.col_inner[x.c] += t;
  }
}

// G1c = Abar1 in T with leading dimension ldg (zero padding rows).
template <class T>
__global__ void pad_copy_kernel(int64_t n, int64_t ldg, const double* __restrict__ G1, T* __restrict__ G1c) {
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n * ldg;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = id / ldg, i = id - j * ldg;
    G1c[id] = i < n ? T(G1[i + j * n]) : T(0);
  }
}

// seg[j (CS+1) + r]: first entry of column j (A_1 part, rows sorted) with row >= r S;
// seg[j (CS+1) + CS] = end of the A_1 part.
__global__ void segment_kernel(int64_t n, int cs, int32_t S, const int32_t* __restrict__ colptr,
                               const int32_t* __restrict__ rowind, const int32_t* __restrict__ split,
                               int32_t* __restrict__ seg) {
  const int64_t total = n * (cs + 1);
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = id / (cs + 1);
    const int r = (int)(id - j * (cs + 1));
    const int32_t end = colptr[j] + split[j];
    int32_t lo = colptr[j], hi = end;
    const int64_t bound = (int64_t)r * S;
    while (lo < hi) {  // first entry with row >= bound (rows are sorted)
      const int32_t mid = lo + ((hi - lo) >> 1);
      if (rowind[mid] < bound) lo = mid + 1;
      else hi = mid;
    }
    seg[id] = r < cs ? lo : end;
  }
}

__global__ void narrow_kernel(int64_t count, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

int gs(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096)); }

}  // namespace

// CSR -> column-sorted CSC of all of A, split[j] = entries of column j in A_1, and the dense
// Grams G1 = A_1^T A_1, G2 = A_2^T A_2.  cnt_fill: 2n ints of scratch.  err (device int):
// NONFINITE for a non-finite value, INVALID_ARG for a column with more than 4096 entries.
cudaError_t sparse_setup(int64_t m, int64_t n, int64_t p, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                         const double* val, SparseCols sc, int32_t* cnt_fill, double* G1, double* G2, int32_t* err,
                         cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(cnt_fill, 0, sizeof(int32_t) * 2 * n, s)) != cudaSuccess) return e;
  csr_check_kernel<<<gs(std::max(m, nnz)), 256, 0, s>>>(m, n, nnz, rowptr, colind, err);
  note_launch();
  csc_count_kernel<<<gs(nnz), 256, 0, s>>>(nnz, n, colind, cnt_fill);
  note_launch();
  exclusive_scan_kernel<<<1, 1024, 0, s>>>(n, cnt_fill, sc.colptr);
  note_launch();
  csc_fill_kernel<<<gs(m), 256, 0, s>>>(m, n, nnz, rowptr, colind, val, sc.colptr, cnt_fill, cnt_fill + n, sc.rowind,
                                        sc.val, err);
  note_launch();
  csc_sort_kernel<<<(unsigned)n, 512, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, sc.split, err);
  note_launch();
  if ((e = cudaMemsetAsync(G1, 0, sizeof(double) * n * n, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(G2, 0, sizeof(double) * n * n, s)) != cudaSuccess) return e;
  sparse_gram_kernel<<<gs(m), 256, 0, s>>>(m, n, p, nnz, rowptr, colind, val, G1, G2);
  note_launch();
  mirror_upper_kernel<<<gs(n * n), 256, 0, s>>>(n, G1);
  note_launch();
  mirror_upper_kernel<<<gs(n * n), 256, 0, s>>>(n, G2);
  note_launch();
  if (sc.val32) {
    narrow_kernel<<<gs(nnz), 256, 0, s>>>(nnz, sc.val, sc.val32);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t sparse_rhs_bar(int64_t n, int64_t p, int64_t k, SparseCols sc, const double* B, int64_t ldb, double* out,
                           int64_t ldo, cudaStream_t s) {
  for (int64_t c0 = 0; c0 < k; c0 += kMaxRhsPerPass) {
    const int kk = (int)std::min<int64_t>(kMaxRhsPerPass, k - c0);
    const double* Bc = B + c0 * ldb;
    double* Oc = out + c0 * ldo;
    switch (kk) {
      case 1: csc_rhs_kernel<1><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
      case 2: csc_rhs_kernel<2><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
      case 3: csc_rhs_kernel<3><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
      case 4: csc_rhs_kernel<4><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
      case 5: csc_rhs_kernel<5><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
      case 6: csc_rhs_kernel<6><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
      case 7: csc_rhs_kernel<7><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
      default: csc_rhs_kernel<8><<<(unsigned)n, 128, 0, s>>>(n, p, sc.colptr, sc.rowind, sc.val, Bc, ldb, Oc, ldo); break;
    }
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {

int64_t cluster_nres(int64_t n, int cs, bool fp32) {
  const int64_t w = fp32 ? 4 : 2;
  return ((n + cs - 1) / cs + w - 1) / w * w;
}

size_t cluster_smem(int64_t n, int64_t p, int cs, bool fp32) {
  const size_t ts = fp32 ? sizeof(float) : sizeof(double);
  const int64_t S = (p + cs - 1) / cs;
  return sizeof(double) * (size_t)((n + 1) & ~1) + ts * (size_t)(cluster_nres(n, cs, fp32) + n + 8 * cs + S);
}

template <class T, int CS>
cudaError_t launch_cluster(const RandArgs* a, const SparseCols* sc, size_t smem, cudaStream_t s, int* max_clusters) {
  auto kern = rkrgs_cluster_kernel<T, CS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((a ? a->k : 1) * CS));
  cfg.blockDim = dim3(32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_clusters) return cudaOccupancyMaxActiveClusters(max_clusters, (void*)kern, &cfg);
  e = cudaLaunchKernelEx(&cfg, kern, *a, *sc);
  note_launch();
  return e;
}

template <class T>
cudaError_t dispatch_cluster(int cs, const RandArgs* a, const SparseCols* sc, size_t smem, cudaStream_t s,
                             int* max_clusters) {
  switch (cs) {
    case 1: return launch_cluster<T, 1>(a, sc, smem, s, max_clusters);
    case 2: return launch_cluster<T, 2>(a, sc, smem, s, max_clusters);
    case 4: return launch_cluster<T, 4>(a, sc, smem, s, max_clusters);
    case 8: return launch_cluster<T, 8>(a, sc, smem, s, max_clusters);
  }
  return cudaErrorInvalidValue;
}

__global__ void reciprocal_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = 1.0 / x[i];
}

}  // namespace

int rkrgs_cluster_plan(int64_t n, int64_t p, bool fp32, int want, double col_entries, int32_t* slice,
                       int32_t* nres) {
  for (int cs = 1; cs <= 8; cs *= 2) {
    if (want > 0 && cs != want) continue;
    const size_t smem = cluster_smem(n, p, cs, fp32);
    if (smem > 200 * 1024) continue;
    // prefer segments that the lanes' registers hold (about 3.5 entries per lane)
    if (want == 0 && cs < 8 && col_entries / cs > 3.5 * 32) continue;
    int clusters = 0;
    cudaError_t e = fp32 ? dispatch_cluster<float>(cs, nullptr, nullptr, smem, nullptr, &clusters)
                         : dispatch_cluster<double>(cs, nullptr, nullptr, smem, nullptr, &clusters);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (clusters >= 1) {
      *slice = (int32_t)((p + cs - 1) / cs);
      *nres = (int32_t)cluster_nres(n, cs, fp32);
      return cs;
    }
  }
  *slice = 0;
  *nres = 0;
  return 0;
}

cudaError_t sparse_chain_prep(int64_t n, SparseCols sc, const double* G1, const double* norms2, bool fp32,
                              cudaStream_t s) {
  reciprocal_kernel<<<gs(n), 256, 0, s>>>(n, norms2, sc.inv_norms2);
  note_launch();
  if (sc.cs > 0) {
    if (fp32) pad_copy_kernel<float><<<gs(n * sc.ldg), 256, 0, s>>>(n, sc.ldg, G1, (float*)sc.G1c);
    else pad_copy_kernel<double><<<gs(n * sc.ldg), 256, 0, s>>>(n, sc.ldg, G1, (double*)sc.G1c);
    note_launch();
    segment_kernel<<<gs(n * (sc.cs + 1)), 256, 0, s>>>(n, sc.cs, sc.slice, sc.colptr, sc.rowind, sc.split, sc.seg);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t rkrgs_sparse_chain(const RandArgs& a, SparseCols sc, bool fp32, cudaStream_t s) {
  if (sc.cs > 0) {
    const size_t smem = cluster_smem(a.n, a.p, sc.cs, fp32);
    return fp32 ? dispatch_cluster<float>(sc.cs, &a, &sc, smem, s, nullptr)
                : dispatch_cluster<double>(sc.cs, &a, &sc, smem, s, nullptr);
  }
  const size_t smem = sizeof(double) * 2 * (size_t)a.n;
  cudaError_t e;
  if (fp32) {
    e = cudaFuncSetAttribute(rkrgs_sparse_chain_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rkrgs_sparse_chain_kernel<float><<<(unsigned)a.k, kChainThreads, smem, s>>>(a, sc);
  } else {
    e = cudaFuncSetAttribute(rkrgs_sparse_chain_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rkrgs_sparse_chain_kernel<double><<<(unsigned)a.k, kChainThreads, smem, s>>>(a, sc);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
