// Sparse A in CSR: the setup products and the parts of the solve that touch A.
//
// The setup transposes A to CSC (columns of A_1 are what the RK and RGS steps of Alg. 2
// read), sorts every column by row so that A_1's entries are a prefix of each column, and
// forms the dense n x n Gram matrices A_1^T A_1 and A_2^T A_2 from the rows' outer
// products.  Everything after that (Cholesky, P, B, H, the outer steps and SP-SCD) works on
// those dense n x n products exactly as for dense A.
#include <algorithm>

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

cudaError_t rkrgs_sparse_chain(const RandArgs& a, SparseCols sc, bool fp32, cudaStream_t s) {
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
