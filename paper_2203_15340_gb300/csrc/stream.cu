// Matrix-free A_2 products v = A_2^T (A_2 x) in one pass over A_2 (the Abar2 x of Alg. 1
// step 6 / Alg. 2 step 5 without forming Abar2).
//
// A_2 is kept as a row-major copy whose rows are padded to a multiple of 128 elements, in
// FP64, FP32 or BF16.  One warp streams one row at a time: every lane loads four
// consecutive elements per 128-wide chunk (16-byte loads for FP32), forms its part of
// u_r = A_2(r,:) x against x in shared memory, the warp reduces u_r with shuffles, and the
// same registers then accumulate v += u_r A_2(r,:).  Each element of A_2 is read from HBM
// exactly once and the next row is loaded before the current one is reduced.  Per-CTA
// partial v's are summed by a second small kernel in a fixed order (deterministic).
//
// The double-FP32 copy (prec 3) holds, for every padded row, the FP32 rounding of each entry
// and then the FP32 rounding of what it leaves (about 48 bits of the entry, the FP64 copy's
// 8 bytes): u_r and v are then carried in double-FP32 (each product split exactly by an
// FMA, sums with their rounding errors kept), on the FP32 pipe at HBM speed, where the
// FP64 stream is bound by GB300's narrow FP64 unit.
#include <cuda_bf16.h>

#include <algorithm>

#include "ils_internal.h"

namespace ils {
namespace {

constexpr int kStreamWarps = 8;

template <typename T>
struct Acc;
template <>
struct Acc<double> {
  using type = double;
};
template <>
struct Acc<float> {
  using type = float;
};
template <>
struct Acc<__nv_bfloat16> {
  using type = float;
};

// Four consecutive elements as accumulator-type values.
template <typename T, typename A>
__device__ __forceinline__ void load4(const T* p, A (&o)[4]);
template <>
__device__ __forceinline__ void load4<double, double>(const double* p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}
template <>
__device__ __forceinline__ void load4<float, float>(const float* p, float (&o)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = a.z;
  o[3] = a.w;
}
template <>
__device__ __forceinline__ void load4<__nv_bfloat16, float>(const __nv_bfloat16* p, float (&o)[4]) {
  const uint2 a = *reinterpret_cast<const uint2*>(p);
  o[0] = __uint_as_float(a.x << 16);
  o[1] = __uint_as_float(a.x & 0xFFFF0000u);
  o[2] = __uint_as_float(a.y << 16);
  o[3] = __uint_as_float(a.y & 0xFFFF0000u);
}

template <typename A>
__device__ __forceinline__ A warp_sum_a(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Where the vector comes from: a plain pointer, or column c of the current iterate buffer
// of a solve in flight (nothing to do once the solve or the column is finished).
struct XSrc {
  const double* x;
  const double* x1;
  const SolveState* st;
  const int32_t* col_done;
  int c;
};

__device__ __forceinline__ const double* resolve_x(const XSrc& src, int64_t n, bool* skip) {
  if (!src.st) {
    *skip = false;
    return src.x;
  }
  *skip = *((volatile const int32_t*)&src.st->done) || src.col_done[src.c];
  const int cur = *((volatile const int32_t*)&src.st->cur);
  return (cur ? src.x1 : src.x) + (int64_t)src.c * n;
}

// Asynchronous global -> shared copies (16 or 8 bytes per lane) that keep several rows
// in flight per warp without holding them in registers.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Lane `lane`'s four elements of every 128-wide chunk of row r: global -> its own slot bytes.
template <typename T, int NT>
__device__ __forceinline__ void issue_row(T* slot, const T* row, int lane) {
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int off = t * 128 + lane * 4;
    if (sizeof(T) == 8) {
      cp_async16(slot + off, row + off);
      cp_async16(slot + off + 2, row + off + 2);
    } else if (sizeof(T) == 4) {
      cp_async16(slot + off, row + off);
    } else {
      cp_async8(slot + off, row + off);
    }
  }
}

// NT = chunks of 128 columns per row (ldr = 128 NT >= n); R rows in flight per warp.
template <typename T, int NT, int R>
__global__ void __launch_bounds__(32 * kStreamWarps)
aq_stream_kernel(int64_t q, int64_t n, const T* __restrict__ Ar, int64_t ldr, XSrc src,
                 typename Acc<T>::type* __restrict__ part) {
  using A = typename Acc<T>::type;
  bool skip;
  const double* __restrict__ x = resolve_x(src, n, &skip);
  if (skip) return;
  extern __shared__ __align__(16) unsigned char stream_smem[];
  __shared__ A xs[128 * NT];
  __shared__ A red[128 * NT];
  for (int64_t j = threadIdx.x; j < 128 * NT; j += blockDim.x) xs[j] = j < n ? (A)x[j] : A(0);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* ring = reinterpret_cast<T*>(stream_smem) + (size_t)w * R * (128 * NT);
  A xv[NT][4];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) xv[t][e] = xs[t * 128 + lane * 4 + e];
  A vacc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) vacc[t][e] = A(0);
  const int64_t gw = (int64_t)blockIdx.x * kStreamWarps + w, nw = (int64_t)gridDim.x * kStreamWarps;
  // Prologue: rows gw, gw + nw, ..., one commit group per row (empty groups past q).
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int64_t r = gw + i * nw;
    if (r < q) issue_row<T, NT>(ring + i * (128 * NT), Ar + r * ldr, lane);
    cp_async_commit();
  }
  int slot = 0;
  for (int64_t r = gw; r < q; r += nw) {
    cp_async_wait<R - 1>();  // the oldest group, this row, has landed (each lane reads its own bytes)
    const T* srow = ring + slot * (128 * NT);
    A cur[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t) load4<T, A>(srow + t * 128 + lane * 4, cur[t]);
    A d = A(0);
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) d = fma(cur[t][e], xv[t][e], d);
    // The slot's values are in registers (consumed above): refill it with row r + R nw.
    const int64_t rn = r + (int64_t)R * nw;
    if (rn < q) issue_row<T, NT>(ring + slot * (128 * NT), Ar + rn * ldr, lane);
    cp_async_commit();
    const A u = warp_sum_a(d);
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) vacc[t][e] = fma(u, cur[t][e], vacc[t][e]);
    slot = (slot + 1 == R) ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  // Warps add their partial v into shared memory one after another (fixed order).
  for (int j = threadIdx.x; j < 128 * NT; j += blockDim.x) red[j] = A(0);
  for (int ww = 0; ww < kStreamWarps; ++ww) {
    __syncthreads();
    if (w == ww) {
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[t * 128 + lane * 4 + e] += vacc[t][e];
    }
  }
  __syncthreads();
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) part[(int64_t)blockIdx.x * n + j] = red[j];
}

// v[j] = sum over CTAs of part[b][j]: 32 columns per CTA, its 8 warps split the partials
// (4 loads in flight per thread) and add their sums in warp order (deterministic).
template <typename A>
__global__ void __launch_bounds__(256) aq_reduce_kernel(int64_t n, int blocks, const A* __restrict__ part,
                                                        double* __restrict__ v, XSrc src) {
  bool skip;
  resolve_x(src, n, &skip);
  if (skip) return;
  __shared__ A red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  A s0 = A(0), s1 = A(0), s2 = A(0), s3 = A(0);
  if (j < n) {
    int b = w;
    for (; b + 24 < blocks; b += 32) {
      s0 += part[(int64_t)b * n + j];
      s1 += part[(int64_t)(b + 8) * n + j];
      s2 += part[(int64_t)(b + 16) * n + j];
      s3 += part[(int64_t)(b + 24) * n + j];
    }
    for (; b < blocks; b += 8) s0 += part[(int64_t)b * n + j];
  }
  red[w][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (w == 0 && j < n) {
    A t = A(0);
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) t += red[ww][lane];
    v[j] = (double)t;
  }
}

template <typename T>
__global__ void rowmajor_copy_kernel(int64_t q, int64_t n, const double* __restrict__ Ac, int64_t lda, T* __restrict__ Ar,
                                     int64_t ldr) {
  // Tiles of 32 x 32 through shared memory: column-major reads, row-major writes.
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + threadIdx.x, c = c0 + k;
    tile[k][threadIdx.x] = (r < q && c < n) ? Ac[r + c * lda] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    if (r < q && c < ldr) Ar[r * ldr + c] = (T)tile[threadIdx.x][k];
  }
}

// (sh, sl) += p + e with the rounding error of sh + p kept in sl.
__device__ __forceinline__ void df_add(float& sh, float& sl, float p, float e) {
  const float t = sh + p;
  const float bp = t - sh;
  sl += ((sh - (t - bp)) + (p - bp)) + e;
  sh = t;
}
// (ah + al)(bh + bl) as p + e: p the FP32 product of the leading parts, e the rest.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& p, float& e) {
  p = ah * bh;
  e = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -p)));
}

// Double-FP32 stream: rows of 2 * 128 NT floats (leading parts, then the rest); R rows in
// flight per warp.  Partial v's (per CTA) are written in FP64.
template <int NT, int R>
__global__ void __launch_bounds__(32 * kStreamWarps)
aq_stream_df_kernel(int64_t q, int64_t n, const float* __restrict__ Ar, XSrc src, double* __restrict__ part) {
  constexpr int LDR = 128 * NT;
  bool skip;
  const double* __restrict__ x = resolve_x(src, n, &skip);
  if (skip) return;
  extern __shared__ __align__(16) unsigned char stream_smem[];
  __shared__ float xsh[LDR], xsl[LDR];
  __shared__ double red[LDR];
  for (int64_t j = threadIdx.x; j < LDR; j += blockDim.x) {
    const double xj = j < n ? x[j] : 0.0;
    const float hi = __double2float_rn(xj);
    xsh[j] = hi;
    xsl[j] = __double2float_rn(xj - (double)hi);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* ring = reinterpret_cast<float*>(stream_smem) + (size_t)w * R * (2 * LDR);
  float xh[NT][4], xl[NT][4], vh[NT][4], vl[NT][4];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      xh[t][e] = xsh[t * 128 + lane * 4 + e];
      xl[t][e] = xsl[t * 128 + lane * 4 + e];
      vh[t][e] = vl[t][e] = 0.f;
    }
  const int64_t gw = (int64_t)blockIdx.x * kStreamWarps + w, nw = (int64_t)gridDim.x * kStreamWarps;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int64_t r = gw + i * nw;
    if (r < q) {
      issue_row<float, NT>(ring + i * (2 * LDR), Ar + r * (2 * LDR), lane);
      issue_row<float, NT>(ring + i * (2 * LDR) + LDR, Ar + r * (2 * LDR) + LDR, lane);
    }
    cp_async_commit();
  }
  int slot = 0;
  for (int64_t r = gw; r < q; r += nw) {
    cp_async_wait<R - 1>();
    const float* srow = ring + slot * (2 * LDR);
    float ah[NT][4], al[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      load4<float, float>(srow + t * 128 + lane * 4, ah[t]);
      load4<float, float>(srow + LDR + t * 128 + lane * 4, al[t]);
    }
    const int64_t rn = r + (int64_t)R * nw;
    if (rn < q) {
      issue_row<float, NT>(ring + slot * (2 * LDR), Ar + rn * (2 * LDR), lane);
      issue_row<float, NT>(ring + slot * (2 * LDR) + LDR, Ar + rn * (2 * LDR) + LDR, lane);
    }
    cp_async_commit();
    // u_r = A_2(r,:) x
    float dh = 0.f, dl = 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float pp, ee;
        df_mul(ah[t][e], al[t][e], xh[t][e], xl[t][e], pp, ee);
        df_add(dh, dl, pp, ee);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, dh, o), ol = __shfl_xor_sync(0xffffffffu, dl, o);
      df_add(dh, dl, oh, ol);
    }
    const float uh0 = __shfl_sync(0xffffffffu, dh, 0), ul0 = __shfl_sync(0xffffffffu, dl, 0);
    const float uh = uh0 + ul0, ul = ul0 - (uh - uh0);  // renormalized
    // v += u_r A_2(r,:)
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float pp, ee;
        df_mul(uh, ul, ah[t][e], al[t][e], pp, ee);
        df_add(vh[t][e], vl[t][e], pp, ee);
      }
    slot = (slot + 1 == R) ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  for (int j = threadIdx.x; j < LDR; j += blockDim.x) red[j] = 0.0;
  for (int ww = 0; ww < kStreamWarps; ++ww) {
    __syncthreads();
    if (w == ww) {
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[t * 128 + lane * 4 + e] += (double)vh[t][e] + (double)vl[t][e];
    }
  }
  __syncthreads();
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) part[(int64_t)blockIdx.x * n + j] = red[j];
}

// Row-major double-FP32 copy: row r holds the FP32 roundings of A(r, :) (ldr of them, zero
// past n) and then the FP32 roundings of what they leave.
__global__ void rowmajor_copy_df_kernel(int64_t q, int64_t n, const double* __restrict__ Ac, int64_t lda,
                                        float* __restrict__ Ar, int64_t ldr) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + threadIdx.x, c = c0 + k;
    tile[k][threadIdx.x] = (r < q && c < n) ? Ac[r + c * lda] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    if (r < q && c < ldr) {
      const double a = tile[threadIdx.x][k];
      const float hi = __double2float_rn(a);
      Ar[r * 2 * ldr + c] = hi;
      Ar[r * 2 * ldr + ldr + c] = __double2float_rn(a - (double)hi);
    }
  }
}

}  // namespace

// Rows are padded to the chunk count of the kernel instantiation that streams them
// (1, 2, 4 or 8 chunks of 128), so the kernel's row stride is always 128 * NT.
static int64_t chunk_bucket(int64_t n) {
  const int64_t nt = (n + 127) / 128;
  return nt <= 1 ? 1 : nt <= 2 ? 2 : nt <= 4 ? 4 : 8 * ((nt + 7) / 8);
}

int64_t aq_row_stride(int64_t n) { return 128 * chunk_bucket(n); }

// Upper bound of the stream grid (sizes the partial-sum buffer): 4 CTAs per SM.
int aq_stream_blocks() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  }
  return 4 * sms;
}

template <typename T>
static cudaError_t copy_rows(int64_t q, int64_t n, const double* Ac, int64_t lda, T* Ar, cudaStream_t s) {
  const int64_t ldr = aq_row_stride(n);
  if (q <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((q + 31) / 32), (unsigned)((ldr + 31) / 32));
  rowmajor_copy_kernel<T><<<grid, dim3(32, 8), 0, s>>>(q, n, Ac, lda, Ar, ldr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t aq_copy_rows(int64_t q, int64_t n, const double* Ac, int64_t lda, void* Ar, int prec, cudaStream_t s) {
  if (prec == 3) {
    const int64_t ldr = aq_row_stride(n);
    if (q <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((q + 31) / 32), (unsigned)((ldr + 31) / 32));
    rowmajor_copy_df_kernel<<<grid, dim3(32, 8), 0, s>>>(q, n, Ac, lda, static_cast<float*>(Ar), ldr);
    note_launch();
    return cudaGetLastError();
  }
  if (prec == 0) return copy_rows<double>(q, n, Ac, lda, static_cast<double*>(Ar), s);
  if (prec == 1) return copy_rows<float>(q, n, Ac, lda, static_cast<float*>(Ar), s);
  return copy_rows<__nv_bfloat16>(q, n, Ac, lda, static_cast<__nv_bfloat16*>(Ar), s);
}

template <typename T, int NT>
static cudaError_t launch_stream(int64_t q, int64_t n, const T* Ar, XSrc x, void* part, double* v, cudaStream_t s) {
  using A = typename Acc<T>::type;
  constexpr int R = sizeof(T) == 8 ? 2 : 4;  // rows in flight per warp
  const size_t smem = sizeof(T) * (size_t)kStreamWarps * R * 128 * NT;
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaFuncSetAttribute(aq_stream_kernel<T, NT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return cudaErrorInvalidValue;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aq_stream_kernel<T, NT, R>, 32 * kStreamWarps, smem) !=
            cudaSuccess ||
        per_sm <= 0)
      per_sm = 1;
    per_sm = std::min(per_sm, 4);
  }
  // One wave of resident CTAs: every warp streams rows until A_2 is exhausted.
  const int blocks = (aq_stream_blocks() / 4) * per_sm;
  aq_stream_kernel<T, NT, R><<<blocks, 32 * kStreamWarps, smem, s>>>(q, n, Ar, 128 * NT, x, static_cast<A*>(part));
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  aq_reduce_kernel<A><<<(unsigned)((n + 31) / 32), 256, 0, s>>>(n, blocks, static_cast<const A*>(part), v, x);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch_stream(int64_t q, int64_t n, const T* Ar, XSrc x, void* part, double* v, cudaStream_t s) {
  const int64_t nt = chunk_bucket(n);  // equals aq_row_stride(n) / 128, the copy's row stride
  if (q <= 0 && !x.st) return cudaMemsetAsync(v, 0, sizeof(double) * n, s);
  if (q <= 0) return cudaErrorInvalidValue;
  if (nt == 1) return launch_stream<T, 1>(q, n, Ar, x, part, v, s);
  if (nt == 2) return launch_stream<T, 2>(q, n, Ar, x, part, v, s);
  if (nt == 4) return launch_stream<T, 4>(q, n, Ar, x, part, v, s);
  if (nt == 8 && sizeof(T) < 8) return launch_stream<T, 8>(q, n, Ar, x, part, v, s);
  return cudaErrorInvalidValue;  // wider rows: the explicit route handles them
}

template <int NT>
static cudaError_t launch_stream_df(int64_t q, int64_t n, const float* Ar, XSrc x, void* part, double* v,
                                   cudaStream_t s) {
  constexpr int R = 2;  // rows in flight per warp (8 bytes per entry, as FP64)
  const size_t smem = sizeof(float) * (size_t)kStreamWarps * R * 2 * 128 * NT;
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaFuncSetAttribute(aq_stream_df_kernel<NT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return cudaErrorInvalidValue;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aq_stream_df_kernel<NT, R>, 32 * kStreamWarps, smem) !=
            cudaSuccess ||
        per_sm <= 0)
      per_sm = 1;
    per_sm = std::min(per_sm, 4);
  }
  const int blocks = (aq_stream_blocks() / 4) * per_sm;
  aq_stream_df_kernel<NT, R><<<blocks, 32 * kStreamWarps, smem, s>>>(q, n, Ar, x, static_cast<double*>(part));
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  aq_reduce_kernel<double><<<(unsigned)((n + 31) / 32), 256, 0, s>>>(n, blocks, static_cast<const double*>(part), v, x);
  note_launch();
  return cudaGetLastError();
}

static cudaError_t dispatch_stream_df(int64_t q, int64_t n, const float* Ar, XSrc x, void* part, double* v,
                                      cudaStream_t s) {
  const int64_t nt = chunk_bucket(n);
  if (q <= 0 && !x.st) return cudaMemsetAsync(v, 0, sizeof(double) * n, s);
  if (q <= 0) return cudaErrorInvalidValue;
  if (nt == 1) return launch_stream_df<1>(q, n, Ar, x, part, v, s);
  if (nt == 2) return launch_stream_df<2>(q, n, Ar, x, part, v, s);
  if (nt == 4) return launch_stream_df<4>(q, n, Ar, x, part, v, s);
  return cudaErrorInvalidValue;  // wider rows: the explicit route handles them
}

template <typename... R>
static cudaError_t by_prec(int prec, int64_t q, int64_t n, const void* Ar, XSrc x, void* part, double* v,
                           cudaStream_t s) {
  if (prec == 3) return dispatch_stream_df(q, n, static_cast<const float*>(Ar), x, part, v, s);
  if (prec == 0) return dispatch_stream<double>(q, n, static_cast<const double*>(Ar), x, part, v, s);
  if (prec == 1) return dispatch_stream<float>(q, n, static_cast<const float*>(Ar), x, part, v, s);
  return dispatch_stream<__nv_bfloat16>(q, n, static_cast<const __nv_bfloat16*>(Ar), x, part, v, s);
}

// v = A_2^T (A_2 x) from the row-major copy Ar (prec 0 FP64, 1 FP32, 2 BF16, 3 double-FP32).
// part holds aq_stream_blocks() * n accumulator values (doubles for prec 0 and 3).
cudaError_t aq_product(int64_t q, int64_t n, const void* Ar, int prec, const double* x, void* part, double* v,
                       cudaStream_t s) {
  return by_prec(prec, q, n, Ar, XSrc{x, nullptr, nullptr, nullptr, 0}, part, v, s);
}

cudaError_t aq_product_iterate(int64_t q, int64_t n, const void* Ar, int prec, const double* X0, const double* X1,
                               const SolveState* st, const int32_t* col_done, int c, void* part, double* v,
                               cudaStream_t s) {
  return by_prec(prec, q, n, Ar, XSrc{X0, X1, st, col_done, c}, part, v, s);
}

}  // namespace ils
