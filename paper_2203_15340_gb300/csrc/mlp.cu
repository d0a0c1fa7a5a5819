// Learned warm start: a three-layer perceptron theta -> x0 with GELU activations,
//   z1 = W1 theta + b1, h1 = gelu(z1), z2 = W2 h1 + b2, h2 = gelu(z2), y = W3 h2 + b3,
// trained on the GPU (FP32 weights, mean-squared error on standardized targets, Adam)
// with the kernels of this file, and evaluated in BF16 (weights and activations rounded
// to BF16, FP32 accumulation) or FP32.  x0 = mu + sigma * y undoes the standardization.
// SP converges from any start (Theorem 2.1), so a poor prediction only costs iterations;
// non-finite predictions are replaced by 0 (the plain start).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "ils_internal.h"
#include "philox.cuh"

struct ils_mlp_s {
  int64_t d_in = 0, d_h = 0, d_out = 0, nparams = 0;
  int64_t cap = 0;  // rows of the activation buffers
  void* block = nullptr;
  cudaStream_t stream = nullptr;
  float* params = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* params16 = nullptr;
  float* mu = nullptr;
  float* sigma = nullptr;
  float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Y = nullptr;
  float *dY = nullptr, *dH = nullptr, *dZ = nullptr;
  double* loss_part = nullptr;
  double* h_loss = nullptr;  // pinned
  int64_t adam_t = 0;
  bool bf16_ready = false;
};

namespace ils {
namespace {

constexpr int kLossBlocks = 64;

struct Layout {
  int64_t W1, b1, W2, b2, W3, b3, total;
};

Layout layout(int64_t d_in, int64_t d_h, int64_t d_out) {
  Layout L;
  L.W1 = 0;
  L.b1 = L.W1 + d_h * d_in;
  L.W2 = L.b1 + d_h;
  L.b2 = L.W2 + d_h * d_h;
  L.W3 = L.b2 + d_h;
  L.b3 = L.W3 + d_out * d_h;
  L.total = L.b3 + d_out;
  return L;
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z) {
  const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float phi = expf(-0.5f * z * z) * 0.3989422804014327f;
  return Phi + z * phi;
}

// Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for every weight and bias of a layer, from
// Philox with counter (index, 0, 0, 0) and the caller's seed as key.
__global__ void init_params_kernel(float* p, Layout L, int64_t d_in, int64_t d_h, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t fan_in = e < L.W2 ? d_in : d_h;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)(e >> 32), 0x4d4c50u, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float u = (float)(w.x >> 8) * (1.0f / 16777216.0f);  // [0, 1)
    const float bound = rsqrtf((float)fan_in);
    p[e] = (2.0f * u - 1.0f) * bound;
  }
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n], optionally GELU), A(m,k) = A[m*a_sm + k*a_sk],
// B(k,n) = B[k*b_sk + n*b_sn]; 32 x 32 tiles, 4 outputs per thread.  RoundA rounds the A
// operand to BF16 (inference with BF16 activations).
template <typename TB, bool RoundA>
__global__ void __launch_bounds__(256)
gemm32_kernel(int64_t M, int64_t N, int64_t K, const float* __restrict__ A, int64_t a_sm, int64_t a_sk,
              const TB* __restrict__ B, int64_t b_sk, int64_t b_sn, float* __restrict__ C, int64_t ldc,
              const float* __restrict__ bias, float* __restrict__ Zout, int gelu) {
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
  const int64_t m0 = (int64_t)blockIdx.y * 32, n0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
#pragma unroll
    for (int rr = ty; rr < 32; rr += 8) {
      const int64_t mm = m0 + rr, kk = k0 + tx;
      float av = (mm < M && kk < K) ? A[mm * a_sm + kk * a_sk] : 0.f;
      if (RoundA) av = round_bf16(av);
      As[rr][tx] = av;
      const int64_t kb = k0 + rr, nn = n0 + tx;
      Bs[rr][tx] = (kb < K && nn < N) ? to_f(B[kb * b_sk + nn * b_sn]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float bv = Bs[kk][tx];
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a] = fmaf(As[ty + 8 * a][kk], bv, acc[a]);
    }
    __syncthreads();
  }
  const int64_t nn = n0 + tx;
  if (nn >= N) return;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t mm = m0 + ty + 8 * a;
    if (mm >= M) continue;
    float v = acc[a] + (bias ? bias[nn] : 0.f);
    if (Zout) Zout[mm * ldc + nn] = v;
    if (gelu) v = gelu_f(v);
    C[mm * ldc + nn] = v;
  }
}

template <typename TB, bool RoundA>
cudaError_t gemm32(int64_t M, int64_t N, int64_t K, const float* A, int64_t a_sm, int64_t a_sk, const TB* B,
                   int64_t b_sk, int64_t b_sn, float* C, int64_t ldc, const float* bias, float* Zout, int gelu,
                   cudaStream_t s) {
  const dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32));
  gemm32_kernel<TB, RoundA><<<grid, 256, 0, s>>>(M, N, K, A, a_sm, a_sk, B, b_sk, b_sn, C, ldc, bias, Zout, gelu);
  note_launch();
  return cudaGetLastError();
}

__global__ void gelu_backward_kernel(int64_t count, const float* __restrict__ dH, const float* __restrict__ Z,
                                     float* __restrict__ dZ) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dZ[e] = dH[e] * gelu_grad_f(Z[e]);
}

// db[o] = sum_b dZ[b][o]
__global__ void column_sum_kernel(int64_t rows, int64_t cols, const float* __restrict__ dZ, float* __restrict__ db) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < cols; o += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int64_t b = 0; b < rows; ++b) s += dZ[b * cols + o];
    db[o] = s;
  }
}

// dY = 2 (Y - Tn) / (rows d_out) with Tn = (T - mu) / sigma; per-block partial sums of
// (Y - Tn)^2 in FP64.  T is sample-contiguous (d_out x rows, column-major), like Y.
__global__ void mse_kernel(int64_t rows, int64_t d_out, const float* __restrict__ Y, const double* __restrict__ T,
                           const float* __restrict__ mu, const float* __restrict__ sigma, float* __restrict__ dY,
                           double* __restrict__ part) {
  const int64_t total = rows * d_out;
  const float scale = 2.0f / (float)total;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e % d_out;
    const float tn = (float)((T[e] - (double)mu[j]) / (double)sigma[j]);
    const float d = Y[e] - tn;
    dY[e] = scale * d;
    acc += (double)d * (double)d;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// One Adam step (Kingma & Ba 2015, Algorithm 1) on the flat parameter array.
__global__ void adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Mean and standard deviation of every target coordinate over `count` samples.
__global__ void target_stats_kernel(int64_t count, int64_t d_out, const double* __restrict__ T, float* __restrict__ mu,
                                    float* __restrict__ sigma) {
  const int64_t j = blockIdx.x;
  double s = 0.0, s2 = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    const double t = T[j + i * d_out];
    s += t;
    s2 += t * t;
  }
  __shared__ double r1[32], r2[32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = s;
    r2[threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += r1[w];
      b += r2[w];
    }
    const double mean = a / (double)count;
    const double var = fmax(b / (double)count - mean * mean, 0.0);
    mu[j] = (float)mean;
    sigma[j] = (float)fmax(sqrt(var), 1e-12);
  }
}

// X[j + i ldx] = mu_j + sigma_j Y[i][j] in FP64; a non-finite prediction becomes 0.
__global__ void destandardize_kernel(int64_t rows, int64_t d_out, const float* __restrict__ Y,
                                     const float* __restrict__ mu, const float* __restrict__ sigma, double* __restrict__ X,
                                     int64_t ldx) {
  const int64_t total = rows * d_out;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d_out, j = e % d_out;
    const double v = (double)mu[j] + (double)sigma[j] * (double)Y[e];
    X[j + i * ldx] = isfinite(v) ? v : 0.0;
  }
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = __float2bfloat16_rn(src[e]);
}

int gsize(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 2048)); }

#define MLP_CK(expr)                            \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return ILS_ERR_CUDA; \
  } while (0)

// Forward pass of `rows` samples (theta row-major rows x d_in) into net->Y.
template <bool BF16>
ils_status forward_rows(ils_mlp net, int64_t rows, const float* theta, cudaStream_t s) {
  const Layout L = layout(net->d_in, net->d_h, net->d_out);
  const int64_t di = net->d_in, dh = net->d_h, dout = net->d_out;
  if (BF16) {
    const __nv_bfloat16* P = net->params16;
    MLP_CK((gemm32<__nv_bfloat16, true>(rows, dh, di, theta, di, 1, P + L.W1, 1, di, net->H1, dh, net->params + L.b1,
                                        net->Z1, 1, s)));
    MLP_CK((gemm32<__nv_bfloat16, true>(rows, dh, dh, net->H1, dh, 1, P + L.W2, 1, dh, net->H2, dh, net->params + L.b2,
                                        net->Z2, 1, s)));
    MLP_CK((gemm32<__nv_bfloat16, true>(rows, dout, dh, net->H2, dh, 1, P + L.W3, 1, dh, net->Y, dout,
                                        net->params + L.b3, nullptr, 0, s)));
  } else {
    const float* P = net->params;
    MLP_CK((gemm32<float, false>(rows, dh, di, theta, di, 1, P + L.W1, 1, di, net->H1, dh, P + L.b1, net->Z1, 1, s)));
    MLP_CK((gemm32<float, false>(rows, dh, dh, net->H1, dh, 1, P + L.W2, 1, dh, net->H2, dh, P + L.b2, net->Z2, 1, s)));
    MLP_CK((gemm32<float, false>(rows, dout, dh, net->H2, dh, 1, P + L.W3, 1, dh, net->Y, dout, P + L.b3, nullptr, 0,
                                 s)));
  }
  return ILS_OK;
}

// Loss and gradient (into net->grad) of `rows` samples against targets T.
ils_status loss_grad_rows(ils_mlp net, int64_t rows, const float* theta, const double* T, cudaStream_t s) {
  const Layout L = layout(net->d_in, net->d_h, net->d_out);
  const int64_t di = net->d_in, dh = net->d_h, dout = net->d_out;
  ils_status st = forward_rows<false>(net, rows, theta, s);
  if (st != ILS_OK) return st;
  mse_kernel<<<kLossBlocks, 256, 0, s>>>(rows, dout, net->Y, T, net->mu, net->sigma, net->dY, net->loss_part);
  note_launch();
  float* g = net->grad;
  const float* P = net->params;
  // layer 3
  MLP_CK((gemm32<float, false>(dout, dh, rows, net->dY, 1, dout, net->H2, dh, 1, g + L.W3, dh, nullptr, nullptr, 0, s)));
  column_sum_kernel<<<gsize(dout), 256, 0, s>>>(rows, dout, net->dY, g + L.b3);
  note_launch();
  MLP_CK((gemm32<float, false>(rows, dh, dout, net->dY, dout, 1, P + L.W3, dh, 1, net->dH, dh, nullptr, nullptr, 0, s)));
  gelu_backward_kernel<<<gsize(rows * dh), 256, 0, s>>>(rows * dh, net->dH, net->Z2, net->dZ);
  note_launch();
  // layer 2
  MLP_CK((gemm32<float, false>(dh, dh, rows, net->dZ, 1, dh, net->H1, dh, 1, g + L.W2, dh, nullptr, nullptr, 0, s)));
  column_sum_kernel<<<gsize(dh), 256, 0, s>>>(rows, dh, net->dZ, g + L.b2);
  note_launch();
  MLP_CK((gemm32<float, false>(rows, dh, dh, net->dZ, dh, 1, P + L.W2, dh, 1, net->dH, dh, nullptr, nullptr, 0, s)));
  gelu_backward_kernel<<<gsize(rows * dh), 256, 0, s>>>(rows * dh, net->dH, net->Z1, net->dZ);
  note_launch();
  // layer 1
  MLP_CK((gemm32<float, false>(dh, di, rows, net->dZ, 1, dh, theta, di, 1, g + L.W1, di, nullptr, nullptr, 0, s)));
  column_sum_kernel<<<gsize(dh), 256, 0, s>>>(rows, dh, net->dZ, g + L.b1);
  note_launch();
  MLP_CK(cudaGetLastError());
  return ILS_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace
}  // namespace ils

using namespace ils;

extern "C" {

ils_status ils_mlp_create(ils_mlp* out, int64_t d_in, int64_t d_hidden, int64_t d_out, uint64_t seed,
                          ils_stream_t stream) {
  if (!out) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  if (d_in < 1 || d_hidden < 1 || d_out < 1 || d_in > 4096 || d_hidden > 4096 || d_out > 16384)
    return ILS_ERR_INVALID_ARG;
  ils_mlp net = new (std::nothrow) ils_mlp_s();
  if (!net) return ILS_ERR_OOM;
  net->d_in = d_in;
  net->d_h = d_hidden;
  net->d_out = d_out;
  net->stream = (cudaStream_t)stream;
  const Layout L = layout(d_in, d_hidden, d_out);
  net->nparams = L.total;
  net->cap = 1024;
  const int64_t np = L.total, cap = net->cap, wid = std::max(d_hidden, d_out);
  size_t off = 0;
  size_t o_params = off; off = align256(off + sizeof(float) * np);
  size_t o_grad = off;   off = align256(off + sizeof(float) * np);
  size_t o_m = off;      off = align256(off + sizeof(float) * np);
  size_t o_v = off;      off = align256(off + sizeof(float) * np);
  size_t o_p16 = off;    off = align256(off + sizeof(__nv_bfloat16) * np);
  size_t o_mu = off;     off = align256(off + sizeof(float) * d_out);
  size_t o_sig = off;    off = align256(off + sizeof(float) * d_out);
  size_t o_act[8];
  for (int i = 0; i < 8; ++i) {
    o_act[i] = off;
    off = align256(off + sizeof(float) * cap * wid);
  }
  size_t o_loss = off;   off = align256(off + sizeof(double) * kLossBlocks);
  if (cudaMallocAsync(&net->block, off, net->stream) != cudaSuccess ||
      cudaMallocHost((void**)&net->h_loss, sizeof(double) * kLossBlocks) != cudaSuccess) {
    cudaGetLastError();
    ils_mlp_destroy(net);
    return ILS_ERR_OOM;
  }
  char* b = static_cast<char*>(net->block);
  net->params = (float*)(b + o_params);
  net->grad = (float*)(b + o_grad);
  net->m = (float*)(b + o_m);
  net->v = (float*)(b + o_v);
  net->params16 = (__nv_bfloat16*)(b + o_p16);
  net->mu = (float*)(b + o_mu);
  net->sigma = (float*)(b + o_sig);
  float** acts[8] = {&net->Z1, &net->H1, &net->Z2, &net->H2, &net->Y, &net->dY, &net->dH, &net->dZ};
  for (int i = 0; i < 8; ++i) *acts[i] = (float*)(b + o_act[i]);
  net->loss_part = (double*)(b + o_loss);
  cudaStream_t s = net->stream;
  init_params_kernel<<<gsize(np), 256, 0, s>>>(net->params, L, d_in, d_hidden, seed);
  note_launch();
  bool ok = cudaGetLastError() == cudaSuccess && cudaMemsetAsync(net->m, 0, sizeof(float) * np, s) == cudaSuccess &&
            cudaMemsetAsync(net->v, 0, sizeof(float) * np, s) == cudaSuccess &&
            cudaMemsetAsync(net->mu, 0, sizeof(float) * d_out, s) == cudaSuccess;
  // sigma = 1: targets are used as given until training sets the standardization.
  if (ok) {
    float* h1 = nullptr;
    ok = cudaMallocHost((void**)&h1, sizeof(float) * d_out) == cudaSuccess;
    if (ok) {
      for (int64_t j = 0; j < d_out; ++j) h1[j] = 1.0f;
      ok = cudaMemcpyAsync(net->sigma, h1, sizeof(float) * d_out, cudaMemcpyHostToDevice, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
      cudaFreeHost(h1);
    }
  }
  if (!ok) {
    cudaGetLastError();
    ils_mlp_destroy(net);
    return ILS_ERR_CUDA;
  }
  *out = net;
  return ILS_OK;
}

int64_t ils_mlp_num_params(ils_mlp net) { return net ? net->nparams : -1; }

ils_status ils_mlp_get_params(ils_mlp net, float* dst, ils_stream_t stream) {
  if (!net || !dst) return ILS_ERR_INVALID_ARG;
  MLP_CK(cudaMemcpyAsync(dst, net->params, sizeof(float) * net->nparams, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return ILS_OK;
}

ils_status ils_mlp_set_params(ils_mlp net, const float* src, ils_stream_t stream) {
  if (!net || !src) return ILS_ERR_INVALID_ARG;
  MLP_CK(cudaMemcpyAsync(net->params, src, sizeof(float) * net->nparams, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  net->bf16_ready = false;
  return ILS_OK;
}

ils_status ils_mlp_loss_grad(ils_mlp net, int64_t count, const float* theta, const double* T, double* loss,
                             float* grad, ils_stream_t stream) {
  if (!net || count < 1 || count > net->cap || !theta || !T || !grad) return ILS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ils_status st = loss_grad_rows(net, count, theta, T, s);
  if (st != ILS_OK) return st;
  MLP_CK(cudaMemcpyAsync(grad, net->grad, sizeof(float) * net->nparams, cudaMemcpyDeviceToDevice, s));
  MLP_CK(cudaMemcpyAsync(net->h_loss, net->loss_part, sizeof(double) * kLossBlocks, cudaMemcpyDeviceToHost, s));
  MLP_CK(cudaStreamSynchronize(s));
  if (loss) {
    double t = 0.0;
    for (int i = 0; i < kLossBlocks; ++i) t += net->h_loss[i];
    *loss = t / (double)(count * net->d_out);
  }
  return ILS_OK;
}

ils_status ils_mlp_train(ils_mlp net, int64_t count, const float* theta, const double* T, int64_t epochs, int64_t batch,
                         double lr, double* final_loss, ils_stream_t stream) {
  if (!net || count < 1 || !theta || !T || epochs < 0 || batch < 1 || batch > net->cap || !(lr > 0.0))
    return ILS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  target_stats_kernel<<<(unsigned)net->d_out, 256, 0, s>>>(count, net->d_out, T, net->mu, net->sigma);
  note_launch();
  MLP_CK(cudaGetLastError());
  double last = 0.0;
  for (int64_t ep = 0; ep < epochs; ++ep) {
    for (int64_t i0 = 0; i0 < count; i0 += batch) {
      const int64_t rows = std::min(batch, count - i0);
      ils_status st = loss_grad_rows(net, rows, theta + i0 * net->d_in, T + i0 * net->d_out, s);
      if (st != ILS_OK) return st;
      net->adam_t += 1;
      const float c1 = 1.0f - powf(0.9f, (float)net->adam_t);
      const float c2 = 1.0f - powf(0.999f, (float)net->adam_t);
      adam_kernel<<<gsize(net->nparams), 256, 0, s>>>(net->nparams, net->params, net->grad, net->m, net->v, (float)lr,
                                                      c1, c2);
      note_launch();
      MLP_CK(cudaGetLastError());
    }
    // loss of the epoch's last minibatch (before its update)
    MLP_CK(cudaMemcpyAsync(net->h_loss, net->loss_part, sizeof(double) * kLossBlocks, cudaMemcpyDeviceToHost, s));
    MLP_CK(cudaStreamSynchronize(s));
    double t = 0.0;
    for (int i = 0; i < kLossBlocks; ++i) t += net->h_loss[i];
    const int64_t rows = count - ((count - 1) / batch) * batch;
    last = t / (double)(rows * net->d_out);
  }
  net->bf16_ready = false;
  if (final_loss) *final_loss = last;
  return ILS_OK;
}

ils_status ils_mlp_forward(ils_mlp net, int64_t count, const float* theta, double* X, int64_t ldx, int bf16,
                           ils_stream_t stream) {
  if (!net || count < 0 || (count > 0 && (!theta || !X)) || ldx < net->d_out) return ILS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (bf16 && !net->bf16_ready) {
    to_bf16_kernel<<<gsize(net->nparams), 256, 0, s>>>(net->nparams, net->params, net->params16);
    note_launch();
    MLP_CK(cudaGetLastError());
    net->bf16_ready = true;
  }
  for (int64_t i0 = 0; i0 < count; i0 += net->cap) {
    const int64_t rows = std::min(net->cap, count - i0);
    ils_status st = bf16 ? forward_rows<true>(net, rows, theta + i0 * net->d_in, s)
                         : forward_rows<false>(net, rows, theta + i0 * net->d_in, s);
    if (st != ILS_OK) return st;
    destandardize_kernel<<<gsize(rows * net->d_out), 256, 0, s>>>(rows, net->d_out, net->Y, net->mu, net->sigma,
                                                                   X + i0 * ldx, ldx);
    note_launch();
    MLP_CK(cudaGetLastError());
  }
  return ILS_OK;
}

ils_status ils_set_warmstart(ils_handle h, ils_mlp net) {
  if (!h) return ILS_ERR_INVALID_ARG;
  if (net && net->d_out != handle_n(h)) return ILS_ERR_INVALID_ARG;
  handle_set_warm_net(h, net);
  return ILS_OK;
}

ils_status ils_solve_param(ils_handle h, ils_mlp net, int64_t k, const float* theta, const double* B, int64_t ldb,
                           double* X, int64_t ldx, double tol, ils_info* info, ils_stream_t stream) {
  if (h && !net) net = handle_warm_net(h);
  if (!h || !net || k < 0) return ILS_ERR_INVALID_ARG;
  if (k == 0) return ils_solve_many(h, 0, B, ldb, X, ldx, 1, tol, info, stream);
  ils_status st = ils_mlp_forward(net, k, theta, X, ldx, 1, stream);  // x0 = net(theta), BF16 inference
  if (st != ILS_OK) return st;
  return ils_solve_many(h, k, B, ldb, X, ldx, 0, tol, info, stream);
}

void ils_mlp_destroy(ils_mlp net) {
  if (!net) return;
  if (net->block) cudaFreeAsync(net->block, net->stream);
  if (net->h_loss) cudaFreeHost(net->h_loss);
  delete net;
}

}  // extern "C"
