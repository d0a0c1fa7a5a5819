// Gram product C = X^T X for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running while a CUDA graph is being
// captured on a stream that forbids allocation, plugins of host applications whose
// allocator owns all device memory, or real-time loops that must never block in the
// allocator.  For them this file provides ils_gram_noalloc: the split-K partial sums
// that the regular Gram path keeps in memory owned by an ils_handle live instead in one
// fixed array in the library's own device memory.  That array is loaded with the library
// and stays resident on every GPU that uses it until the process exits.
#include <mutex>

#include "ils_internal.h"

namespace {

// 2^21 doubles = 16 MiB of split-K partial sums, shared by every call on a device.
constexpr size_t kNoAllocScratchElems = size_t(1) << 21;
constexpr int64_t kNoAllocMaxN = 1024;  // at least two K slices of n x n partials fit
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gram_scratch[kNoAllocScratchElems];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_gram_scratch on the current device, looked up once per device.
// In host code the symbol itself is only a host-side stand-in, never a device address.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ils_status ils_gram_noalloc(int64_t K, int64_t n, const double* X, int64_t ldx, double* C, int64_t ldc,
                                       ils_stream_t stream) {
  if (n < 1 || n > kNoAllocMaxN || K < 0 || ldx < (K > 0 ? K : 1) || ldc < n || !C || (K > 0 && !X))
    return ILS_ERR_INVALID_ARG;
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return ils::record_cuda_error(e, "ils_gram_noalloc: device address of the scratch array",
                                                      __LINE__);
  // Every partial sum the reduction reads is written first by the same call, so the
  // array needs no clearing between calls.
  e = ils::gemm_tn_f64_capped(K, n, X, ldx, C, ldc, scratch, kNoAllocScratchElems, (cudaStream_t)stream);
  if (e != cudaSuccess) return ils::record_cuda_error(e, "ils_gram_noalloc: Gram launch", __LINE__);
  return ILS_OK;
}
