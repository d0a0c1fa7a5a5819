// Route choice for SP (options.route = auto): the explicit route forms Abar2 = A_2^T A_2 and
// B = P Abar2 once and then iterates on n x n operators; the matrix-free route never forms
// them and streams A_2 (its row-major copies) in every product.  The choice minimises
//   explicit:    q n^2 / R_gram + 2 n^3 / R_f32                        (Abar2 and B)
//   matrix-free: q n (8 + s) / R_copy + T_lo (a_s + q n s / BW_s) + T_64 (a_8 + q n 8 / BW_8)
// with s the bytes of the low-precision copy (0 in FP64), T_lo and T_64 the expected number
// of low-precision and FP64 streams of a solve (plus one stream per Lanczos step when the
// handle estimates kappa and rho), and the rates measured once per process on
// synthetic inputs of a fixed size (split or FP64 Gram throughput in the method's flops;
// each copy's stream timed at two sizes, giving its bandwidth and its fixed cost a per stream).  n^2-sized per-step work is common to both and left out.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "ils_internal.h"

namespace ils {
namespace {

struct Rates {
  bool ready = false;
  double gram_split = 0.0;  // flop/s of the FP64-accurate Gram (split digits), in p n^2 units
  double gram_f64 = 0.0;    // the same for the FP64 FMA Gram
  double bw[4] = {};        // bytes/s of the A_2 stream: FP64, FP32, BF16, double-FP32 copies
  double lat[4] = {};       // fixed seconds per stream (launches and the reduction)
  double copy = 0.0;        // bytes/s of building the row-major copies
};
std::mutex g_rates_mu;
Rates g_rates;

__global__ void fill_kernel(int64_t count, double* x, uint32_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)e * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    x[e] = (double)(h & 0xFFFFFF) / 16777216.0 - 0.5;
  }
}

// Measure the rates on a K x n = 16384 x 512 Gram (126 CTAs of the split kernel, as on the
// problems this chooses for) and q x 256 streams with q = 262144 and 16384 (the larger one
// beyond L2 in every precision).  About 1.3 GB of device memory, freed before returning.
cudaError_t calibrate(Rates* r) {
  const int64_t K = 16384, n_g = 512, n = 256, q = 262144;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* mem = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const GramSplitWork gw = gram_split_work(K, n_g);
  const size_t n_x = std::max<size_t>((size_t)K * n_g, (size_t)q * n);
  size_t gemm_work = gemm_tn_work_elems(K, n_g, n_g, true, nullptr);
  const size_t bytes = 8 * n_x + 8 * (size_t)n_g * n_g + 2 * gw.slice_elems + 8 * gw.partial_elems + 4 * n_g + 16 +
                       8 * std::max<size_t>(gemm_work, 1) + 8 * (size_t)q * aq_row_stride(n) +
                       8 * (size_t)aq_stream_blocks() * n + 16 * n + 4096;
  if (e == cudaSuccess) e = cudaMalloc(&mem, bytes);
  if (e != cudaSuccess) goto done;
  {
    char* p = static_cast<char*>(mem);
    auto take = [&](size_t b) {
      char* o = p;
      p += (b + 255) & ~size_t(255);
      return o;
    };
    double* X = (double*)take(8 * n_x);
    double* C = (double*)take(8 * (size_t)n_g * n_g);
    void* slices = take(2 * gw.slice_elems);
    double* partial = (double*)take(8 * gw.partial_elems);
    int* exps = (int*)take(4 * n_g);
    int32_t* err = (int32_t*)take(16);
    double* work = (double*)take(8 * std::max<size_t>(gemm_work, 1));
    void* rows = take(8 * (size_t)q * aq_row_stride(n));
    void* part = take(8 * (size_t)aq_stream_blocks() * n);
    double* v = (double*)take(8 * n);
    double* xv = (double*)take(8 * n);
    fill_kernel<<<1024, 256, 0, s>>>((int64_t)n_x, X, 12345u);
    fill_kernel<<<1, 256, 0, s>>>(n, xv, 777u);
    note_launch(2);
    float ms = 0.f;
    auto timed = [&](auto&& fn, int reps) -> double {
      fn();  // warm-up
      cudaEventRecord(e0, s);
      for (int i = 0; i < reps; ++i) fn();
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
      return (double)ms * 1e-3 / reps;
    };
    if ((e = cudaMemsetAsync(err, 0, 4, s)) != cudaSuccess) goto done;
    const double t_split = timed([&] { gram_split_tc(K, n_g, X, K, C, n_g, slices, partial, exps, err, s); }, 3);
    const double t_f64 = timed([&] { gemm_tn_f64(K, n_g, n_g, X, K, X, K, K, C, n_g, true, false, work, s); }, 1);
    double t_copy = 0.0, t_bw[4] = {};
    double t_small[4] = {};
    const int64_t q_small = 16384;
    for (int prec = 0; prec < 4; ++prec) {
      const double tc = timed([&] { aq_copy_rows(q, n, X, q, rows, prec, s); }, 1);
      t_copy = std::max(t_copy, tc / (double)(q * n * (prec == 0 || prec == 3 ? 16 : prec == 1 ? 12 : 10)));
      t_bw[prec] = timed([&] { aq_product(q, n, rows, prec, xv, part, v, s); }, 5);
      aq_copy_rows(q_small, n, X, q_small, rows, prec, s);
      t_small[prec] = timed([&] { aq_product(q_small, n, rows, prec, xv, part, v, s); }, 5);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    if (t_split <= 0.0 || t_f64 <= 0.0) {
      e = cudaErrorUnknown;
      goto done;
    }
    r->gram_split = (double)K * n_g * n_g / t_split;
    r->gram_f64 = (double)K * n_g * n_g / t_f64;
    const double elem[4] = {8.0, 4.0, 2.0, 8.0};
    for (int prec = 0; prec < 4; ++prec) {  // t = lat + bytes / bw through the two sizes
      const double b1 = (double)q * n * elem[prec], b0 = (double)q_small * n * elem[prec];
      const double dt = t_bw[prec] - t_small[prec];
      r->bw[prec] = dt > 0.0 ? (b1 - b0) / dt : 1e12;
      r->lat[prec] = std::max(0.0, t_small[prec] - b0 / r->bw[prec]);
    }
    r->copy = t_copy > 0.0 ? 1.0 / t_copy : 1e12;
    r->ready = true;
  }
done:
  if (mem) cudaFree(mem);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

}  // namespace

cudaError_t route_prefers_matrix_free(int64_t q, int64_t n, int precision, bool split_gram, int estimate_steps,
                                      bool* mf, double* model) {
  Rates r;
  {
    std::lock_guard<std::mutex> lock(g_rates_mu);
    if (!g_rates.ready) {
      const cudaError_t e = calibrate(&g_rates);
      if (e != cudaSuccess) return e;
    }
    r = g_rates;
  }
  const double s_lo = precision == ILS_FP32_REFINE ? 4.0 : (precision == ILS_BF16_REFINE ? 2.0 : 0.0);
  const int lo = precision == ILS_FP32_REFINE ? 1 : 2;
  // Expected streams per solve: mixed precision about three refinements of three sweeps plus
  // four FP64 residuals; FP64 SP about twelve iterations, each with one FP64 stream.
  const double t_lo = precision == ILS_FP64 ? 0.0 : 9.0;
  const double t_64 = precision == ILS_FP64 ? 12.0 : 4.0;
  const double gram = (precision == ILS_FP64 && !split_gram) ? r.gram_f64 : r.gram_split;
  const double f32_rate = 20e12;  // B = P Abar2 by the FP32 GEMM
  const double qd = (double)q, nd = (double)n;
  const double explicit_cost = qd * nd * nd / gram + 2.0 * nd * nd * nd / f32_rate;
  // With estimates the matrix-free route streams A_2 once per Lanczos step (the explicit
  // route's Lanczos works on n x n operators held on chip beside the setup).
  const int est_prec = precision == ILS_FP64 ? 0 : lo;
  const double est_bytes = precision == ILS_FP64 ? 8.0 : s_lo;
  const int acc = precision == ILS_FP64 ? 0 : 3;  // the residuals' copy: FP64, or double-FP32
  const double mf_cost = qd * nd * (8.0 + s_lo) / r.copy +
                         (t_lo > 0.0 ? t_lo * (r.lat[lo] + qd * nd * s_lo / r.bw[lo]) : 0.0) +
                         t_64 * (r.lat[acc] + qd * nd * 8.0 / r.bw[acc]) +
                         estimate_steps * (r.lat[est_prec] + qd * nd * est_bytes / r.bw[est_prec]);
  *mf = n <= 512 && mf_cost < explicit_cost;
  if (model) {
    model[0] = explicit_cost;
    model[1] = mf_cost;
    model[2] = r.gram_split;
    model[3] = r.gram_f64;
    model[4] = r.bw[0];
    model[5] = r.bw[1];
    model[6] = r.bw[2];
    model[7] = r.copy;
  }
  return cudaSuccess;
}

}  // namespace ils
