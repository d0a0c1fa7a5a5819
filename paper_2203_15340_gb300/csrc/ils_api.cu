// C ABI of the ILS solver: handle life cycle, setup (Alg. 1 steps 2-4) and the
// outer-iteration driver.  All device memory of a handle is one stream-ordered
// allocation carved into aligned pieces.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ils_internal.h"

using namespace ils;

struct ils_handle_s {
  int64_t m = 0, n = 0, p = 0, q = 0;
  ils_options opt{};
  cudaStream_t stream = nullptr;
  void* block = nullptr;  // the single device allocation
  size_t block_bytes = 0;
  // setup products
  double* A = nullptr;  // m x n copy, ld m
  double* G1 = nullptr; // Abar1 = A_1^T A_1
  double* G2 = nullptr; // Abar2 = A_2^T A_2
  double* L = nullptr;  // Cholesky factor of Abar1 (lower)
  double* P = nullptr;  // Abar1^{-1}
  double* Bt = nullptr; // B^T = (P Abar2)^T
  double* H = nullptr;  // Abar1 - Abar2
  double* work = nullptr;
  // per-solve workspace (one pass of up to kMaxRhsPerPass columns)
  double* bbar = nullptr;
  double* cvec = nullptr;
  double* bnorm2 = nullptr;
  double* X0 = nullptr;
  double* X1 = nullptr;
  int32_t* col_done = nullptr;
  double* col_rr = nullptr;
  int64_t* col_iters = nullptr;
  double* partials = nullptr;
  double* bhat = nullptr;        // n x kMaxRhsPerPass (randomized methods)
  double* col_target2 = nullptr; // kMaxRhsPerPass
  int64_t* col_inner = nullptr;  // kMaxRhsPerPass
  double* inv_diag = nullptr;    // 2n: reciprocal Cholesky pivots (Abar1, H)
  double* Dinv = nullptr;        // inverses of L's 32 x 32 diagonal blocks
  double* norms2 = nullptr;      // n: ||A_1(:,j)||^2
  double* inv_norms2 = nullptr;  // n: 1 / ||A_1(:,j)||^2
  double* cum = nullptr;         // n: running sum of norms2
  double* vec_scratch = nullptr; // RK-RGS w and e when they do not fit in shared memory
  bool vec_in_smem = true;
  double* alias_prob = nullptr;  // n: Vose alias table of the column law (options.sampler = 1)
  int32_t* alias_idx = nullptr;  // n
  int32_t* picks = nullptr;      // diagnostic pick record (ils_record_picks), caller's memory
  int64_t picks_cap = 0;
  unsigned long long* inner_ns = nullptr;  // device time of chain 0 (globaltimer ns)
  char* res = nullptr;                     // the pass's results gathered for one copy (kResBytes)
  float* Hh = nullptr;                     // H row-scaled in double-FP32 form (one-cluster solve)
  float* Hl = nullptr;
  int32_t* He = nullptr;
  unsigned long long* h_inner_ns = nullptr;
  // estimates (options.estimate): [0] lambda_min(H), [1] lambda_max(H), [2] rho, [3] kappa,
  // [4] 1 / kappa^2 (the tolerance scale of ILS_STOP_ERR_BOUND), [5] Lanczos steps (H),
  // [6] Lanczos steps (rho), [7] status
  double* est = nullptr;
  double* h_est = nullptr;
  float* lz_work = nullptr;      // matrix-free Lanczos vectors
  ils_mlp warm_net = nullptr;    // ils_set_warmstart (not owned)
  std::string tune_cache;        // options.tune_cache, copied at setup
  // overlapped setup with estimates: kappa(H) and rho on a fourth stream beside the inverse
  cudaStream_t s_est = nullptr;
  cudaEvent_t ev_p = nullptr, ev_estk = nullptr, ev_est = nullptr;  // P formed; kappa ready; all ready
  // mixed precision (options.precision != ILS_FP64)
  float* L32 = nullptr;
  float* P32 = nullptr;
  float* G2_32 = nullptr;
  float* Bt32 = nullptr;
  void* Bt16 = nullptr;
  float* r32 = nullptr;
  float* c32 = nullptr;
  float* d32a = nullptr;
  float* d32b = nullptr;
  // matrix-free route: row-major copies of A_2 streamed every step
  bool mf = false;
  void* Aq64r = nullptr;    // FP64 copy (residuals; plain SP products)
  void* Aq_lo = nullptr;    // FP32 or BF16 copy (mixed-precision sweeps)
  void* sp_part = nullptr;  // per-CTA partial products
  double* vbuf = nullptr;   // n x kMaxRhsPerPass
  double* d64 = nullptr;    // n x kMaxRhsPerPass
  float* t32 = nullptr;     // n x kMaxRhsPerPass
  // split tensor-core Gram (options.gram == ILS_GRAM_SPLIT)
  void* gs_slices = nullptr;
  double* gs_partial = nullptr;
  int* gs_exps = nullptr;
  int32_t* gs_err = nullptr;
  // sparse A (ils_setup_csr): column-sorted CSC copy; no dense copy of A is kept
  bool sparse = false;
  int64_t nnz = 0;
  SparseCols sc{};
  int32_t* cnt_fill = nullptr;  // 2n
  int32_t* sp_err = nullptr;
  double* stash64 = nullptr;   // 2 x 1024: the Cholesky panels' diagonal-block stash
  // Overlapped mixed setup (single handles, split Grams): A_2^T A_2 runs on a second stream
  // beside A_1^T A_1; Abar1 is inverted in FP32 on the handle's stream while a third stream
  // forms H and tests it in FP32 (a failed FP32 pivot is settled by the FP64 factorization).
  bool overlap = false;
  bool l64_valid = true;  // L holds the FP64 factor of the current Abar1 (else formed on demand)
  bool pending = false;   // a setup enqueued by ils_refactor_async whose status is not yet read
  cudaStream_t s_aux = nullptr, s_h = nullptr;  // A_2^T A_2 and A^T J b; H and its test
  cudaStream_t s_b = nullptr;                    // B = P Abar2 beside the one-cluster solve (FP32 refinement)
  cudaEvent_t ev_b = nullptr;                    // B formed there
  bool b_async = false;                          // the last setup formed B on s_b (wait for ev_b before use)
  bool b_deferred = false;                       // ... and left it to be enqueued (ensure_b)
  cudaEvent_t ev_pb = nullptr;                   // P and Abar2 in FP32 formed (the inverse's status set)
  cudaEvent_t ev_start = nullptr, ev_g2 = nullptr, ev_g1 = nullptr;
  cudaEvent_t ev_split2 = nullptr, ev_mma = nullptr;  // A_2's digits split; both Grams' products done
  cudaEvent_t ev_hs = nullptr;                        // H's double-FP32 split formed
  cudaEvent_t ev_hd = nullptr, ev_h = nullptr;  // H formed; H tested (status copied)
  cudaEvent_t ev_acopy = nullptr, ev_rhs = nullptr;  // A copied; A^T J b ready (solve after an async setup)
  void* gs_slices2 = nullptr;
  double* gs_partial2 = nullptr;
  int* gs_exps2 = nullptr;
  float* H32 = nullptr;
  float* gj = nullptr;   // exchange buffers of the explicit FP32 inverse of Abar1
  float* gj2 = nullptr;  // and of the FP32 test of H
  float* stash32 = nullptr;
  int32_t* dstatus2 = nullptr;
  SolveState* st = nullptr;
  int32_t* dstatus = nullptr;
  uint32_t* coop_sync = nullptr;  // grid-barrier words of the one-launch solve
  // pinned host mirrors
  SolveState* h_st = nullptr;
  int32_t* h_status = nullptr;
  double* h_rr = nullptr;     // kMaxRhsPerPass
  double* h_bn = nullptr;     // kMaxRhsPerPass
  int64_t* h_iters = nullptr; // kMaxRhsPerPass
  int64_t* h_inner = nullptr; // kMaxRhsPerPass
  // state of the solve pass in flight (between pass_begin and pass_end)
  SpIterArgs pa{};
  RandArgs pra{};
  MixedArgs pma{};
  int64_t pass_k = 0;
  int64_t pass_launched = 0;
  bool pass_mixed = false;
  // setup phase timing (options.timing != 0)
  cudaEvent_t ev[15] = {};  // 6, 7: around the Abar1 Gram's tensor-core kernel; 8-10: the solve; 11, 12: kappa;
                            // 13, 14: H formed (waits done, then formed)
  double t_ms[14] = {};
};

namespace ils {
static std::atomic<int64_t> g_launches{0};
void note_launch(int64_t count) { g_launches.fetch_add(count, std::memory_order_relaxed); }
int64_t handle_n(ils_handle h) { return h->n; }
ils_mlp handle_warm_net(ils_handle h) { return h->warm_net; }
void handle_set_warm_net(ils_handle h, ils_mlp net) { h->warm_net = net; }
}  // namespace ils

namespace ils {
std::mutex g_route_mu;
double g_route_model[9] = {};  // the last automatic route decision (ils_route_model)
thread_local char g_last_error[256] = "";

ils_status record_cuda_error(cudaError_t e, const char* what, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (line %d): %s", what, line, cudaGetErrorString(e));
  cudaGetLastError();
  return ILS_ERR_CUDA;
}
}  // namespace ils

namespace {

#define ILS_CK(expr)                                                     \
  do {                                                                   \
    cudaError_t e_ = (expr);                                             \
    if (e_ != cudaSuccess) return record_cuda_error(e_, #expr, __LINE__); \
  } while (0)

__global__ void init_state_kernel(SolveState* st, int64_t max_outer, int32_t* col_done, int64_t* col_inner,
                                  int k) {
  if (threadIdx.x == 0) {
    st->done = 0;
    st->cur = 0;
    st->status = 0;
    st->pad0 = 0;
    st->iters = 0;
    st->max_outer = max_outer;
    st->inner_total = 0;
    st->counter = 0u;
    st->pad1 = 0u;
  }
  if (threadIdx.x < kMaxRhsPerPass) {
    col_done[threadIdx.x] = (threadIdx.x < k) ? 0 : 1;
    col_inner[threadIdx.x] = 0;
  }
}

__global__ void transpose_kernel(int64_t n, const double* src, double* dst, int64_t ldd) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (uint32_t)e % (uint32_t)n, j = (uint32_t)e / (uint32_t)n;  // n * n < 2^31
    dst[j + i * ldd] = src[i + j * n];
  }
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

constexpr int64_t kMaxN = 16384;  // n x n FP64 products stay below 2^31 elements

struct Carver {
  char* base;
  size_t off = 0;
  bool dry;
  template <class T>
  T* take(size_t count) {
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off = align_up(off + sizeof(T) * count);
    return p;
  }
};

void carve(ils_handle h, Carver& c, size_t work_elems) {
  const size_t nn = (size_t)h->n * (size_t)h->n;
  const size_t nk = (size_t)h->n * kMaxRhsPerPass;
  h->A = c.take<double>(h->sparse ? 1 : (size_t)h->m * (size_t)h->n);
  h->G1 = c.take<double>(nn);
  h->G2 = c.take<double>(nn);
  h->L = c.take<double>(nn);
  h->P = c.take<double>(nn);
  h->Bt = c.take<double>(nn);
  h->H = c.take<double>(nn);
  h->work = c.take<double>(std::max<size_t>(work_elems, 1));
  h->bbar = c.take<double>(nk);
  h->cvec = c.take<double>(nk);
  h->bnorm2 = c.take<double>(kMaxRhsPerPass);
  h->X0 = c.take<double>(nk);
  h->X1 = c.take<double>(nk);
  h->col_done = c.take<int32_t>(kMaxRhsPerPass);
  h->col_rr = c.take<double>(kMaxRhsPerPass);
  h->col_iters = c.take<int64_t>(kMaxRhsPerPass);
  // per-CTA partial sums: of the SP step launches, or of the one-launch solve (a CTA per SM)
  h->partials = c.take<double>(std::max<size_t>((size_t)sp_iterate_blocks(h->n) * kMaxRhsPerPass, 2048));
  h->coop_sync = c.take<uint32_t>(4);
  h->bhat = c.take<double>(nk);
  h->col_target2 = c.take<double>(kMaxRhsPerPass);
  h->col_inner = c.take<int64_t>(kMaxRhsPerPass);
  h->inv_diag = c.take<double>(2 * (size_t)h->n);
  h->Dinv = c.take<double>((size_t)((h->n + 31) / 32) * 1024);
  h->norms2 = c.take<double>((size_t)h->n);
  h->inv_norms2 = c.take<double>((size_t)h->n);
  h->cum = c.take<double>((size_t)h->n);
  h->vec_in_smem = rkrgs_vec_fits(h->n, h->p);
  if (h->sparse) h->vec_in_smem = false;
  const bool need_scratch = h->opt.method == ILS_SP_RK_RGS && !h->vec_in_smem;
  h->vec_scratch = c.take<double>(need_scratch ? (size_t)kMaxRhsPerPass * 2 * (size_t)h->p : 1);
  const bool alias = h->opt.method == ILS_SP_RK_RGS && h->opt.sampler == 1;
  h->alias_prob = c.take<double>(alias ? (size_t)h->n : 1);
  h->alias_idx = c.take<int32_t>(alias ? (size_t)h->n : 1);
  h->inner_ns = c.take<unsigned long long>(1);
  h->res = c.take<char>(kResBytes);
  h->est = c.take<double>(16);
  h->lz_work = c.take<float>(h->mf && h->opt.estimate ? lz_mf_work_floats(h->n) + (size_t)h->n * h->n : 1);
  if (h->mf) {
    const size_t rows = (size_t)h->q * (size_t)aq_row_stride(h->n);
    h->Aq64r = c.take<double>(rows);
    h->Aq_lo = h->opt.precision == ILS_FP64 ? c.take<uint16_t>(1)
               : (h->opt.precision == ILS_FP32_REFINE ? (void*)c.take<float>(rows) : (void*)c.take<uint16_t>(rows));
    h->sp_part = c.take<double>((size_t)aq_stream_blocks() * (size_t)h->n);
    h->vbuf = c.take<double>(nk);
    h->d64 = c.take<double>(nk);
    h->t32 = c.take<float>(nk);
  }
  if (h->opt.precision != ILS_FP64) {
    const size_t nn = (size_t)h->n * (size_t)h->n;
    h->L32 = c.take<float>(nn);
    h->P32 = c.take<float>(nn);
    h->G2_32 = c.take<float>(nn);
    h->Bt32 = c.take<float>(nn);
    h->Bt16 = c.take<uint16_t>(h->opt.precision == ILS_BF16_REFINE ? nn : 1);
    h->r32 = c.take<float>(nk);
    h->c32 = c.take<float>(nk);
    h->d32a = c.take<float>(nk);
    h->d32b = c.take<float>(nk);
    if (h->opt.method == ILS_SP && !h->mf && !h->sparse && h->n <= kClusterSolveMaxN) {
      h->Hh = c.take<float>(nn);
      h->Hl = c.take<float>(nn);
      h->He = c.take<int32_t>((size_t)h->n);
    }
  }
  if (h->opt.gram == ILS_GRAM_SPLIT) {
    GramSplitWork w1 = gram_split_work(h->p, h->n), w2 = gram_split_work(h->q, h->n);
    h->gs_slices = c.take<uint16_t>(std::max(w1.slice_elems, w2.slice_elems));
    h->gs_partial = c.take<double>(std::max(w1.partial_elems, w2.partial_elems));
    h->gs_exps = c.take<int>((size_t)h->n);
    h->gs_err = c.take<int32_t>(1);
    if (h->overlap) {
      h->gs_slices2 = c.take<uint16_t>(w2.slice_elems);
      h->gs_partial2 = c.take<double>(w2.partial_elems);
      h->gs_exps2 = c.take<int>((size_t)h->n);
      h->H32 = c.take<float>((size_t)h->n * (size_t)h->n);
      h->stash32 = c.take<float>(2 * 1024);  // panel flags of the FP32 factorizations
      h->gj = c.take<float>(spd_inverse_scratch_floats(h->n));
      h->gj2 = c.take<float>(spd_inverse_scratch_floats(h->n));
      h->dstatus2 = c.take<int32_t>(1);
    }
  }
  if (h->sparse) {
    const size_t nnz = (size_t)std::max<int64_t>(h->nnz, 1);
    h->sc.colptr = c.take<int32_t>((size_t)h->n + 1);
    h->sc.rowind = c.take<int32_t>(nnz);
    h->sc.val = c.take<double>(nnz);
    h->sc.val32 = h->opt.precision == ILS_FP32_REFINE && h->opt.method == ILS_SP_RK_RGS ? c.take<float>(nnz) : nullptr;
    h->sc.split = c.take<int32_t>((size_t)h->n);
    const bool chain = h->opt.method == ILS_SP_RK_RGS;
    h->sc.seg = c.take<int32_t>(chain && h->sc.cs > 0 ? (size_t)h->n * (h->sc.cs + 1) : 1);
    h->sc.inv_norms2 = c.take<double>(chain ? (size_t)h->n : 1);
    h->sc.G1c = chain && h->sc.cs > 0 ? c.take<double>((size_t)h->n * h->sc.ldg) : nullptr;
    h->cnt_fill = c.take<int32_t>(2 * (size_t)h->n);
    h->sp_err = c.take<int32_t>(1);
  }
  h->st = c.take<SolveState>(1);
  h->dstatus = c.take<int32_t>(1);
  h->stash64 = c.take<double>(2 * 1024);
}

size_t setup_work_elems(int64_t m, int64_t n, int64_t p, int64_t q) {
  (void)m;
  size_t w = 0;
  w = std::max(w, gemm_tn_work_elems(p, n, n, true, nullptr));
  w = std::max(w, gemm_tn_work_elems(q, n, n, true, nullptr));
  w = std::max(w, gemm_tn_work_elems(n, n, n, false, nullptr));
  return w;
}

ils_status validate_options(const ils_options* o) {
  if (o->method < ILS_SP || o->method > ILS_SP_SCD) return ILS_ERR_INVALID_ARG;
  if (o->precision < ILS_FP64 || o->precision > ILS_BF16_REFINE) return ILS_ERR_INVALID_ARG;
  if (o->max_outer < 0 || o->max_inner < 0 || o->check_every < 0) return ILS_ERR_INVALID_ARG;
  if (o->gram != ILS_GRAM_FP64 && o->gram != ILS_GRAM_SPLIT) return ILS_ERR_INVALID_ARG;
  if (!(o->theta > 0.0)) return ILS_ERR_INVALID_ARG;
  if (!(o->theta_decay >= 0.0 && o->theta_decay <= 1.0) || !(o->theta_min >= 0.0)) return ILS_ERR_INVALID_ARG;
  if (o->stop_rule < ILS_STOP_RELRES || o->stop_rule > ILS_STOP_ERR_BOUND) return ILS_ERR_INVALID_ARG;
  if (o->alpha_mode < 0 || o->alpha_mode > 1 || o->sampler < 0 || o->sampler > 1) return ILS_ERR_INVALID_ARG;
  if (o->inner_form < 0 || o->inner_form > 1 || o->wait_limit_ns < 0) return ILS_ERR_INVALID_ARG;
  if (o->lanczos_steps < 0 || o->lanczos_steps > 256) return ILS_ERR_INVALID_ARG;
  return ILS_OK;
}

// Squared relres target of a solve's `tol` under options.stop_rule: relres <= tol (tol^2), Sec. 5's
// RR = relres^2 <= tol (tol), or kappa_est relres <= tol (tol^2, scaled on the device by
// 1 / kappa_est^2 through tol_scale_of).
double tol2_of(ils_handle h, double tol) { return h->opt.stop_rule == ILS_STOP_PAPER_RR ? tol : tol * tol; }
const double* tol_scale_of(ils_handle h) { return h->opt.stop_rule == ILS_STOP_ERR_BOUND ? h->est + 4 : nullptr; }

cudaError_t mark(ils_handle h, int i) {
  if (!h->opt.timing) return cudaSuccess;
  if (!h->ev[i]) {
    cudaError_t e = cudaEventCreate(&h->ev[i]);
    if (e != cudaSuccess) return e;
  }
  return cudaEventRecord(h->ev[i], h->stream);
}

// Timing events 6 and 7 (around the Abar1 Gram's tensor-core kernel), created on demand.
cudaEvent_t timing_event(ils_handle h, int i) {
  if (!h->opt.timing) return nullptr;
  if (!h->ev[i] && cudaEventCreate(&h->ev[i]) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return h->ev[i];
}

void collect_timings(ils_handle h) {
  for (double& t : h->t_ms) t = 0.0;
  if (!h->opt.timing) return;
  float ms = 0.f;
  // events: 0 start(copy) 1 after copy 2 after gram1 3 after gram2 4 after cholesky 5 end
  auto el = [&](int a, int b) {
    if (h->ev[a] && h->ev[b] && cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]) == cudaSuccess) return (double)ms;
    cudaGetLastError();
    return 0.0;
  };
  h->t_ms[0] = el(1, 2);
  h->t_ms[1] = el(2, 3);
  h->t_ms[2] = el(3, 4);
  h->t_ms[3] = el(4, 5);
  h->t_ms[4] = el(0, 5);
  h->t_ms[5] = el(0, 1);
  h->t_ms[6] = el(6, 7);
  h->t_ms[7] = el(5, 8);
  h->t_ms[8] = el(8, 9);
  h->t_ms[9] = el(9, 10);
  h->t_ms[10] = el(0, 11);
  h->t_ms[11] = el(11, 12);
  h->t_ms[12] = el(0, 13);
  h->t_ms[13] = el(0, 14);
}

// Lanczos estimates (options.estimate) of kappa(H) (standard Lanczos on H) and rho (Lanczos
// on Abar2 P in the P inner product), enqueued on s; either operator may be absent.  The
// results reach h_est with the same stream's work.
ils_status enqueue_estimates(ils_handle h, cudaStream_t s, const void* Hm, int h64, const void* G2m, int g64,
                             const void* Pm, int p64) {
  LanczosProblem pr[2];
  int cnt = 0;
  const int steps = h->opt.lanczos_steps > 0 ? h->opt.lanczos_steps : 24;
  double* kap_out = h->est + 8;
  double* rho_out = h->est + 12;
  if (Hm) pr[cnt++] = LanczosProblem{h->n, Hm, nullptr, h64, 0, steps, 0, kap_out};
  if (G2m && Pm) pr[cnt++] = LanczosProblem{h->n, G2m, Pm, g64, p64, steps, 0, rho_out};
  if (cnt == 0) return ILS_OK;
  ILS_CK(lanczos_extremes(cnt, pr, s));
  ILS_CK(estimates_finish(Hm ? kap_out : nullptr, (G2m && Pm) ? rho_out : nullptr, h->est, s));
  ILS_CK(cudaMemcpyAsync(h->h_est, h->est, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return ILS_OK;
}

// Matrix-free estimates: kappa(Abar1) by standard Lanczos on Abar1, rho by Lanczos on
// (A_2^T A_2) P streaming A_2 once per step, and kappa(H) <= kappa(Abar1) / (1 - rho).
ils_status enqueue_estimates_mf(ils_handle h) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  const int steps = h->opt.lanczos_steps > 0 ? h->opt.lanczos_steps : 24;
  double* kap_out = h->est + 8;
  double* rho_out = h->est + 12;
  LanczosProblem pr = {n, h->G1, nullptr, 1, 0, steps, 0, kap_out};
  ILS_CK(lanczos_extremes(1, &pr, s));
  float* w = h->lz_work;
  const float* P32 = h->P32;
  if (h->opt.precision == ILS_FP64) {  // an FP32 copy of P for the estimate
    float* pc = w + lz_mf_work_floats(n);
    ILS_CK(convert_f64_to_f32(n * n, h->P, pc, s));
    P32 = pc;
  }
  const int prec = h->opt.precision == ILS_FP64 ? 0 : (h->opt.precision == ILS_FP32_REFINE ? 1 : 2);
  const void* Ar = prec == 0 ? h->Aq64r : h->Aq_lo;
  ILS_CK(lz_mf_init(n, P32, w, s));
  for (int j = 0; j < steps; ++j) {
    ILS_CK(aq_product(h->q, n, Ar, prec, lz_mf_vector(n, w), h->sp_part, h->vbuf, s));
    ILS_CK(lz_mf_step(n, P32, h->vbuf, w, j, s));
  }
  ILS_CK(lz_mf_finish(n, w, rho_out, s));
  ILS_CK(estimates_finish(kap_out, rho_out, h->est, s, /*gram_bound=*/true));
  ILS_CK(cudaMemcpyAsync(h->h_est, h->est, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return ILS_OK;
}

// Matrix-free route after Abar1: Cholesky of Abar1, P (FP64, or FP32 for the mixed
// precisions) and the row-major copies of A_2 that every step streams.  Abar2 and H are
// never formed, so the SPD test of (1.3) reduces to Abar1's pivots; a matrix with
// rho(B) >= 1 shows up as a residual that does not decrease (NO_CONVERGENCE).
ils_status compute_setup_mf(ils_handle h) {
  cudaStream_t s = h->stream;
  const int64_t m = h->m, n = h->n, p = h->p, q = h->q;
  h->l64_valid = true;
  ILS_CK(mark(h, 3));
  ILS_CK(cudaMemcpyAsync(h->L, h->G1, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
  ILS_CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int32_t), s));
  {
    double* mats[2] = {h->L, h->L};
    double* invd[2] = {h->inv_diag, h->inv_diag};
    ILS_CK(cholesky_f64_batch(n, 1, mats, invd, h->stash64, h->dstatus, s));
  }
  ILS_CK(mark(h, 4));
  ILS_CK(cudaMemcpyAsync(h->h_status, h->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (h->opt.gram == ILS_GRAM_SPLIT)
    ILS_CK(cudaMemcpyAsync(h->h_status + 1, h->gs_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  // the FP64-accurate copy: FP64 for FP64 SP, double-FP32 for the refinement's residuals
  ILS_CK(aq_copy_rows(q, n, h->A + p, m, h->Aq64r, h->opt.precision == ILS_FP64 ? 0 : 3, s));
  if (h->opt.precision != ILS_FP64) {
    ILS_CK(aq_copy_rows(q, n, h->A + p, m, h->Aq_lo, h->opt.precision == ILS_FP32_REFINE ? 1 : 2, s));
    ILS_CK(mixed_setup(n, h->L, nullptr, h->opt.precision, h->L32, h->P32, nullptr, nullptr, nullptr,
                       reinterpret_cast<float*>(h->Dinv), s));
  } else {
    ILS_CK(set_identity_f64(n, h->P, n, s));
    ILS_CK(trsm_binv_f64(n, n, h->L, h->Dinv, h->P, n, true, true, s));
  }
  if (h->opt.estimate) {
    const ils_status es = enqueue_estimates_mf(h);
    if (es != ILS_OK) return es;
  }
  ILS_CK(mark(h, 5));
  return ILS_OK;
}

ils_status compute_products(ils_handle h);

// Sparse A: CSC copy and both Grams from the CSR input, then the dense n x n products.
ils_status compute_setup_sparse(ils_handle h, const int32_t* rowptr, const int32_t* colind, const double* val) {
  cudaStream_t s = h->stream;
  ILS_CK(mark(h, 0));
  ILS_CK(mark(h, 1));
  ILS_CK(cudaMemsetAsync(h->sp_err, 0, sizeof(int32_t), s));
  ILS_CK(cudaMemsetAsync(h->est, 0, 16 * sizeof(double), s));
  ILS_CK(sparse_setup(h->m, h->n, h->p, h->nnz, rowptr, colind, val, h->sc, h->cnt_fill, h->G1, h->G2, h->sp_err, s));
  ILS_CK(cudaMemcpyAsync(h->h_status + 2, h->sp_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ILS_CK(mark(h, 2));
  if (h->opt.method != ILS_SP) ILS_CK(column_cumsum_f64(h->n, h->G1, h->norms2, h->cum, s, h->inv_norms2));
  if (h->opt.method == ILS_SP_RK_RGS && h->opt.sampler == 1)
    ILS_CK(alias_table_f64(h->n, h->norms2, h->alias_prob, h->alias_idx, s));
  if (h->opt.method == ILS_SP_RK_RGS)
    ILS_CK(sparse_chain_prep(h->n, h->sc, h->G1, h->norms2, h->opt.precision == ILS_FP32_REFINE, s));
  ILS_CK(mark(h, 3));
  return compute_products(h);
}

// All setup products for the current contents of h->A.
ils_status compute_setup_overlap(ils_handle h, const double* src = nullptr, int64_t lda_src = 0);

ils_status compute_setup(ils_handle h) {
  if (h->overlap) return compute_setup_overlap(h);
  cudaStream_t s = h->stream;
  const int64_t m = h->m, n = h->n, p = h->p, q = h->q;
  ILS_CK(mark(h, 1));
  ILS_CK(cudaMemsetAsync(h->est, 0, 16 * sizeof(double), s));
  // Abar1 = A_1^T A_1, Abar2 = A_2^T A_2 (Alg. 1 steps 2-3; Alg. 2 step 2; Alg. 5 step 2).
  if (h->opt.gram == ILS_GRAM_SPLIT) {
    ILS_CK(cudaMemsetAsync(h->gs_err, 0, sizeof(int32_t), s));
    ILS_CK(gram_split_tc(p, n, h->A, m, h->G1, n, h->gs_slices, h->gs_partial, h->gs_exps, h->gs_err, s,
                         timing_event(h, 6), timing_event(h, 7)));
  } else {
    ILS_CK(gemm_tn_f64(p, n, n, h->A, m, h->A, m, p, h->G1, n, true, false, h->work, s));
  }
  ILS_CK(mark(h, 2));
  if (h->opt.method != ILS_SP) ILS_CK(column_cumsum_f64(n, h->G1, h->norms2, h->cum, s, h->inv_norms2));
  if (h->opt.method == ILS_SP_RK_RGS && h->opt.sampler == 1)
    ILS_CK(alias_table_f64(n, h->norms2, h->alias_prob, h->alias_idx, s));
  if (h->mf) return compute_setup_mf(h);
  if (h->opt.gram == ILS_GRAM_SPLIT) {
    ILS_CK(gram_split_tc(q, n, h->A + p, m, h->G2, n, h->gs_slices, h->gs_partial, h->gs_exps, h->gs_err, s));
  } else {
    ILS_CK(gemm_tn_f64(q, n, n, h->A + p, m, h->A + p, m, q, h->G2, n, true, false, h->work, s));
  }
  ILS_CK(mark(h, 3));
  return compute_products(h);
}

// Everything after the Grams: H = Abar1 - Abar2, the Cholesky factors of Abar1 and H,
// P and B (Alg. 1 steps 2-3).
ils_status compute_products(ils_handle h) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  h->l64_valid = true;
  ILS_CK(axpby_mat_f64(n, 1.0, h->G1, -1.0, h->G2, h->H, s));
  if (h->Hh) ILS_CK(split_rows_df(n, h->H, h->Hh, h->Hl, h->He, s));
  // Cholesky of Abar1; the explicit inverse of Alg. 1 step 2 is formed from it.
  ILS_CK(cudaMemcpyAsync(h->L, h->G1, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
  ILS_CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int32_t), s));
  // Condition (1.3): H = A^T J A must be SPD as well (Abar1 SPD alone does not give
  // rho(B) < 1).  Its Cholesky runs in the P buffer, which is overwritten below; both
  // factorizations share each panel's launches.
  ILS_CK(cudaMemcpyAsync(h->P, h->H, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
  {
    double* mats[2] = {h->L, h->P};
    double* invd[2] = {h->inv_diag, h->inv_diag + n};
    ILS_CK(cholesky_f64_batch(n, 2, mats, invd, h->stash64, h->dstatus, s));
  }
  ILS_CK(mark(h, 4));
  ILS_CK(cudaMemcpyAsync(h->h_status, h->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (h->opt.gram == ILS_GRAM_SPLIT)
    ILS_CK(cudaMemcpyAsync(h->h_status + 1, h->gs_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  // P and B are formed without waiting for the pivot status; setup_finish reports it
  // (products of a rejected matrix are never used).  The randomized methods never apply
  // P or B (Alg. 2 and 5 use Abar1, Abar2 and H only), so they skip both.
  if (h->opt.method != ILS_SP) {
  } else if (h->opt.precision != ILS_FP64) {
    // Mixed precision: P and B for the correction sweeps in FP32 (B also in BF16).
    ILS_CK(mixed_setup(n, h->L, h->G2, h->opt.precision, h->L32, h->P32, h->G2_32, h->Bt32, h->Bt16,
                       reinterpret_cast<float*>(h->Dinv), s));
  } else {
    // P = L^{-T} L^{-1} (Alg. 1 step 2), B^T = (P Abar2)^T = Abar2 P (Alg. 1 step 3).
    ILS_CK(set_identity_f64(n, h->P, n, s));
    ILS_CK(trsm_binv_f64(n, n, h->L, h->Dinv, h->P, n, true, true, s));
    ILS_CK(gemm_tn_f64(n, n, n, h->G2, n, h->P, n, n, h->Bt, n, false, false, h->work, s));
  }
  if (h->opt.estimate) {
    ils_status es;
    if (h->opt.method != ILS_SP || h->opt.estimate == 2) es = enqueue_estimates(h, s, h->H, 1, nullptr, 0, nullptr, 0);
    else if (h->opt.precision != ILS_FP64) es = enqueue_estimates(h, s, h->H, 1, h->G2_32, 0, h->P32, 0);
    else es = enqueue_estimates(h, s, h->H, 1, h->G2, 1, h->P, 1);
    if (es != ILS_OK) return es;
  }
  ILS_CK(mark(h, 5));
  return ILS_OK;
}

// Mixed precision with split Grams on one handle: the second stream computes Abar2 while
// the handle's stream computes Abar1.  The handle's stream then forms P = Abar1^{-1}
// (Alg. 1 step 2) by block Gauss-Jordan elimination, while a third stream, once both Grams
// are done, forms H = Abar1 - Abar2 and tests it for condition (1.3) the same way; B
// follows P.  Both eliminations run in FP32: the correction sweeps only need P to FP32
// accuracy (the FP64 residuals of the refinement supply the rest).  A pivot that fails in
// FP32 sends setup_finish to the FP64 factorization of that matrix, which then decides.
// Where the inverse's tiles do not fit one cooperative wave, both matrices are factored by
// Cholesky in FP32 on the handle's stream instead and P is formed from the factor.
//
// With src, the new A is read from the caller's buffer (leading dimension lda_src) and the
// digit splits write the handle's copy of it on the way (no separate copy pass); ev_acopy
// is recorded on the handle's stream once A_1's rows are copied (A_2's are copied on the
// second stream before its Gram).
ils_status compute_setup_overlap(ils_handle h, const double* src, int64_t lda_src) {
  cudaStream_t s = h->stream, a = h->s_aux;
  const int64_t m = h->m, n = h->n, p = h->p, q = h->q;
  const bool copy = src != nullptr;
  if (!copy) {
    src = h->A;
    lda_src = m;
  }
  // The previous setup's test of H may still run on the third stream: it reads G1, G2 and H32
  // (and its estimates on the fourth: H32, G2_32 and P32).
  ILS_CK(cudaStreamWaitEvent(s, h->ev_h, 0));
  if (h->ev_est) ILS_CK(cudaStreamWaitEvent(s, h->ev_est, 0));
  // the previous B still reads P32 and Abar2 (a deferred one was never enqueued: dropped)
  if (h->b_async && !h->b_deferred) ILS_CK(cudaStreamWaitEvent(s, h->ev_b, 0));
  h->b_async = false;
  h->b_deferred = false;
  ILS_CK(cudaMemsetAsync(h->est, 0, 16 * sizeof(double), s));
  ILS_CK(mark(h, 1));
  h->h_status[0] = 0;
  h->l64_valid = false;
  ILS_CK(cudaMemsetAsync(h->gs_err, 0, sizeof(int32_t), s));
  ILS_CK(cudaMemsetAsync(h->dstatus2, 0, sizeof(int32_t), s));
  ILS_CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int32_t), s));
  ILS_CK(cudaEventRecord(h->ev_start, s));
  ILS_CK(cudaStreamWaitEvent(a, h->ev_start, 0));
  // Abar1 = A_1^T A_1 here, Abar2 = A_2^T A_2 there (Alg. 1 steps 2-3).  Abar1 is enqueued
  // first: the inverse waits for it alone.
  ILS_CK(gram_split_tc(p, n, src, lda_src, h->G1, n, h->gs_slices, h->gs_partial, h->gs_exps, h->gs_err, s,
                       timing_event(h, 6), timing_event(h, 7), copy ? h->A : nullptr, m,
                       copy ? h->ev_acopy : nullptr));
  ILS_CK(gram_split_tc(q, n, src + p, lda_src, h->G2, n, h->gs_slices2, h->gs_partial2, h->gs_exps2, h->gs_err, a,
                       nullptr, nullptr, copy ? h->A + p : nullptr, m));
  ILS_CK(convert_f64_to_f32(n * n, h->G2, h->G2_32, a));  // Abar2 in FP32, for B
  ILS_CK(cudaEventRecord(h->ev_g2, a));
  ILS_CK(cudaEventRecord(h->ev_g1, s));
  ILS_CK(mark(h, 2));
  ILS_CK(convert_f64_to_f32(n * n, h->G1, h->L32, s));  // Abar1, both triangles
  ILS_CK(mark(h, 3));
  // P = Abar1^{-1} right after the Abar1 Gram; H = Abar1 - Abar2 is formed and tested on
  // the third stream once both Grams are done (the second stream stays free for A^T J b).
  const float* mat1[2] = {h->L32, nullptr};
  float* out1[2] = {h->P32, nullptr};
  int32_t* st1[2] = {h->dstatus, nullptr};
  const cudaError_t gj = spd_inverse_f32(n, 1, mat1, out1, h->gj, st1, s);
  const bool inverted = gj == cudaSuccess;
  if (inverted) {
    cudaStream_t t = h->s_h;
    ILS_CK(cudaStreamWaitEvent(t, h->ev_g1, 0));
    ILS_CK(cudaStreamWaitEvent(t, h->ev_g2, 0));
    if (timing_event(h, 13)) ILS_CK(cudaEventRecord(h->ev[13], t));
    ILS_CK(diff_mat_f64_f32(n, h->G1, h->G2, h->H, h->H32, t));  // H = Abar1 - Abar2, and in FP32
    ILS_CK(cudaEventRecord(h->ev_hd, t));
    if (timing_event(h, 14)) ILS_CK(cudaEventRecord(h->ev[14], t));
    if (h->Hh) ILS_CK(split_rows_df(n, h->H, h->Hh, h->Hl, h->He, t));  // for the one-cluster solve
    ILS_CK(cudaEventRecord(h->ev_hs, t));
    // The SPD test of H runs on beside the rest of the setup and the next solve; its status
    // is read by setup_check, which synchronizes this stream first.
    const float* mat2[2] = {h->H32, nullptr};
    float* out2[2] = {nullptr, nullptr};
    int32_t* st2[2] = {h->dstatus2, nullptr};
    ILS_CK(spd_inverse_f32(n, 1, mat2, out2, h->gj2, st2, t, /*wide_first=*/true));
    ILS_CK(cudaMemcpyAsync(h->h_status + 3, h->dstatus2, sizeof(int32_t), cudaMemcpyDeviceToHost, t));
    ILS_CK(cudaEventRecord(h->ev_h, t));
    if (h->opt.estimate) {
      // kappa(H) once H is formed, beside the inverse; rho once P is formed.
      cudaStream_t e = h->s_est;
      const int steps = h->opt.lanczos_steps > 0 ? h->opt.lanczos_steps : 24;
      ILS_CK(cudaEventRecord(h->ev_p, s));
      ILS_CK(cudaStreamWaitEvent(e, h->ev_hd, 0));
      if (timing_event(h, 11)) ILS_CK(cudaEventRecord(h->ev[11], e));
      LanczosProblem pk = {n, h->H32, nullptr, 0, 0, steps, 0, h->est + 8};
      ILS_CK(lanczos_extremes(1, &pk, e));
      ILS_CK(estimates_finish(h->est + 8, nullptr, h->est, e));
      ILS_CK(cudaEventRecord(h->ev_estk, e));
      if (timing_event(h, 12)) ILS_CK(cudaEventRecord(h->ev[12], e));
      if (h->opt.estimate != 2) {  // rho as well
        ILS_CK(cudaStreamWaitEvent(e, h->ev_p, 0));
        LanczosProblem pr = {n, h->G2_32, h->P32, 0, 0, steps, 0, h->est + 12};
        ILS_CK(lanczos_extremes(1, &pr, e));
        ILS_CK(estimates_finish(nullptr, h->est + 12, h->est, e));
      }
      ILS_CK(cudaMemcpyAsync(h->h_est, h->est, 8 * sizeof(double), cudaMemcpyDeviceToHost, e));
      ILS_CK(cudaEventRecord(h->ev_est, e));
    }
  } else {
    if (gj != cudaErrorNotSupported) ILS_CK(gj);
    cudaGetLastError();
    ILS_CK(cudaStreamWaitEvent(s, h->ev_g2, 0));
    ILS_CK(diff_mat_f64_f32(n, h->G1, h->G2, h->H, h->H32, s));
    if (h->Hh) ILS_CK(split_rows_df(n, h->H, h->Hh, h->Hl, h->He, s));
    ILS_CK(lower_to_f32(n, h->G1, h->L32, s));
    ILS_CK(cholesky_f32_pair(n, h->L32, h->H32, reinterpret_cast<float*>(h->inv_diag),
                             reinterpret_cast<float*>(h->inv_diag + n), h->stash32, h->dstatus, h->dstatus2, s));
  }
  ILS_CK(mark(h, 4));
  ILS_CK(cudaStreamWaitEvent(s, h->ev_g2, 0));
  if (inverted) ILS_CK(cudaEventRecord(h->ev_pb, s));  // P and Abar2 in FP32 are formed
  if (inverted && h->Hh && h->opt.precision == ILS_FP32_REFINE) {
    // The one-cluster FP32 refinement sweeps with P and Abar2 (B d + c = P (Abar2 d + r)) and
    // never reads B: B is left to ensure_b, which the solve calls once its own kernels are
    // enqueued (so that B's CTAs never hold the SMs the solve's cluster waits for), and every
    // path that reads B before it.
    h->b_async = true;
    h->b_deferred = true;
  } else if (inverted)
    ILS_CK(mixed_setup_b(n, nullptr, h->opt.precision, h->P32, h->G2_32, h->Bt32, h->Bt16, s));
  else
    ILS_CK(mixed_setup(n, nullptr, h->G2, h->opt.precision, h->L32, h->P32, h->G2_32, h->Bt32, h->Bt16,
                       reinterpret_cast<float*>(h->Dinv), s));
  if (inverted) {
    ILS_CK(cudaStreamWaitEvent(s, h->ev_hs, 0));  // the solve's residuals read H (and its split)
  } else {
    ILS_CK(cudaMemcpyAsync(h->h_status + 3, h->dstatus2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (h->opt.estimate) {
      const ils_status es = h->opt.estimate == 2 ? enqueue_estimates(h, s, h->H, 1, nullptr, 0, nullptr, 0)
                                                 : enqueue_estimates(h, s, h->H, 1, h->G2_32, 0, h->P32, 0);
      if (es != ILS_OK) return es;
      ILS_CK(cudaEventRecord(h->ev_estk, s));
      ILS_CK(cudaEventRecord(h->ev_est, s));
    }
  }
  // The inverse's and the Grams' status words: read by setup_check, which synchronizes the
  // stream of H's test first, so their copies ride there, off the solve's stream.
  cudaStream_t st_copy = inverted ? h->s_h : s;
  if (inverted) ILS_CK(cudaStreamWaitEvent(st_copy, h->ev_pb, 0));
  ILS_CK(cudaMemcpyAsync(h->h_status + 6, h->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, st_copy));
  ILS_CK(cudaMemcpyAsync(h->h_status + 1, h->gs_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st_copy));
  ILS_CK(mark(h, 5));
  return ILS_OK;
}

// B = P Abar2 (FP32, and its BF16 copy) of a setup that deferred it: enqueued on s_b behind
// everything now on the handle's stream (and behind P and Abar2), marked by ev_b.
cudaError_t ensure_b(ils_handle h) {
  if (!h->b_deferred) return cudaSuccess;
  h->b_deferred = false;
  cudaError_t e = cudaEventRecord(h->ev_b, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_b, h->ev_b, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_b, h->ev_pb, 0);
  if (e == cudaSuccess)
    e = mixed_setup_b(h->n, nullptr, h->opt.precision, h->P32, h->G2_32, h->Bt32, h->Bt16, h->s_b);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_b, h->s_b);
  return e;
}

// BReady callback of the fused solve: B's event, its formation enqueued first if deferred.
cudaError_t b_ready_event(void* ctx, cudaEvent_t* ev) {
  ils_handle h = static_cast<ils_handle>(ctx);
  const cudaError_t e = ensure_b(h);
  *ev = h->b_async ? h->ev_b : nullptr;
  return e;
}

// FP64 Cholesky of Abar1 into L (status in h_status[0]), for handles whose setup factored
// it in FP32 only.  Synchronizes the handle's stream.
ils_status factor_f64_now(ils_handle h) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  ILS_CK(cudaMemcpyAsync(h->L, h->G1, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
  ILS_CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int32_t), s));
  double* mats[2] = {h->L, h->L};
  double* invd[2] = {h->inv_diag, h->inv_diag};
  ILS_CK(cholesky_f64_batch(n, 1, mats, invd, h->stash64, h->dstatus, s));
  ILS_CK(cudaMemcpyAsync(h->h_status, h->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ILS_CK(cudaStreamSynchronize(s));
  h->l64_valid = true;
  return ILS_OK;
}

// The status of the setup enqueued by compute_setup, once its stream has been synchronized;
// runs the FP64 factorizations that settle failed FP32 tests (*redone: P and B were formed
// again from the FP64 factor).
ils_status setup_check(ils_handle h, bool* redone) {
  if (redone) *redone = false;
  if (h->overlap && h->s_h) ILS_CK(cudaStreamSynchronize(h->s_h));  // the test of H
  if (h->s_est) ILS_CK(cudaStreamSynchronize(h->s_est));             // the estimates
  if (h->mf && h->opt.estimate && h->h_est[7] != 0.0) return (ils_status)(int)h->h_est[7];  // rho >= 1
  if (h->sparse && h->h_status[2] != 0) return (ils_status)h->h_status[2];
  h->h_status[1] = h->opt.gram == ILS_GRAM_SPLIT ? h->h_status[1] : 0;
  if (h->h_status[1] != 0) return h->h_status[1] == 2 ? ILS_ERR_NONFINITE : ILS_ERR_TIMEOUT;
  if (h->overlap && h->h_status[6] != 0) {
    // An FP32 pivot of Abar1 failed: the FP64 factorization decides, and the FP32
    // products are formed again from it.
    const ils_status fs = factor_f64_now(h);
    if (fs != ILS_OK) return fs;
    if (*h->h_status != 0) return (ils_status)*h->h_status;
    // B from the FP32 inverse is done (a deferred one was never enqueued)
    if (h->b_async && !h->b_deferred) ILS_CK(cudaStreamWaitEvent(h->stream, h->ev_b, 0));
    h->b_async = false;  // P and B are formed again here, on the handle's stream
    h->b_deferred = false;
    ILS_CK(mixed_setup(h->n, h->L, h->G2, h->opt.precision, h->L32, h->P32, h->G2_32, h->Bt32, h->Bt16,
                       reinterpret_cast<float*>(h->Dinv), h->stream));
    if (redone) *redone = true;
  }
  if (*h->h_status != 0) return (ils_status)*h->h_status;
  if (h->overlap && h->h_status[3] != 0) {
    // The FP32 test of H failed: the FP64 factorization decides (in the P buffer).
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    ILS_CK(cudaMemcpyAsync(h->P, h->H, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
    ILS_CK(cudaMemsetAsync(h->dstatus2, 0, sizeof(int32_t), s));
    double* mats[2] = {h->P, h->P};
    double* invd[2] = {h->inv_diag + n, h->inv_diag + n};
    ILS_CK(cholesky_f64_batch(n, 1, mats, invd, h->stash64, h->dstatus2, s));
    ILS_CK(cudaMemcpyAsync(h->h_status + 3, h->dstatus2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ILS_CK(cudaStreamSynchronize(s));
    if (h->h_status[3] != 0) return (ils_status)h->h_status[3];
  }
  return ILS_OK;
}

// Wait for the setup enqueued by compute_setup and report its pivot / input status.
ils_status setup_finish(ils_handle h) {
  ILS_CK(cudaStreamSynchronize(h->stream));
  return setup_check(h, nullptr);
}

// Autotune the sweep shapes for this handle's n once per process (mixed precision only).
ils_status tune_handle(ils_handle h) {
  if (h->opt.precision == ILS_FP64 || h->opt.method != ILS_SP) return ILS_OK;
  // the tuning times sweeps with B: only then does the handle's stream wait for it
  if (h->b_async && (!h->tune_cache.empty() || !sweeps_tuned(h->n, h->opt.precision))) {
    ILS_CK(ensure_b(h));
    ILS_CK(cudaStreamWaitEvent(h->stream, h->ev_b, 0));
  }
  ILS_CK(tune_sweeps(h->n, h->opt.precision, h->P32, h->mf ? nullptr : h->Bt32, h->Bt16, h->r32, h->d32a, h->st,
                     h->stream, h->tune_cache.empty() ? nullptr : h->tune_cache.c_str()));
  return ILS_OK;
}

void free_handle(ils_handle h) {
  if (!h) return;
  if (h->block) cudaFreeAsync(h->block, h->stream);
  for (cudaStream_t x : {h->s_aux, h->s_h, h->s_est, h->s_b})
    if (x) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  for (cudaEvent_t e : {h->ev_start, h->ev_g2, h->ev_g1, h->ev_hd, h->ev_h, h->ev_acopy, h->ev_rhs, h->ev_split2,
                        h->ev_mma, h->ev_hs, h->ev_b, h->ev_pb, h->ev_p,
                        h->ev_estk, h->ev_est})
    if (e) cudaEventDestroy(e);
  if (h->h_st) cudaFreeHost(h->h_st);
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

// One pass over kk <= kMaxRhsPerPass right-hand sides, in three phases so that many
// handles can have passes in flight on different streams: pass_begin enqueues A^T J b,
// the start vector and the device state; pass_launch enqueues outer steps (each returns
// at once after completion); pass_end synchronizes, launches more steps if needed and
// collects the results.
ils_status pass_begin(ils_handle h, int64_t c0, int64_t kk, const double* B, int64_t ldb, const double* X,
                      int64_t ldx, int x0_zero, double tol) {
  const int method = h->opt.method;
  cudaStream_t s = h->stream;
  const int64_t m = h->m, n = h->n, p = h->p;
  if (c0 == 0 && timing_event(h, 8)) ILS_CK(cudaEventRecord(h->ev[8], s));  // the solve's first work
  // bbar = A^T J b (Alg. 1 step 4), c = P bbar.
  if (h->sparse) {
    ILS_CK(sparse_rhs_bar(n, p, kk, h->sc, B, ldb, h->bbar, n, s));
    ILS_CK(sq_norms_cols_f64(n, kk, h->bbar, n, h->bnorm2, s));
  } else if (h->pending && h->overlap) {
    // After an asynchronous setup, A^T J b needs only the copy of A: the second stream
    // forms it beside the setup's last products.
    cudaStream_t a = h->s_aux;
    ILS_CK(cudaStreamWaitEvent(a, h->ev_acopy, 0));
    ILS_CK(rhs_bar_f64(m, n, p, kk, h->A, m, B, ldb, h->bbar, n, a));
    ILS_CK(sq_norms_cols_f64(n, kk, h->bbar, n, h->bnorm2, a));
    ILS_CK(cudaEventRecord(h->ev_rhs, a));
    ILS_CK(cudaStreamWaitEvent(s, h->ev_rhs, 0));
  } else {
    ILS_CK(rhs_bar_f64(m, n, p, kk, h->A, m, B, ldb, h->bbar, n, s));
    ILS_CK(sq_norms_cols_f64(n, kk, h->bbar, n, h->bnorm2, s));
  }
  if (h->opt.precision == ILS_FP64 && !h->mf) ILS_CK(gemv_cols_f64(n, kk, h->P, n, h->bbar, n, h->cvec, n, s));
  if (x0_zero) {
    ILS_CK(cudaMemsetAsync(h->X0, 0, sizeof(double) * n * kk, s));
  } else {
    ILS_CK(cudaMemcpy2DAsync(h->X0, sizeof(double) * n, X, sizeof(double) * ldx, sizeof(double) * n, kk,
                             cudaMemcpyDeviceToDevice, s));
  }
  init_state_kernel<<<1, 32, 0, s>>>(h->st, h->opt.max_outer, h->col_done, h->col_inner, (int)kk);
  note_launch();
  ILS_CK(cudaGetLastError());
  SpIterArgs a;
  a.n = n;
  a.k = kk;
  const bool mixed = h->opt.precision != ILS_FP64;
  const bool warm = method != ILS_SP && h->opt.warm_inner != 0;  // inner solves start at x_k
  a.mode = h->mf ? (mixed ? 4 : 3) : ((mixed || warm) ? 2 : (method == ILS_SP ? 0 : 1));
  a.vvec = h->vbuf;
  a.pad = 0;
  a.Bt = h->mf ? h->P : (method == ILS_SP ? h->Bt : h->G2);
  a.H = h->mf ? h->G1 : h->H;
  a.cvec = method == ILS_SP ? h->cvec : h->bbar;
  a.bhat_out = h->bhat;
  a.theta2 = h->opt.theta * h->opt.theta;
  a.theta_decay = h->opt.theta_decay;
  a.theta_min2 = h->opt.theta_min * h->opt.theta_min;
  a.col_target2 = h->col_target2;
  a.bbar = h->bbar;
  a.bnorm2 = h->bnorm2;
  a.X0 = h->X0;
  a.X1 = h->X1;
  a.tol2 = tol2_of(h, tol);
  a.tol_scale = tol_scale_of(h);
  a.wait_ns = h->opt.wait_limit_ns;
  a.col_done = h->col_done;
  a.col_rr = h->col_rr;
  a.col_iters = h->col_iters;
  a.partials = h->partials;
  a.st = h->st;
  RandArgs ra;
  ra.n = n;
  ra.k = kk;
  ra.m = m;
  ra.p = p;
  ra.A = h->A;
  ra.G1 = h->G1;
  ra.norms2 = h->norms2;
  ra.inv_norms2 = h->inv_norms2;
  ra.cum = h->cum;
  ra.bhat = h->bhat;
  ra.X0 = h->X0;
  ra.X1 = h->X1;
  ra.col_done = h->col_done;
  ra.col_target2 = h->col_target2;
  ra.col_inner = h->col_inner;
  ra.st = h->st;
  ra.seed = h->opt.seed;
  ra.chain0 = c0;
  ra.max_inner = h->opt.max_inner > 0 ? h->opt.max_inner : 200 * n;
  ra.check_every = h->opt.check_every > 0 ? h->opt.check_every : n;
  ra.greedy = h->opt.scd_sampler == 1 ? 1 : 0;
  ra.same_index = h->opt.scd_sampler == 2 ? 1 : 0;
  ra.vec_in_smem = h->vec_in_smem ? 1 : 0;
  ra.correction = (mixed && h->sparse && method == ILS_SP_RK_RGS) || warm ? 1 : 0;
  ra.vec_scratch = h->vec_scratch;
  ra.alpha_fixed = method == ILS_SP_SCD && h->opt.alpha_mode == 1 ? h->opt.alpha_fixed : 0;
  ra.gram_form = h->opt.inner_form;
  ra.alias = method == ILS_SP_RK_RGS && h->opt.sampler == 1 ? 1 : 0;
  ra.alias_prob = h->alias_prob;
  ra.alias_idx = h->alias_idx;
  ra.picks = c0 == 0 ? h->picks : nullptr;
  ra.picks_cap = h->picks_cap;
  ra.inner_ns = c0 == 0 ? h->inner_ns : nullptr;
  if (c0 == 0 && method != ILS_SP) ILS_CK(cudaMemsetAsync(h->inner_ns, 0, sizeof(unsigned long long), s));
  MixedArgs ma;
  ma.n = n;
  ma.k = kk;
  ma.sweeps = h->opt.sweeps > 0 ? h->opt.sweeps : 3;
  ma.pad = 0;
  ma.r = h->bhat;
  ma.r32 = h->r32;
  ma.c32 = h->c32;
  ma.d32[0] = h->d32a;
  ma.d32[1] = h->d32b;
  ma.P32 = h->P32;
  ma.Bt32 = h->Bt32;
  ma.Bt16 = h->Bt16;
  ma.X0 = h->X0;
  ma.X1 = h->X1;
  ma.col_done = h->col_done;
  ma.st = h->st;
  ma.Hh = h->Hh;
  ma.Hl = h->Hl;
  ma.He = h->He;
  ma.A2_32 = h->b_async ? h->G2_32 : nullptr;  // sweeps from P and Abar2 where B is formed beside
  h->pa = a;
  h->pra = ra;
  h->pma = ma;
  h->pass_k = kk;
  h->pass_launched = 0;
  h->pass_mixed = mixed;
  return ILS_OK;
}

// Enqueue up to `count` more outer steps of the pass in flight (never past max_outer + 1).
ils_status pass_launch(ils_handle h, int64_t count) {
  cudaStream_t s = h->stream;
  const int method = h->opt.method;
  const int64_t cap = h->opt.max_outer + 1;
  const int64_t todo = std::min(count, cap - h->pass_launched);
  if (todo > 0 && h->pass_launched == 0 && h->pass_mixed && !h->mf && !h->sparse && h->pass_k == 1) {
    // One right-hand side on the explicit route: the whole refinement in one launch.  Under
    // the error-bound stop, a provisional launch runs beside the kappa estimate and a second
    // one, after it, applies the final rule (solve_fused.cu).
    const bool split = h->opt.stop_rule == ILS_STOP_ERR_BOUND && h->ev_estk;
    BReady b_wait;
    if (h->b_async) {
      b_wait.fn = b_ready_event;
      b_wait.ctx = h;
    }
    const cudaError_t e =
        mixed_solve_fused(h->pa, h->pma, h->opt.precision, h->coop_sync, s, split ? 1 : 0, b_wait);
    if (e == cudaSuccess) {
      if (split) {
        ILS_CK(cudaStreamWaitEvent(s, h->ev_estk, 0));
        ILS_CK(mixed_solve_fused(h->pa, h->pma, h->opt.precision, h->coop_sync, s, 2, b_wait));
      }
      ILS_CK(ensure_b(h));  // B behind the solve's kernels, where it was deferred
      h->pass_launched = cap;
      return ILS_OK;
    }
    if (e != cudaErrorNotSupported) ILS_CK(e);
  }
  // every other path reads kappa_est from its first step on, and B
  if (h->pass_launched == 0 && h->opt.stop_rule == ILS_STOP_ERR_BOUND && h->ev_estk)
    ILS_CK(cudaStreamWaitEvent(s, h->ev_estk, 0));
  if (h->pass_launched == 0 && h->b_async) {
    ILS_CK(ensure_b(h));
    ILS_CK(cudaStreamWaitEvent(s, h->ev_b, 0));
  }
  for (int64_t i = 0; i < todo; ++i) {
    if (h->mf) {
      for (int c = 0; c < (int)h->pass_k; ++c)
        ILS_CK(aq_product_iterate(h->q, h->n, h->Aq64r, h->opt.precision == ILS_FP64 ? 0 : 3, h->X0, h->X1, h->st,
                                  h->col_done, c, h->sp_part,
                                  h->vbuf + c * h->n, s));
    }
    ILS_CK(sp_iterate_f64(h->pa, s));
    if (h->sparse && method == ILS_SP_RK_RGS)
      ILS_CK(rkrgs_sparse_chain(h->pra, h->sc, h->pass_mixed, s));
    else if (h->pass_mixed && h->mf)
      ILS_CK(mixed_correct_mf(h->pma, h->opt.precision, h->q, h->Aq_lo, h->sp_part, h->vbuf, h->d64, h->t32, s));
    else if (h->pass_mixed) ILS_CK(mixed_correct(h->pma, h->opt.precision, s));
    else if (method != ILS_SP) ILS_CK(rand_chain_f64(h->pra, method, s));
  }
  h->pass_launched += todo;
  return ILS_OK;
}

int64_t first_chunk(ils_handle h) {
  if (h->opt.precision != ILS_FP64) return 4;  // three refinements and the final test, typically
  return h->opt.method == ILS_SP ? 16 : 4;
}

ils_status pass_finish_enqueue(ils_handle h, double* X, int64_t ldx);
void pass_collect(ils_handle h, ils_info* agg);

ils_status pass_end(ils_handle h, double* X, int64_t ldx, ils_info* agg) {
  cudaStream_t s = h->stream;
  const int64_t cap = h->opt.max_outer + 1;
  int64_t chunk = std::max<int64_t>(first_chunk(h), 1);
  // The answer and the per-column results (with the state) are enqueued with the first
  // state read, so a pass that finished within its first chunk costs one host round trip;
  // if it has not, they are enqueued again once it has.
  if (h->pra.chain0 == 0 && timing_event(h, 9)) ILS_CK(cudaEventRecord(h->ev[9], s));
  ils_status st = pass_finish_enqueue(h, X, ldx);
  if (st != ILS_OK) return st;
  ILS_CK(cudaStreamSynchronize(s));
  if (h->h_st->done) {
    pass_collect(h, agg);
    return ILS_OK;
  }
  for (;;) {
    if (h->h_st->done || h->pass_launched >= cap) break;
    chunk = std::min<int64_t>(chunk * 2, 1024);
    if ((st = pass_launch(h, chunk)) != ILS_OK) return st;
    ILS_CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    ILS_CK(cudaStreamSynchronize(s));
  }
  if (!h->h_st->done) return ILS_ERR_TIMEOUT;  // cannot happen: the cap launch always finishes
  if ((st = pass_finish_enqueue(h, X, ldx)) != ILS_OK) return st;
  ILS_CK(cudaStreamSynchronize(s));
  pass_collect(h, agg);
  return ILS_OK;
}

// The answer of the pass to X and the per-column results to the pinned host mirrors
// (enqueued only; nothing here waits, so it can be captured in a graph).
ils_status pass_finish_enqueue(ils_handle h, double* X, int64_t ldx) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n, kk = h->pass_k;
  const bool inner_time = h->opt.method != ILS_SP && h->pra.chain0 == 0;
  const ResultGather g = {h->st, h->col_rr, h->bnorm2, h->col_iters, h->col_inner,
                          inner_time ? h->inner_ns : nullptr, h->res, kk};
  ILS_CK(copy_final_f64(n, kk, h->X0, h->X1, h->st, X, ldx, s, &g));
  // one copy of the state and every per-column result (the inner time only where it was
  // measured: the copy stops short of it otherwise)
  ILS_CK(cudaMemcpyAsync(h->h_st, h->res, inner_time ? kResBytes : kResInnerNs, cudaMemcpyDeviceToHost, s));
  if (h->pra.chain0 == 0 && timing_event(h, 10)) ILS_CK(cudaEventRecord(h->ev[10], s));
  return ILS_OK;
}

// Fold the host mirrors of a finished pass into *agg (after a synchronization).
void pass_collect(ils_handle h, ils_info* agg) {
  const int64_t kk = h->pass_k;
  const bool mixed = h->pass_mixed;
  for (int64_t c = 0; c < kk; ++c) {
    const double bn = h->h_bn[c];
    const double rel = bn > 0.0 ? std::sqrt(h->h_rr[c] / bn) : std::sqrt(h->h_rr[c]);
    agg->relres = std::max(agg->relres, rel);
    if (rel != rel) agg->relres = rel;
    if (mixed && h->pra.correction) {
      agg->refinements = std::max<int64_t>(agg->refinements, h->h_iters[c]);
      agg->outer_iters = std::max<int64_t>(agg->outer_iters, h->h_iters[c]);
    } else if (mixed) {
      agg->refinements = std::max<int64_t>(agg->refinements, h->h_iters[c]);
      agg->outer_iters = std::max<int64_t>(agg->outer_iters, h->h_iters[c] * h->pma.sweeps);
    } else {
      agg->outer_iters = std::max<int64_t>(agg->outer_iters, h->h_iters[c]);
    }
    agg->inner_iters = std::max<int64_t>(agg->inner_iters, h->h_inner[c]);
  }
  const int32_t st = h->h_st->status;
  if (st != 0 && agg->status == 0) agg->status = st;
}

// ---------------------------------------------------------------------------------------
// Wide SP (many right-hand sides at once, FP64, explicit route): with k columns the
// products of Alg. 1 are dense GEMMs, bbar = A^T J B (m x n x k), c = P bbar, and per step
// B X_k and H X_k (n x n x k), so one pass covers every column instead of passes of
// kMaxRhsPerPass.  A column stops on the same test as the narrow path and keeps x_k.
// ---------------------------------------------------------------------------------------
constexpr int kWideMinRhs = 32;
constexpr int kWideThreads = 256;

__global__ void __launch_bounds__(kWideThreads)
wide_step_kernel(int64_t n, const double* __restrict__ BX, const double* __restrict__ HX,
                 const double* __restrict__ bb, const double* __restrict__ cc, const double* __restrict__ bn,
                 const double* __restrict__ Xa, double* __restrict__ Xb, int32_t* __restrict__ done,
                 double* __restrict__ rr_out, int64_t* __restrict__ iters, int64_t it, int64_t max_outer, double tol2,
                 const double* __restrict__ tol_scale, int32_t* __restrict__ remaining, int32_t* __restrict__ status) {
  const int64_t c = blockIdx.x;
  const size_t off = (size_t)c * n;
  __shared__ double red[kWideThreads / 32];
  __shared__ int finish;
  if (done[c]) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Xb[off + i] = Xa[off + i];
    return;
  }
  double part = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = bb[off + i] - HX[off + i];
    part = fma(r, r, part);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double rr = 0.0;
    for (int w = 0; w < kWideThreads / 32; ++w) rr += red[w];
    const bool finite = isfinite(rr);
    const bool conv = finite && rr <= tol2 * (tol_scale ? *tol_scale : 1.0) * bn[c];
    finish = (!finite || conv || it >= max_outer) ? 1 : 0;
    if (finish) {
      done[c] = 1;
      rr_out[c] = rr;
      iters[c] = it;
      atomicSub(remaining, 1);
      if (!finite) atomicCAS(status, 0, ILS_ERR_NONFINITE);
      else if (!conv) atomicCAS(status, 0, ILS_ERR_NO_CONVERGENCE);
    }
  }
  __syncthreads();
  if (finish) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Xb[off + i] = Xa[off + i];  // return x_k
  } else {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Xb[off + i] = BX[off + i] + cc[off + i];
  }
}

__global__ void wide_init_kernel(int64_t k, int32_t* done, int32_t* remaining, int32_t* status) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x)
    done[c] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *remaining = (int32_t)k;
    *status = 0;
  }
}

ils_status wide_solve(ils_handle h, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx, int x0_zero,
                      double tol, ils_info* agg) {
  cudaStream_t s = h->stream;
  const int64_t m = h->m, n = h->n, p = h->p;
  const size_t nk = (size_t)n * (size_t)k;
  const size_t work = std::max(gemm_tn_work_elems(m, n, k, false, nullptr), gemm_tn_work_elems(n, n, k, false, nullptr));
  Carver dry{nullptr, 0, true};
  auto layout = [&](Carver& c, double** bufs, double** bn, double** rr, int64_t** it, int32_t** dn, int32_t** rem,
                    int32_t** stt, double** wk) {
    for (int i = 0; i < 6; ++i) bufs[i] = c.take<double>(nk);
    *bn = c.take<double>(k);
    *rr = c.take<double>(k);
    *it = c.take<int64_t>(k);
    *dn = c.take<int32_t>(k);
    *rem = c.take<int32_t>(1);
    *stt = c.take<int32_t>(1);
    *wk = c.take<double>(std::max<size_t>(work, 1));
  };
  double* bufs[6];
  double *bn, *rr, *wk;
  int64_t* itv;
  int32_t *dn, *rem, *stt;
  layout(dry, bufs, &bn, &rr, &itv, &dn, &rem, &stt, &wk);
  void* block = nullptr;
  if (cudaMallocAsync(&block, dry.off, s) != cudaSuccess) {
    cudaGetLastError();
    return ILS_ERR_OOM;
  }
  Carver real{(char*)block, 0, false};
  layout(real, bufs, &bn, &rr, &itv, &dn, &rem, &stt, &wk);
  double *bb = bufs[0], *cc = bufs[1], *Xa = bufs[2], *Xb = bufs[3], *BX = bufs[4], *HX = bufs[5];
  ils_status st = ILS_OK;
  auto ck = [&](cudaError_t e, const char* what, int line) {
    if (e != cudaSuccess && st == ILS_OK) st = record_cuda_error(e, what, line);
    return st == ILS_OK;
  };
  // bbar = A^T J B (Alg. 1 step 4), c = P bbar
  ck(gemm_tn_f64(m, n, k, h->A, m, B, ldb, p, bb, n, false, false, wk, s), "gemm bbar", __LINE__);
  if (st == ILS_OK) ck(sq_norms_cols_f64(n, k, bb, n, bn, s), "norms", __LINE__);
  if (st == ILS_OK) ck(gemm_tn_f64(n, n, k, h->P, n, bb, n, n, cc, n, false, false, wk, s), "gemm c", __LINE__);
  if (st == ILS_OK) {
    if (x0_zero) ck(cudaMemsetAsync(Xa, 0, sizeof(double) * nk, s), "memset", __LINE__);
    else ck(cudaMemcpy2DAsync(Xa, sizeof(double) * n, X, sizeof(double) * ldx, sizeof(double) * n, k,
                              cudaMemcpyDeviceToDevice, s), "copy x0", __LINE__);
  }
  if (st == ILS_OK) {
    wide_init_kernel<<<(unsigned)std::min<int64_t>((k + 255) / 256, 1024), 256, 0, s>>>(k, dn, rem, stt);
    note_launch();
    ck(cudaGetLastError(), "wide init", __LINE__);
  }
  int32_t* h_rem = h->h_status + 4;
  int32_t* h_stt = h->h_status + 5;
  for (int64_t it = 0; st == ILS_OK && it <= h->opt.max_outer; ++it) {
    // x_{k+1} = B x_k + c (Alg. 1 step 6) and r_k = bbar - H x_k, for every column at once
    ck(gemm_tn_f64(n, n, k, h->Bt, n, Xa, n, n, BX, n, false, false, wk, s), "gemm B x", __LINE__);
    if (st == ILS_OK) ck(gemm_tn_f64(n, n, k, h->H, n, Xa, n, n, HX, n, false, false, wk, s), "gemm H x", __LINE__);
    if (st != ILS_OK) break;
    wide_step_kernel<<<(unsigned)k, kWideThreads, 0, s>>>(n, BX, HX, bb, cc, bn, Xa, Xb, dn, rr, itv, it,
                                                          h->opt.max_outer, tol2_of(h, tol), tol_scale_of(h), rem,
                                                          stt);
    note_launch();
    if (!ck(cudaGetLastError(), "wide step", __LINE__)) break;
    std::swap(Xa, Xb);
    ck(cudaMemcpyAsync(h_rem, rem, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "d2h", __LINE__);
    if (st == ILS_OK) ck(cudaStreamSynchronize(s), "sync", __LINE__);
    if (st == ILS_OK && *h_rem == 0) break;
  }
  // Every column has finished (the step with it == max_outer finishes the rest): Xa holds
  // each column's returned iterate.
  std::vector<double> hrr(k), hbn(k);
  std::vector<int64_t> hit(k);
  if (st == ILS_OK)
    ck(cudaMemcpy2DAsync(X, sizeof(double) * ldx, Xa, sizeof(double) * n, sizeof(double) * n, k,
                         cudaMemcpyDeviceToDevice, s), "copy x", __LINE__);
  if (st == ILS_OK) ck(cudaMemcpyAsync(hrr.data(), rr, sizeof(double) * k, cudaMemcpyDeviceToHost, s), "d2h", __LINE__);
  if (st == ILS_OK) ck(cudaMemcpyAsync(hbn.data(), bn, sizeof(double) * k, cudaMemcpyDeviceToHost, s), "d2h", __LINE__);
  if (st == ILS_OK) ck(cudaMemcpyAsync(hit.data(), itv, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, s), "d2h", __LINE__);
  if (st == ILS_OK) ck(cudaMemcpyAsync(h_stt, stt, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "d2h", __LINE__);
  if (st == ILS_OK) ck(cudaStreamSynchronize(s), "sync", __LINE__);
  cudaFreeAsync(block, s);
  if (st != ILS_OK) return st;
  for (int64_t c = 0; c < k; ++c) {
    const double rel = hbn[c] > 0.0 ? std::sqrt(hrr[c] / hbn[c]) : std::sqrt(hrr[c]);
    agg->relres = std::max(agg->relres, rel);
    if (rel != rel) agg->relres = rel;
    agg->outer_iters = std::max<int64_t>(agg->outer_iters, hit[c]);
  }
  if (*h_stt != 0 && agg->status == 0) agg->status = *h_stt;
  return ILS_OK;
}

ils_status sp_pass(ils_handle h, int64_t c0, int64_t kk, const double* B, int64_t ldb, double* X, int64_t ldx,
                   int x0_zero, double tol, ils_info* agg) {
  ils_status st = pass_begin(h, c0, kk, B, ldb, X, ldx, x0_zero, tol);
  if (st != ILS_OK) return st;
  if ((st = pass_launch(h, first_chunk(h))) != ILS_OK) return st;
  return pass_end(h, X, ldx, agg);
}

// Validate a problem, allocate its handle and carve its device memory (stream-ordered
// on `stream`); nothing is computed yet.
ils_status create_handle(ils_handle* out, int64_t m, int64_t n, int64_t p, int64_t q, const double* A, int64_t lda,
                         const ils_options* o, cudaStream_t stream, int64_t sparse_nnz = -1,
                         bool overlap_ok = true) {
  *out = nullptr;
  const bool sparse = sparse_nnz >= 0;
  if (n < 1 || n > kMaxN || p < n || q < 0 || m != p + q || m > ((int64_t)1 << 31)) return ILS_ERR_INVALID_ARG;
  if (!sparse && (lda < m || !A)) return ILS_ERR_INVALID_ARG;
  if (sparse && sparse_nnz >= ((int64_t)1 << 31)) return ILS_ERR_INVALID_ARG;
  ils_options opt;
  if (o) opt = *o;
  else ils_options_default(&opt);
  if (validate_options(&opt) != ILS_OK) return ILS_ERR_INVALID_ARG;
  if (opt.route < ILS_ROUTE_AUTO || opt.route > ILS_ROUTE_MATRIX_FREE) return ILS_ERR_INVALID_ARG;
  if (opt.stop_rule == ILS_STOP_ERR_BOUND && opt.estimate == 0) opt.estimate = 2;  // the rule reads kappa_est
  if (opt.estimate < 0 || opt.estimate > 2) return ILS_ERR_INVALID_ARG;
  if (opt.estimate && n > 4096) return ILS_ERR_INVALID_ARG;  // the Lanczos clusters hold n <= 4096
  if (opt.method == ILS_SP_SCD && opt.alpha_mode == 1 && (opt.alpha_fixed < 1 || opt.alpha_fixed > n))
    return ILS_ERR_INVALID_ARG;
  // The Gram-space chain keeps three n-vectors in registers (n <= 8192); the sparse chains have
  // their own column sampling (inverse CDF) and column form.
  if (opt.inner_form == 1 && (opt.method != ILS_SP_RK_RGS || sparse || n > 8192)) return ILS_ERR_INVALID_ARG;
  if (opt.sampler == 1 && (opt.method != ILS_SP_RK_RGS || sparse)) return ILS_ERR_INVALID_ARG;
  if (sparse) {
    // The Grams of a sparse A come from its stored entries (FP64); the route is explicit.
    if (opt.route == ILS_ROUTE_MATRIX_FREE) return ILS_ERR_INVALID_ARG;
    const bool chain32 = opt.method == ILS_SP_RK_RGS && opt.precision == ILS_FP32_REFINE;
    if (opt.precision != ILS_FP64 && opt.method != ILS_SP && !chain32) return ILS_ERR_INVALID_ARG;
    opt.gram = ILS_GRAM_FP64;
    opt.route = ILS_ROUTE_EXPLICIT;
  } else if (opt.precision != ILS_FP64) {
    if (opt.method != ILS_SP) return ILS_ERR_INVALID_ARG;  // mixed precision refines the SP method
    opt.gram = ILS_GRAM_SPLIT;  // the FP64 refinement needs FP64-accurate Grams; these are the fast ones
  }
  if (opt.sweeps < 0) return ILS_ERR_INVALID_ARG;
  if (opt.chain_ctas != 0 && opt.chain_ctas != -1 && opt.chain_ctas != 1 && opt.chain_ctas != 2 &&
      opt.chain_ctas != 4 && opt.chain_ctas != 8)
    return ILS_ERR_INVALID_ARG;
  bool mf = false;
  if (opt.route == ILS_ROUTE_MATRIX_FREE) {
    if (opt.method != ILS_SP || n > 512 || q < 1) return ILS_ERR_INVALID_ARG;
    mf = true;
  } else if (opt.route == ILS_ROUTE_AUTO && opt.method == ILS_SP && n <= 512 && q > 0 && !sparse) {
    // The route that minimises setup + expected iterations by measured rates (route_tune.cu).
    bool pick = false;
    double model[8];
    const bool split = opt.gram == ILS_GRAM_SPLIT || opt.precision != ILS_FP64;
    const int est_steps = opt.estimate ? (opt.lanczos_steps > 0 ? opt.lanczos_steps : 24) : 0;
    if (route_prefers_matrix_free(q, n, opt.precision, split, est_steps, &pick, model) == cudaSuccess) {
      mf = pick;
      std::lock_guard<std::mutex> lock(g_route_mu);
      std::memcpy(g_route_model, model, sizeof(model));
      g_route_model[8] = pick ? 1.0 : 0.0;
    } else {
      cudaGetLastError();
      mf = q > 32 * n;  // no measurement possible: the size rule
    }
  }
  ils_handle h = new (std::nothrow) ils_handle_s();
  if (!h) return ILS_ERR_OOM;
  h->m = m;
  h->n = n;
  h->p = p;
  h->q = q;
  h->opt = opt;
  if (opt.tune_cache) h->tune_cache = opt.tune_cache;
  h->opt.tune_cache = nullptr;  // the handle keeps its own copy of the path
  h->mf = mf;
  h->sparse = sparse;
  h->nnz = sparse ? sparse_nnz : 0;
  h->stream = stream;
  h->overlap = overlap_ok && !sparse && !mf && opt.method == ILS_SP && opt.precision != ILS_FP64 &&
               opt.gram == ILS_GRAM_SPLIT && q > 0 && !opt.factor64;
  if (sparse && opt.method == ILS_SP_RK_RGS && opt.chain_ctas >= 0) {
    const double col_entries = (double)sparse_nnz * ((double)p / (double)m) / (double)n;  // A_1 entries per column
    const bool fp32 = opt.precision == ILS_FP32_REFINE;
    h->sc.cs = rkrgs_cluster_plan(n, p, fp32, opt.chain_ctas, col_entries, &h->sc.slice, &h->sc.nres);
    h->sc.ldg = (int32_t)((n + (fp32 ? 3 : 1)) / (fp32 ? 4 : 2) * (fp32 ? 4 : 2));
    if (opt.chain_ctas > 0 && h->sc.cs != opt.chain_ctas) {
      free_handle(h);
      return ILS_ERR_INVALID_ARG;  // the requested cluster does not fit
    }
  }
  const size_t work = sparse ? gemm_tn_work_elems(n, n, n, false, nullptr) : setup_work_elems(m, n, p, q);
  Carver dry{nullptr, 0, true};
  carve(h, dry, work);
  h->block_bytes = dry.off;
  if (cudaMallocAsync(&h->block, h->block_bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    h->block = nullptr;
    free_handle(h);
    return ILS_ERR_OOM;
  }
  Carver real{(char*)h->block, 0, false};
  carve(h, real, work);
  if (h->overlap) {
    // The kappa estimate's cluster becomes ready beside the cooperative inverse: its stream
    // gets the highest priority, so the block scheduler places it first.
    int lo_prio = 0, hi_prio = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) == cudaSuccess &&
              cudaStreamCreateWithFlags(&h->s_aux, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&h->s_h, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&h->s_b, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t* e : {&h->ev_start, &h->ev_g2, &h->ev_g1, &h->ev_hd, &h->ev_h, &h->ev_acopy, &h->ev_rhs,
                           &h->ev_split2, &h->ev_mma, &h->ev_hs, &h->ev_b, &h->ev_pb})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (h->opt.estimate) {
      ok = ok && cudaStreamCreateWithPriority(&h->s_est, cudaStreamNonBlocking, hi_prio) == cudaSuccess;
      for (cudaEvent_t* e : {&h->ev_p, &h->ev_estk, &h->ev_est})
        ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      free_handle(h);
      return ILS_ERR_CUDA;
    }
  }
  // pinned host block: the gathered results (the device layout of h->res), then the setup
  // status words and the estimates
  const size_t host_bytes = align_up(kResBytes) + align_up(sizeof(int32_t) * 64) + align_up(8 * sizeof(double));
  char* hb = nullptr;
  if (cudaMallocHost((void**)&hb, host_bytes) != cudaSuccess) {
    cudaGetLastError();
    free_handle(h);
    return ILS_ERR_OOM;
  }
  h->h_st = (SolveState*)(hb + kResSt);
  h->h_rr = (double*)(hb + kResRr);
  h->h_bn = (double*)(hb + kResBn);
  h->h_iters = (int64_t*)(hb + kResIters);
  h->h_inner = (int64_t*)(hb + kResInner);
  h->h_inner_ns = (unsigned long long*)(hb + kResInnerNs);
  hb += align_up(kResBytes);
  h->h_status = (int32_t*)hb;
  hb += align_up(sizeof(int32_t) * 64);
  h->h_est = (double*)hb;
  for (int i = 0; i < 8; ++i) h->h_est[i] = 0.0;
  *h->h_inner_ns = 0ull;
  *out = h;
  return ILS_OK;
}

}  // namespace

extern "C" {

const char* ils_last_error(void) { return g_last_error; }

const char* ils_status_string(ils_status st) {
  switch (st) {
    case ILS_OK: return "ok";
    case ILS_ERR_INVALID_ARG: return "invalid argument";
    case ILS_ERR_NOT_SPD: return "A^T J A (or A_1^T A_1) is not symmetric positive definite";
    case ILS_ERR_NO_CONVERGENCE: return "outer-iteration cap reached before the tolerance";
    case ILS_ERR_NONFINITE: return "non-finite value in the input or the iteration";
    case ILS_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case ILS_ERR_CUDA: return "CUDA runtime error";
    case ILS_ERR_OOM: return "device memory allocation failed";
  }
  return "unknown status";
}

ils_status ils_options_default(ils_options* o) {
  if (!o) return ILS_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->method = ILS_SP;
  o->precision = ILS_FP64;
  o->gram = ILS_GRAM_FP64;
  o->max_outer = 20000;
  o->max_inner = 0;
  o->theta = 0.1;
  o->theta_decay = 1.0;
  o->theta_min = 0.0;
  o->check_every = 0;
  o->scd_sampler = 0;
  o->seed = 0;
  return ILS_OK;
}

ils_status ils_setup(ils_handle* out, int64_t m, int64_t n, int64_t p, int64_t q, const double* A, int64_t lda,
                     const ils_options* o, ils_stream_t stream) {
  if (!out) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  ils_handle h = nullptr;
  ils_status st = create_handle(&h, m, n, p, q, A, lda, o, (cudaStream_t)stream);
  if (st != ILS_OK) return st;
  st = ils_refactor(h, A, lda, stream);
  if (st != ILS_OK) {
    free_handle(h);
    return st;
  }
  *out = h;
  return ILS_OK;
}

ils_status ils_setup_csr(ils_handle* out, int64_t m, int64_t n, int64_t p, int64_t q, int64_t nnz,
                         const int32_t* rowptr, const int32_t* colind, const double* val, const ils_options* o,
                         ils_stream_t stream) {
  if (!out) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  if (nnz < 0 || !rowptr || (nnz > 0 && (!colind || !val))) return ILS_ERR_INVALID_ARG;
  ils_handle h = nullptr;
  ils_status st = create_handle(&h, m, n, p, q, nullptr, 0, o, (cudaStream_t)stream, nnz);
  if (st != ILS_OK) return st;
  st = compute_setup_sparse(h, rowptr, colind, val);
  if (st == ILS_OK) st = setup_finish(h);
  if (st == ILS_OK && h->opt.timing) collect_timings(h);
  if (st == ILS_OK) st = tune_handle(h);
  if (st != ILS_OK) {
    free_handle(h);
    return st;
  }
  *out = h;
  return ILS_OK;
}

ils_status ils_refactor(ils_handle h, const double* A, int64_t lda, ils_stream_t stream) {
  if (!h || !A || lda < h->m || h->sparse) return ILS_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  cudaStream_t s = h->stream;
  h->pending = false;
  ILS_CK(mark(h, 0));
  ils_status st;
  if (h->overlap) {  // the digit splits copy A into the handle
    st = compute_setup_overlap(h, A, lda);
  } else {
    ILS_CK(copy_matrix_f64(h->m, h->n, A, lda, h->A, s));
    st = compute_setup(h);
  }
  if (st == ILS_OK) st = setup_finish(h);
  if (st == ILS_OK && h->opt.timing) collect_timings(h);
  if (st == ILS_OK) st = tune_handle(h);
  return st;
}

ils_status ils_refactor_async(ils_handle h, const double* A, int64_t lda, ils_stream_t stream) {
  if (!h || !A || lda < h->m || h->sparse) return ILS_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  cudaStream_t s = h->stream;
  h->pending = false;
  ILS_CK(mark(h, 0));
  ils_status st;
  if (h->overlap) {  // the digit splits copy A into the handle and record ev_acopy
    st = compute_setup_overlap(h, A, lda);
  } else {
    ILS_CK(copy_matrix_f64(h->m, h->n, A, lda, h->A, s));
    st = compute_setup(h);
  }
  if (st != ILS_OK) return st;
  h->pending = true;
  // The sweep shapes are tuned once per process; that first time waits for the setup.
  return tune_handle(h);
}

ils_status ils_aq_product(ils_handle h, const double* x, double* v, int prec, ils_stream_t stream) {
  if (!h || !x || !v || prec < 0 || prec > 2 || !h->mf) return ILS_ERR_INVALID_ARG;
  const void* Ar = prec == 0 ? h->Aq64r : h->Aq_lo;
  if (prec != 0 && (h->opt.precision == ILS_FP64 || (prec == 1) != (h->opt.precision == ILS_FP32_REFINE)))
    return ILS_ERR_INVALID_ARG;
  const int kind = prec == 0 && h->opt.precision != ILS_FP64 ? 3 : prec;  // the mixed handles' double-FP32 copy
  ILS_CK(aq_product(h->q, h->n, Ar, kind, x, h->sp_part, v, (cudaStream_t)stream));
  return ILS_OK;
}

int ils_get_timings(ils_handle h, double* out, int count) {
  if (!h || !out || count < 0) return -1;
  const int c = count < 14 ? count : 14;
  for (int i = 0; i < c; ++i) out[i] = h->t_ms[i];
  return c;
}

int64_t ils_kernel_launches(void) { return ils::g_launches.load(std::memory_order_relaxed); }

int ils_tuned_shape(int64_t n, int64_t k, int bf16, int* warps, int* blocks) {
  return ils::ils_tuned_shape_impl(n, k, bf16, warps, blocks);
}

ils_status solve_many_now(ils_handle h, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                          int x0_zero, double tol, ils_info* info);

// The fields of ils_info beyond the iteration counts: the estimates, the certificate
// err_bound = kappa_est * relres and the times.
void fill_info_extras(ils_handle h, ils_info* agg, std::chrono::steady_clock::time_point t0) {
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  agg->t_solve_ms = ms;
  agg->t_setup_ms = h->t_ms[4];
  agg->t_inner_ms = h->opt.method != ILS_SP ? (double)*h->h_inner_ns * 1e-6 : 0.0;
  if (h->opt.estimate) {
    agg->rho_est = h->h_est[2];
    agg->kappa_est = h->h_est[3];
    agg->err_bound = agg->kappa_est * agg->relres;
  }
}

ils_status solve_many_checked(ils_handle h, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                              int x0_zero, double tol, ils_info* info, ils_stream_t stream);

ils_status ils_solve_many(ils_handle h, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                          int x0_zero, double tol, ils_info* info, ils_stream_t stream) {
  const auto t0 = std::chrono::steady_clock::now();
  ils_info agg;
  std::memset(&agg, 0, sizeof(agg));
  const ils_status st = solve_many_checked(h, k, B, ldb, X, ldx, x0_zero, tol, &agg, stream);
  if (h && st != ILS_ERR_INVALID_ARG) {
    fill_info_extras(h, &agg, t0);
    if (h->opt.timing) collect_timings(h);  // the solve's marks (the call synchronized)
  }
  if (info) *info = agg;
  return st;
}

ils_status solve_many_checked(ils_handle h, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                              int x0_zero, double tol, ils_info* info, ils_stream_t stream) {
  if (!h || k < 0 || (k > 0 && (!B || !X)) || ldb < h->m || ldx < h->n || !(tol >= 0.0))
    return ILS_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  if (h->pending) {
    // The setup was enqueued without a wait: solve behind it, then read its status (the
    // solve synchronized the stream).  A failed setup's status replaces the solve's; where
    // an FP64 factorization had to settle a failed FP32 test and formed P and B again, the
    // solve runs again on them.
    ils_info agg;
    std::memset(&agg, 0, sizeof(agg));
    ils_status st = solve_many_now(h, k, B, ldb, X, ldx, x0_zero, tol, &agg);
    h->pending = false;
    bool redone = false;
    const ils_status sst = setup_check(h, &redone);
    if (sst == ILS_OK && h->opt.timing) collect_timings(h);
    if (sst != ILS_OK) {
      agg.status = sst;
      if (info) *info = agg;
      return sst;
    }
    if (redone) return solve_many_checked(h, k, B, ldb, X, ldx, x0_zero, tol, info, stream);
    if (info) *info = agg;
    return st;
  }
  ils_info agg;
  std::memset(&agg, 0, sizeof(agg));
  const ils_status st = solve_many_now(h, k, B, ldb, X, ldx, x0_zero, tol, &agg);
  if (info) *info = agg;
  return st;
}

// The solve proper (ils_solve_many after its checks).
ils_status solve_many_now(ils_handle h, int64_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                          int x0_zero, double tol, ils_info* info) {
  ils_info& agg = *info;
  if (k >= kWideMinRhs && h->opt.method == ILS_SP && h->opt.precision == ILS_FP64 && !h->mf && !h->sparse) {
    ils_status st = wide_solve(h, k, B, ldb, X, ldx, x0_zero, tol, &agg);
    if (st != ILS_OK) agg.status = st;
    return (ils_status)agg.status;
  }
  if (k >= kWideMinRhs && h->opt.method == ILS_SP && h->opt.precision != ILS_FP64 && !h->mf && !h->sparse) {
    // Many right-hand sides, mixed precision: the FP64-accurate A^T J B and residuals as split
    // digit products on the tensor cores, FP32 sweeps (wide_mixed.cu).
    if (h->opt.stop_rule == ILS_STOP_ERR_BOUND && h->ev_estk) ILS_CK(cudaStreamWaitEvent(h->stream, h->ev_estk, 0));
    WideMixedArgs wa;
    wa.m = h->m;
    wa.n = h->n;
    wa.p = h->p;
    wa.A = h->A;
    wa.H = h->H;
    wa.P32 = h->P32;
    wa.Bt32 = h->Bt32;
    wa.sweeps = h->opt.sweeps > 0 ? h->opt.sweeps : 3;
    wa.max_outer = h->opt.max_outer;
    wa.tol2 = tol2_of(h, tol);
    wa.tol_scale = tol_scale_of(h);
    WideMixedResult wr;
    if (h->b_async) {
      ILS_CK(ensure_b(h));
      ILS_CK(cudaStreamWaitEvent(h->stream, h->ev_b, 0));
    }
    ILS_CK(wide_mixed_solve(wa, k, B, ldb, X, ldx, x0_zero, &wr, h->h_status + 8, h->stream));
    agg.relres = wr.relres;
    agg.refinements = wr.refinements;
    agg.outer_iters = wr.refinements * wa.sweeps;
    if (wr.status != 0) agg.status = wr.status;
    return (ils_status)agg.status;
  }
  for (int64_t c0 = 0; c0 < k; c0 += kMaxRhsPerPass) {
    const int64_t kk = std::min<int64_t>(kMaxRhsPerPass, k - c0);
    ils_status st = sp_pass(h, c0, kk, B + c0 * ldb, ldb, X + c0 * ldx, ldx, x0_zero, tol, &agg);
    if (st != ILS_OK) {
      agg.status = st;
      return st;
    }
  }
  return (ils_status)agg.status;
}

ils_status ils_solve(ils_handle h, const double* b, double* x, int x0_zero, double tol, ils_info* info,
                     ils_stream_t stream) {
  if (!h) return ILS_ERR_INVALID_ARG;
  return ils_solve_many(h, 1, b, h->m, x, h->n, x0_zero, tol, info, stream);
}

ils_status ils_get_matrix(ils_handle h, int which, double* dst, int64_t ldd, ils_stream_t stream) {
  if (!h || !dst || ldd < h->n || which < 0 || which > 4) return ILS_ERR_INVALID_ARG;
  // P exists for FP64 SP handles, B for those on the explicit route
  if (which >= 3 && (h->opt.method != ILS_SP || h->opt.precision != ILS_FP64)) return ILS_ERR_INVALID_ARG;
  if ((which == 1 || which == 4) && h->mf) return ILS_ERR_INVALID_ARG;  // never formed there
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = h->n;
  const double* src = nullptr;
  switch (which) {
    case 0: src = h->G1; break;
    case 1: src = h->G2; break;
    case 2:
      if (!h->l64_valid) {
        ILS_CK(cudaStreamSynchronize(s));
        const ils_status fs = factor_f64_now(h);
        if (fs != ILS_OK) return fs;
      }
      ILS_CK(copy_lower_zero_upper_f64(n, h->L, dst, ldd, s));
      return ILS_OK;
    case 3: src = h->P; break;
    case 4: {
      transpose_kernel<<<256, 256, 0, s>>>(n, h->Bt, dst, ldd);
      note_launch();
      ILS_CK(cudaGetLastError());
      return ILS_OK;
    }
  }
  ILS_CK(cudaMemcpy2DAsync(dst, sizeof(double) * ldd, src, sizeof(double) * n, sizeof(double) * n, n,
                           cudaMemcpyDeviceToDevice, s));
  return ILS_OK;
}

int ils_route_model(double* out, int count) {
  if (!out || count < 0) return -1;
  std::lock_guard<std::mutex> lock(ils::g_route_mu);
  const int c = count < 9 ? count : 9;
  for (int i = 0; i < c; ++i) out[i] = ils::g_route_model[i];
  return c;
}

ils_status ils_set_wait_limit(ils_handle h, int64_t limit_ns) {
  if (!h || limit_ns < 0) return ILS_ERR_INVALID_ARG;
  h->opt.wait_limit_ns = limit_ns;
  return ILS_OK;
}

ils_status ils_record_picks(ils_handle h, int32_t* picks, int64_t capacity) {
  if (!h || h->sparse || capacity < 0 || (picks && capacity == 0)) return ILS_ERR_INVALID_ARG;
  h->picks = picks;
  h->picks_cap = picks ? capacity : 0;
  return ILS_OK;
}

void ils_destroy(ils_handle h) { free_handle(h); }

// ---------------------------------------------------------------------------------------
// Batches of independent problems: each problem keeps its own handle; handles are spread
// round-robin over internal streams so their kernels run concurrently, and every host
// synchronization is deferred until all problems have been enqueued.
// ---------------------------------------------------------------------------------------
struct ils_batch_s {
  std::vector<ils_handle> h;
  std::vector<ils_problem> probs;   // the caller's A of every problem (re-read by a captured refactor)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;  // one per internal stream (join)
  cudaEvent_t fork = nullptr;
  // captured solve (ils_batch_capture / ils_batch_run)
  cudaGraphExec_t exec = nullptr;
  bool cap_refactor = false;
  int64_t cap_steps = 0;
  int64_t cap_launches = 0;  // kernels per replay
  std::vector<double*> cap_X;
  std::vector<int64_t> cap_ldx;
};

namespace {
constexpr int kBatchStreams = 16;

void free_batch(ils_batch b) {
  if (!b) return;
  for (ils_handle h : b->h) free_handle(h);
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  delete b;
}

// Internal streams wait for the caller's stream (fork); the caller's stream waits for
// the internal streams (join).
cudaError_t batch_fork(ils_batch b, cudaStream_t user) {
  cudaError_t e = cudaEventRecord(b->fork, user);
  for (size_t i = 0; e == cudaSuccess && i < b->streams.size(); ++i) e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
  return e;
}

cudaError_t batch_join(ils_batch b, cudaStream_t user) {
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; e == cudaSuccess && i < b->streams.size(); ++i) {
    e = cudaEventRecord(b->events[i], b->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, b->events[i], 0);
  }
  return e;
}
}  // namespace

ils_status ils_batch_setup(ils_batch* out, int64_t count, const ils_problem* probs, const ils_options* o,
                           ils_stream_t stream) {
  if (!out) return ILS_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !probs) return ILS_ERR_INVALID_ARG;
  ils_batch b = new (std::nothrow) ils_batch_s();
  if (!b) return ILS_ERR_OOM;
  const int ns = (int)std::min<int64_t>(count, kBatchStreams);
  b->streams.assign(ns, nullptr);
  b->events.assign(ns, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < ns; ++i)
    ok = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok || batch_fork(b, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return ILS_ERR_CUDA;
  }
  b->h.assign(count, nullptr);
  b->probs.assign(probs, probs + count);
  ils_status st = ILS_OK;
  for (int64_t i = 0; i < count && st == ILS_OK; ++i) {
    const ils_problem& pr = probs[i];
    cudaStream_t s = b->streams[i % ns];
    st = create_handle(&b->h[i], pr.m, pr.n, pr.p, pr.q, pr.A, pr.lda, o, s, -1, false);
    if (st != ILS_OK) break;
    ils_handle h = b->h[i];
    if (copy_matrix_f64(h->m, h->n, pr.A, pr.lda, h->A, s) != cudaSuccess) {
      cudaGetLastError();
      st = ILS_ERR_CUDA;
      break;
    }
    st = compute_setup(h);
  }
  for (int64_t i = 0; i < count && st == ILS_OK; ++i) st = setup_finish(b->h[i]);
  for (int64_t i = 0; i < count && st == ILS_OK; ++i) st = tune_handle(b->h[i]);
  if (st == ILS_OK && batch_join(b, (cudaStream_t)stream) != cudaSuccess) st = ILS_ERR_CUDA;
  if (st != ILS_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return ILS_OK;
}

ils_status ils_batch_solve(ils_batch b, int64_t k, const double* const* B, const int64_t* ldb, double* const* X,
                           const int64_t* ldx, int x0_zero, double tol, ils_info* infos, ils_stream_t stream) {
  if (!b || k < 0 || !(tol >= 0.0) || (k > 0 && (!B || !X))) return ILS_ERR_INVALID_ARG;
  const int64_t count = (int64_t)b->h.size();
  for (int64_t i = 0; i < count && k > 0; ++i) {
    const int64_t lb = ldb ? ldb[i] : b->h[i]->m, lx = ldx ? ldx[i] : b->h[i]->n;
    if (!B[i] || !X[i] || lb < b->h[i]->m || lx < b->h[i]->n) return ILS_ERR_INVALID_ARG;
  }
  std::vector<ils_info> agg(count);
  for (auto& a : agg) std::memset(&a, 0, sizeof(a));
  if (batch_fork(b, (cudaStream_t)stream) != cudaSuccess) return ILS_ERR_CUDA;
  ils_status worst = ILS_OK;
  for (int64_t c0 = 0; c0 < k; c0 += kMaxRhsPerPass) {
    const int64_t kk = std::min<int64_t>(kMaxRhsPerPass, k - c0);
    for (int64_t i = 0; i < count; ++i) {
      ils_handle h = b->h[i];
      const int64_t lb = ldb ? ldb[i] : h->m, lx = ldx ? ldx[i] : h->n;
      ils_status st = pass_begin(h, c0, kk, B[i] + c0 * lb, lb, X[i] + c0 * lx, lx, x0_zero, tol);
      if (st == ILS_OK) st = pass_launch(h, first_chunk(h));
      if (st != ILS_OK) return st;
    }
    for (int64_t i = 0; i < count; ++i) {
      ils_handle h = b->h[i];
      const int64_t lx = ldx ? ldx[i] : h->n;
      ils_status st = pass_end(h, X[i] + c0 * lx, lx, &agg[i]);
      if (st != ILS_OK) return st;
    }
  }
  if (batch_join(b, (cudaStream_t)stream) != cudaSuccess) return ILS_ERR_CUDA;
  for (int64_t i = 0; i < count; ++i) {
    if (infos) infos[i] = agg[i];
    if (agg[i].status != ILS_OK && worst == ILS_OK) worst = (ils_status)agg[i].status;
  }
  return worst;
}

ils_status ils_batch_capture(ils_batch b, int refactor, int64_t k, const double* const* B, const int64_t* ldb,
                             double* const* X, const int64_t* ldx, int x0_zero, double tol, int64_t steps,
                             ils_stream_t stream) {
  if (!b || k < 1 || k > kMaxRhsPerPass || !B || !X || !(tol >= 0.0) || steps < 1) return ILS_ERR_INVALID_ARG;
  const int64_t count = (int64_t)b->h.size();
  for (int64_t i = 0; i < count; ++i) {
    const int64_t lb = ldb ? ldb[i] : b->h[i]->m, lx = ldx ? ldx[i] : b->h[i]->n;
    if (!B[i] || !X[i] || lb < b->h[i]->m || lx < b->h[i]->n) return ILS_ERR_INVALID_ARG;
  }
  cudaStream_t user = (cudaStream_t)stream;
  if (user == nullptr) return ILS_ERR_INVALID_ARG;  // the legacy stream cannot be captured
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const int64_t launches0 = ils_kernel_launches();
  ILS_CK(cudaStreamBeginCapture(user, cudaStreamCaptureModeRelaxed));
  ils_status st = batch_fork(b, user) == cudaSuccess ? ILS_OK : ILS_ERR_CUDA;
  b->cap_X.assign(count, nullptr);
  b->cap_ldx.assign(count, 0);
  for (int64_t i = 0; i < count && st == ILS_OK; ++i) {
    ils_handle h = b->h[i];
    const int64_t lb = ldb ? ldb[i] : h->m, lx = ldx ? ldx[i] : h->n;
    b->cap_X[i] = X[i];
    b->cap_ldx[i] = lx;
    if (refactor) {
      const ils_problem& pr = b->probs[i];
      if (copy_matrix_f64(h->m, h->n, pr.A, pr.lda, h->A, h->stream) != cudaSuccess)
        st = ILS_ERR_CUDA;
      if (st == ILS_OK) st = compute_setup(h);
    }
    if (st == ILS_OK) st = pass_begin(h, 0, k, B[i], lb, X[i], lx, x0_zero, tol);
    if (st == ILS_OK) st = pass_launch(h, steps);
    if (st == ILS_OK && cudaMemcpyAsync(h->h_st, h->st, sizeof(SolveState), cudaMemcpyDeviceToHost, h->stream) !=
                            cudaSuccess)
      st = ILS_ERR_CUDA;
    if (st == ILS_OK) st = pass_finish_enqueue(h, X[i], lx);
  }
  if (st == ILS_OK && batch_join(b, user) != cudaSuccess) st = ILS_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(user, &graph);
  if (st == ILS_OK && ec != cudaSuccess) st = record_cuda_error(ec, "cudaStreamEndCapture", __LINE__);
  if (st == ILS_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
    if (ei != cudaSuccess) st = record_cuda_error(ei, "cudaGraphInstantiate", __LINE__);
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  if (st != ILS_OK) {
    b->exec = nullptr;
    return st;
  }
  b->cap_refactor = refactor != 0;
  b->cap_steps = steps;
  b->cap_launches = ils_kernel_launches() - launches0;
  return ILS_OK;
}

ils_status ils_batch_run(ils_batch b, ils_info* infos, ils_stream_t stream) {
  if (!b || !b->exec) return ILS_ERR_INVALID_ARG;
  cudaStream_t user = (cudaStream_t)stream;
  ILS_CK(cudaGraphLaunch(b->exec, user));
  note_launch(b->cap_launches);
  ILS_CK(cudaStreamSynchronize(user));
  const int64_t count = (int64_t)b->h.size();
  ils_status worst = ILS_OK;
  for (int64_t i = 0; i < count; ++i) {
    ils_handle h = b->h[i];
    ils_info agg;
    std::memset(&agg, 0, sizeof(agg));
    if (b->cap_refactor) {
      h->h_status[1] = h->opt.gram == ILS_GRAM_SPLIT ? h->h_status[1] : 0;
      ils_status sst = h->h_status[1] != 0 ? (h->h_status[1] == 2 ? ILS_ERR_NONFINITE : ILS_ERR_TIMEOUT)
                                           : (ils_status)*h->h_status;
      if (sst != ILS_OK) {
        agg.status = sst;
        if (infos) infos[i] = agg;
        if (worst == ILS_OK) worst = sst;
        continue;
      }
    }
    h->pass_launched = b->cap_steps;
    if (h->h_st->done) {
      pass_collect(h, &agg);  // the graph already stored x and the per-column results
    } else {
      ils_status st = pass_end(h, b->cap_X[i], b->cap_ldx[i], &agg);  // more steps than captured
      if (st != ILS_OK) return st;
    }
    if (infos) infos[i] = agg;
    if (agg.status != ILS_OK && worst == ILS_OK) worst = (ils_status)agg.status;
  }
  return worst;
}

ils_handle ils_batch_handle(ils_batch b, int64_t i) {
  if (!b || i < 0 || i >= (int64_t)b->h.size()) return nullptr;
  return b->h[i];
}

void ils_batch_destroy(ils_batch b) { free_batch(b); }

}  // extern "C"
