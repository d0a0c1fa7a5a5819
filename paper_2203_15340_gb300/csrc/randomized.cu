// Inner randomized solvers of SP-RK-RGS (Alg. 2 steps 7-12) and SP-SCD (Alg. 5 steps
// 6-12) on a dense A.  Each inner solve is a sequential chain of cheap steps, so one CTA
// runs one chain (one right-hand side); independent chains run on different SMs.  Random
// draws come from Philox4x32-10 with the counter layout (t_lo, t_hi, k, chain) and key
// (seed_lo, seed_hi).
//
// The SCD chain and the Gram-space RK-RGS chain keep their n-vectors in registers
// (element s of a vector lives in thread s mod T, slot s / T), so a step touches global
// memory only for the one or two columns of Abar1 it applies.
#include <cmath>

#include "ils_internal.h"
#include "philox.cuh"

namespace ils {
namespace {

// Smallest j with cum[j] > u * cum[n-1] (inverse CDF of the column law of Alg. 2 steps 8/10).
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

// Vose alias draw: column floor(u n), kept with its acceptance probability, else its alias.
// The fraction u n - floor(u n) is the second uniform (exact: u has 53 bits, n < 2^15).
__device__ __forceinline__ int alias_pick(const double* prob, const int32_t* alias, int n, double u) {
  const double x = u * (double)n;
  int j = (int)x;
  if (j >= n) j = n - 1;
  return (x - (double)j) < prob[j] ? j : alias[j];
}

// Rank i in 1..n with P(i) = (n+1)/(n i (i+1)): the law of the position (in decreasing
// |r|) of the index Alg. 5 picks when alpha ~ U{1..n} and the alpha-subset is uniform.
__device__ __forceinline__ int scd_rank(double u, int n) {
  const double num = u * (double)n;
  double i = ceil(num / ((double)(n + 1) - num));
  if (i < 1.0) i = 1.0;
  if (i > (double)n) i = (double)n;
  return (int)i;
}

// Fixed subset size alpha (Sec. 4): the pick is the i-th largest |r_s| with
// P(rank > i) = C(n-i, alpha) / C(n, alpha).  The survival function is evaluated as a
// product of exact-integer ratios taken left to right: over s < alpha of (n-i-s)/(n-s)
// for alpha <= kAlphaSearchMax (then the rank is found by bisection), else over s < i of
// (n-alpha-s)/(n-s) (then by a scan from i = 1; the expected rank (n+1)/(alpha+1) is
// small).  Both forms are non-increasing in i after rounding, so the result is the
// smallest i with survival <= 1 - u.
constexpr int kAlphaSearchMax = 16;

__device__ double fixed_survival(int i, int n, int alpha) {
  double prod = 1.0;
  for (int s = 0; s < alpha; ++s) {
    const int num = n - i - s;
    if (num <= 0) return 0.0;
    prod = __dmul_rn(prod, __ddiv_rn((double)num, (double)(n - s)));
  }
  return prod;
}

__device__ int scd_fixed_rank(double u, int n, int alpha) {
  const double thr = 1.0 - u;
  int hi = n - alpha + 1;
  if (alpha <= kAlphaSearchMax) {
    int lo = 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (fixed_survival(mid, n, alpha) <= thr) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  }
  int i = 1;
  double prod = __ddiv_rn((double)(n - alpha), (double)n);
  while (i < hi && !(prod <= thr)) {
    prod = __dmul_rn(prod, __ddiv_rn((double)(n - alpha - i), (double)(n - i)));
    ++i;
  }
  return i;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Key order of the SCD selection: larger |r| first, then lower index.  |r| is compared
// through its bit pattern (for non-negative doubles the unsigned integer order is the
// numeric order), so the selection runs on the integer pipes, not the scarce FP64 one.
// NaN patterns map to 0; a NaN in r also makes ||r||^2 non-finite, which ends the chain.
__device__ __forceinline__ unsigned long long abs_key(double v) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  return a > 0x7ff0000000000000ull ? 0ull : a;
}

__device__ __forceinline__ bool key_greater(unsigned long long a, int i, unsigned long long b, int j) {
  return a > b || (a == b && i < j);
}


// ---------------------------------------------------------------------------------------
// Rank selection over a register-resident vector: element s of r is r[s / T] of thread
// s mod T.  One call returns the index of the i-th largest |r_s| (ties to the lower
// index) together with r_j, and ||r||^2 of the same vector:
//   * i <= kTop: every warp takes its own top min(i, kTop) by that many warp-argmax rounds
//     (shuffles only), warp 0 merges the candidates of all warps (the global top i are
//     among them) -- two block barriers in all;
//   * i > kTop: radix selection on the 64-bit keys, eight 8-bit digits from the top with
//     a 256-bin shared histogram each, then the (rank among equal keys)-th lowest index.
// Under the rank law P(i <= 8) = (n+1)/n * 8/9, so the radix path is the exception.
// ---------------------------------------------------------------------------------------
constexpr int kTop = 8;
constexpr int kMaxWarps = 32;

struct SelSmem {
  unsigned long long cand_bits[kMaxWarps][kTop];  // raw bits of r (sign kept)
  int cand_idx[kMaxWarps][kTop];
  double warp_rr[kMaxWarps];
  int hist[256];
  unsigned long long prefix;
  int remaining;
  int res_idx;
  double res_val;
  double rr;
  // per-step scalars, formed by one thread (the FP64 pipe issues two operations a clock per
  // SM: an FP64 scalar repeated by every thread would cost more than the step's vector work)
  double delta;
  int stop;     // 1: the inner stop test holds (or ||r||^2 is not finite)
  int rank;     // rank of the next pick
};

constexpr int kNone = 0x7fffffff;

// warp argmax of (key, index) that carries the raw value bits of the winner along
__device__ __forceinline__ void warp_argmax_v(unsigned long long& a, int& i, unsigned long long& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long oa = __shfl_xor_sync(0xffffffffu, a, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    if (key_greater(oa, oi, a, i)) {
      a = oa;
      i = oi;
      v = ov;
    }
  }
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// i <= kTop.  Leaves the pick in sm.res_idx / sm.res_val (res_idx = -1 if none).  Also
// reduces ||r||^2 (rpart: this thread's partial) into sm.rr.  Two block barriers.
template <int T, int RPT, class Decide>
__device__ void select_fast(const double (&r)[RPT], int n, int i, double rpart, SelSmem& sm, Decide& decide) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int W = T / 32;
  const int rounds = i < kTop ? i : kTop;
  uint32_t taken = 0;
  unsigned long long keep_v = 0ull;
  int keep_i = kNone;
  for (int q = 0; q < rounds; ++q) {
    unsigned long long ba = 0ull, bv = 0ull;
    int bi = kNone;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int s = threadIdx.x + u * T;
      const unsigned long long ka = abs_key(r[u]);
      if (s < n && !(taken & (1u << u)) && key_greater(ka, s, ba, bi)) {
        ba = ka;
        bi = s;
        bv = dbits(r[u]);
      }
    }
    warp_argmax_v(ba, bi, bv);
    if (bi != kNone && (bi % T) == (int)threadIdx.x) taken |= 1u << (bi / T);
    if (lane == q) {
      keep_i = bi;
      keep_v = bv;
    }
  }
  rpart = warp_sum(rpart);
  if (lane < kTop) {
    sm.cand_bits[w][lane] = keep_v;
    sm.cand_idx[w][lane] = lane < rounds ? keep_i : kNone;
  }
  if (lane == 0) sm.warp_rr[w] = rpart;
  __syncthreads();
  if (w == 0) {
    unsigned long long cb[kTop];
    int ci[kTop];
#pragma unroll
    for (int q = 0; q < kTop; ++q) {
      cb[q] = lane < W ? sm.cand_bits[lane][q] : 0ull;
      ci[q] = lane < W ? sm.cand_idx[lane][q] : kNone;
    }
    uint32_t tk = 0;
    int wi = kNone;
    unsigned long long wv = 0ull;
    for (int q = 0; q < i; ++q) {
      unsigned long long ba = 0ull, bv = 0ull;
      int bi = kNone, bslot = 0;
#pragma unroll
      for (int u = 0; u < kTop; ++u) {
        const unsigned long long ka = abs_key(__longlong_as_double((long long)cb[u]));
        if (ci[u] != kNone && !(tk & (1u << u)) && key_greater(ka, ci[u], ba, bi)) {
          ba = ka;
          bi = ci[u];
          bv = cb[u];
          bslot = u;
        }
      }
      const int mine = bi;
      warp_argmax_v(ba, bi, bv);
      if (bi != kNone && bi == mine) tk |= 1u << bslot;  // indices are distinct: one lane owns it
      wi = bi;
      wv = bv;
    }
    double rr = lane < W ? sm.warp_rr[lane] : 0.0;
    rr = warp_sum(rr);
    if (lane == 0) {
      sm.res_idx = wi == kNone ? -1 : wi;
      sm.res_val = __longlong_as_double((long long)wv);
      sm.rr = rr;
      decide(true);
    }
  }
  __syncthreads();
}

// ||r||^2 alone (no pick), into sm.rr by thread 0 (valid for every thread after the next
// barrier the caller places).  One block barrier here.
template <int T>
__device__ void block_sum_sm(double rpart, SelSmem& sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int W = T / 32;
  rpart = warp_sum(rpart);
  if (lane == 0) sm.warp_rr[w] = rpart;
  __syncthreads();
  if (w == 0) {
    double v = lane < W ? sm.warp_rr[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) sm.rr = v;
  }
}

// i > kTop (any i <= number of valid entries): radix selection on the 64-bit keys.  Leaves
// the pick in sm.res_idx / sm.res_val.
template <int T, int RPT, class Decide>
__device__ void select_radix(const double (&r)[RPT], int n, int i, SelSmem& sm, Decide& decide) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int W = T / 32;
  unsigned long long prefix = 0ull, mask = 0ull;
  int rem = i;
  for (int shift = 56; shift >= 0; shift -= 8) {
    __syncthreads();  // the previous pass's histogram has been read
    for (int b = threadIdx.x; b < 256; b += T) sm.hist[b] = 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int s = threadIdx.x + u * T;
      const unsigned long long ka = abs_key(r[u]);
      if (s < n && (ka & mask) == prefix) atomicAdd(&sm.hist[(int)((ka >> shift) & 255ull)], 1);
    }
    __syncthreads();
    if (w == 0) {
      int c[8], tot = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        c[q] = sm.hist[255 - 8 * lane - q];  // lane L: bins 255-8L down to 248-8L
        tot += c[q];
      }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - tot;
      const unsigned ball = __ballot_sync(0xffffffffu, excl < rem && rem <= incl);
      if (ball == 0u) {
        if (lane == 0) {
          sm.remaining = 0;
          sm.prefix = prefix;
        }
      } else if (lane == __ffs(ball) - 1) {
        int acc = excl, digit = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (acc + c[q] >= rem) {
            digit = 255 - 8 * lane - q;
            break;
          }
          acc += c[q];
        }
        sm.prefix = prefix | ((unsigned long long)digit << shift);
        sm.remaining = rem - acc;
      }
    }
    __syncthreads();
    prefix = sm.prefix;
    rem = sm.remaining;
    mask |= 255ull << shift;
    if (rem <= 0) break;
  }
  // the rem-th lowest index among the entries whose key equals prefix
  int last = -1;
  unsigned long long lastv = 0ull;
  for (int q = 0; q < rem; ++q) {
    int best = kNone;
    unsigned long long bv = 0ull;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int s = threadIdx.x + u * T;
      if (s < n && s > last && s < best && abs_key(r[u]) == prefix) {
        best = s;
        bv = dbits(r[u]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int ob = __shfl_xor_sync(0xffffffffu, best, o);
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (ob < best) {
        best = ob;
        bv = ov;
      }
    }
    __syncthreads();
    if (lane == 0) {
      sm.cand_idx[w][0] = best;
      sm.cand_bits[w][0] = bv;
    }
    __syncthreads();
    best = lane < W ? sm.cand_idx[lane][0] : kNone;
    bv = lane < W ? sm.cand_bits[lane][0] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int ob = __shfl_xor_sync(0xffffffffu, best, o);
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (ob < best) {
        best = ob;
        bv = ov;
      }
    }
    if (best == kNone) break;
    last = best;
    lastv = bv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sm.res_idx = (rem > 0 && last >= 0) ? last : -1;
    sm.res_val = __longlong_as_double((long long)lastv);
    decide(false);
  }
  __syncthreads();
}

// The buffer the chain writes: the outer step (sp_iter mode 1) has already made `cur` point
// at x_{k+1}'s buffer; in correction form (mode 2) `cur` still holds x_k, updated in place.
struct ChainIo {
  double* xout;
};

__device__ __forceinline__ ChainIo chain_io(const RandArgs& a, int c) {
  const int cur = *((volatile int32_t*)&a.st->cur);
  ChainIo io;
  io.xout = (cur ? a.X1 : a.X0) + (size_t)c * a.n;
  return io;
}

// ---------------------------------------------------------------------------------------
// SP-SCD inner chain (Alg. 5 steps 5-12) for column blockIdx.x of the pass, r in registers.
// Cold start: beta = 0, r = bhat (step 5); x_{k+1} = beta (step 13), accumulated straight in
// the output buffer.  Correction form (warm start beta = x_k): bhat holds r_k = bbar - H x_k
// = bhat - Abar1 x_k and the steps add to x_k in place.
// ---------------------------------------------------------------------------------------
template <int T, int RPT>
__global__ void __launch_bounds__(T, 1) scd_chain_kernel(RandArgs a) {
  const int c = blockIdx.x;
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done) || a.col_done[c]) return;
  const uint64_t t_start = global_ns();
  const int n = (int)a.n;
  const ChainIo io = chain_io(a, c);
  const uint32_t k = (uint32_t)(st->iters - 1);  // outer index of the iterate being built
  extern __shared__ double idiag[];              // 1 / Abar1_jj = 1 / ||A_1(:,j)||^2
  __shared__ SelSmem sm;
  const double* bhat = a.bhat + (size_t)c * n;
  double r[RPT];
  double part = 0.0;
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int s = threadIdx.x + u * T;
    r[u] = s < n ? bhat[s] : 0.0;
    part = fma(r[u], r[u], part);
    if (s < n) {
      idiag[s] = a.inv_norms2[s];
      if (!a.correction) io.xout[s] = 0.0;  // beta = 0
    }
  }
  const double target2 = a.col_target2[c];
  const bool record = a.picks && c == 0 && k == 0;
  const int alpha = (int)a.alpha_fixed;
  const uint32_t chain = (uint32_t)(a.chain0 + c);
  int64_t t = 0;
  // Rank of the pick of step tt (Alg. 5 steps 7-9 in rank form; thread 0 only).
  auto draw_rank = [&](int64_t tt) -> int {
    if (alpha > 0 && alpha >= n) return 1;
    if (alpha <= 0 && a.greedy) return 1;
    double u0, u1;
    step_uniforms(a.seed, chain, k, (uint64_t)tt, &u0, &u1);
    return alpha > 0 ? scd_fixed_rank(u0, n, alpha) : scd_rank(u0, n);
  };
  // One thread: the stop test on ||r_t||^2, delta = r_j / Abar1_jj (steps 10-11, by the
  // precomputed reciprocal) and the
  // rank of the next step's pick.
  auto decide = [&](bool check_stop) {
    if (check_stop && !(sm.rr > target2)) {
      sm.stop = 1;
      if (!isfinite(sm.rr)) atomicCAS(&st->status, 0, ILS_ERR_NONFINITE);
      return;
    }
    const int j = sm.res_idx;
    if (j < 0) {
      sm.stop = 1;
      atomicCAS(&st->status, 0, ILS_ERR_NONFINITE);
      return;
    }
    sm.stop = 0;
    sm.delta = sm.res_val * idiag[j];
    sm.rank = t + 1 < a.max_inner ? draw_rank(t + 1) : 1;
  };
  if (threadIdx.x == 0) sm.rank = a.max_inner > 0 ? draw_rank(0) : 1;
  __syncthreads();
  for (; t < a.max_inner; ++t) {
    const int i = sm.rank;
    if (i <= kTop) {
      select_fast<T, RPT>(r, n, i, part, sm, decide);
    } else {
      block_sum_sm<T>(part, sm);
      if (threadIdx.x == 0) {
        sm.stop = !(sm.rr > target2) ? 1 : 0;
        if (sm.stop && !isfinite(sm.rr)) atomicCAS(&st->status, 0, ILS_ERR_NONFINITE);
      }
      __syncthreads();
      if (sm.stop) break;
      select_radix<T, RPT>(r, n, i, sm, decide);
    }
    if (sm.stop) break;
    const int j = sm.res_idx;
    const double delta = sm.delta;
    if (threadIdx.x == (unsigned)(j % T)) io.xout[j] += delta;
    if (record && threadIdx.x == 0 && t < a.picks_cap) a.picks[t] = j;
    const double* gj = a.G1 + (size_t)j * n;
    part = 0.0;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int s = threadIdx.x + u * T;
      if (s < n) r[u] = fma(-delta, __ldg(gj + s), r[u]);
      part = fma(r[u], r[u], part);
    }
  }
  if (threadIdx.x == 0) {
    a.col_inner[c] += t;
    if (a.inner_ns && c == 0) atomicAdd(a.inner_ns, (unsigned long long)(global_ns() - t_start));
  }
}

constexpr int kChainThreads = 512;
constexpr int kChainWarps = kChainThreads / 32;

// Block-wide sum, result broadcast to every thread.  red has kChainWarps + 1 slots.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // red may still be read from the previous call
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < kChainWarps ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[kChainWarps] = t;
  }
  __syncthreads();
  return red[kChainWarps];
}

__device__ __forceinline__ void draw_columns(const RandArgs& a, const double* cum, const double* aprob,
                                             const int32_t* aidx, int n, uint32_t chain, uint32_t k, int64_t t,
                                             int* j1, int* j2) {
  double u0, u1;
  step_uniforms(a.seed, chain, k, (uint64_t)t, &u0, &u1);
  if (a.alias) {
    *j1 = alias_pick(aprob, aidx, n, u0);
    *j2 = a.same_index ? *j1 : alias_pick(aprob, aidx, n, u1);
  } else {
    *j1 = invcdf_pick(cum, n, u0);
    *j2 = a.same_index ? *j1 : invcdf_pick(cum, n, u1);
  }
}

// ---------------------------------------------------------------------------------------
// SP-RK-RGS inner chain, column form (Alg. 2 steps 6-12) for column blockIdx.x of the pass.
// w (length p) and the maintained e = w - A_1 z live in shared memory when they fit,
// otherwise in a global scratch slice of the chain.  The RGS step reads A_1^T (w - A_1 z)
// restricted to column j2, which is A_1(:,j2)^T e.  In correction form bhat holds
// r_k = bbar - H x_k, the chain solves Abar1 d = r_k from 0 and adds d to x_k in place.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kChainThreads) rkrgs_chain_kernel(RandArgs a) {
  const int c = blockIdx.x;
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done) || a.col_done[c]) return;
  const uint64_t t_start = global_ns();
  const int n = (int)a.n;
  const int64_t p = a.p, m = a.m;
  const ChainIo io = chain_io(a, c);
  const uint32_t k = (uint32_t)(st->iters - 1);
  extern __shared__ double smem[];
  double* z = smem;             // n
  double* cum = smem + n;       // n (inverse CDF) or the alias table (n doubles + n ints)
  double* aprob = cum;
  int32_t* aidx = reinterpret_cast<int32_t*>(smem + 2 * n);
  const int vec0 = a.alias ? 2 * n + (n + 1) / 2 : 2 * n;
  double* w;
  double* e;
  if (a.vec_in_smem) {
    w = smem + vec0;
    e = w + p;
  } else {
    w = a.vec_scratch + (size_t)c * 2 * p;
    e = w + p;
  }
  __shared__ double red[kChainWarps + 1];
  __shared__ int draw[2];
  __shared__ double coef;
  __shared__ int stop_flag;
  const double* bhat = a.bhat + (size_t)c * n;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    z[s] = 0.0;
    if (a.alias) {
      aprob[s] = a.alias_prob[s];
      aidx[s] = a.alias_idx[s];
    } else {
      cum[s] = a.cum[s];
    }
  }
  for (int64_t r = threadIdx.x; r < p; r += blockDim.x) {
    w[r] = 0.0;
    e[r] = 0.0;
  }
  __syncthreads();
  const double target2 = a.col_target2[c];
  const int64_t check = a.check_every;
  const bool record = a.picks && c == 0 && k == 0;
  const uint32_t chain = (uint32_t)(a.chain0 + c);
  // Block sum of the threads' shares; thread 0 then forms the step's scalar from it.
  auto reduce0 = [&](double v) -> double {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) red[wp] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
      for (int i = 0; i < kChainWarps; ++i) tot += red[i];
    return tot;  // thread 0 only
  };
  int64_t t = 0;
  bool stop = false;
  for (; t < a.max_inner && !stop; ++t) {
    if (threadIdx.x == 0) {
      draw_columns(a, cum, aprob, aidx, n, chain, k, t, &draw[0], &draw[1]);
      if (record && 2 * t + 1 < a.picks_cap) {
        a.picks[2 * t] = draw[0];
        a.picks[2 * t + 1] = draw[1];
      }
    }
    __syncthreads();
    const int j1 = draw[0], j2 = draw[1];
    // RK step on A_1^T w = bhat (step 9).
    const double* a1 = a.A + (size_t)j1 * m;
    double part = 0.0;
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) part = fma(a1[r], w[r], part);
    const double dot1 = reduce0(part);
    if (threadIdx.x == 0) coef = (bhat[j1] - dot1) / a.norms2[j1];
    __syncthreads();
    const double delta = coef;
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) {
      const double av = a1[r];
      w[r] = fma(delta, av, w[r]);
      e[r] = fma(delta, av, e[r]);
    }
    // RGS step on A_1 z = w with the updated w (step 11).
    const double* a2 = a.A + (size_t)j2 * m;
    part = 0.0;
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) part = fma(a2[r], e[r], part);
    const double dot2 = reduce0(part);
    if (threadIdx.x == 0) {
      coef = dot2 / a.norms2[j2];
      z[j2] += coef;
    }
    __syncthreads();
    const double eps = coef;
    for (int64_t r = threadIdx.x; r < p; r += blockDim.x) e[r] = fma(-eps, a2[r], e[r]);
    if ((t + 1) % check == 0) {
      // Inner stop test: ||bhat - Abar1 z||^2 <= target2.
      part = 0.0;
      for (int row = threadIdx.x; row < n; row += blockDim.x) {
        const double* g = a.G1 + (size_t)row * n;  // column `row` = row `row` (symmetric)
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = fma(g[j], z[j], acc);
        const double rv = bhat[row] - acc;
        part = fma(rv, rv, part);
      }
      const double res2 = reduce0(part);
      if (threadIdx.x == 0) stop_flag = res2 <= target2 ? 1 : 0;
      __syncthreads();
      stop = stop_flag != 0;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    if (a.correction) io.xout[s] += z[s];  // x_k + d
    else io.xout[s] = z[s];                // x_{k+1} = z (step 13)
  }
  if (threadIdx.x == 0) {
    a.col_inner[c] += t;
    if (a.inner_ns && c == 0) atomicAdd(a.inner_ns, (unsigned long long)(global_ns() - t_start));
  }
}

// ---------------------------------------------------------------------------------------
// SP-RK-RGS inner chain in Gram form (not in the paper): w = A_1 y is carried as g = Abar1 y
// and A_1 z as h = Abar1 z, both in registers, so a step applies two columns of Abar1
// (O(n)) instead of two columns of A_1 and two p-vectors (O(p)):
//   delta = (bhat_j1 - g_j1) / Abar1_{j1 j1};  g += delta Abar1(:, j1)          (step 9)
//   eps   = (g_j2 - h_j2) / Abar1_{j2 j2};     z_j2 += eps;  h += eps Abar1(:, j2)  (step 11)
// The same draws give the column form's iterates in exact arithmetic.  z accumulates in
// the output buffer (x_k itself in correction form).  The inner stop reads ||bhat - h||.
// ---------------------------------------------------------------------------------------
template <int T, int RPT>
__global__ void __launch_bounds__(T, 1) rkrgs_gram_chain_kernel(RandArgs a) {
  const int c = blockIdx.x;
  SolveState* st = a.st;
  if (*((volatile int32_t*)&st->done) || a.col_done[c]) return;
  const uint64_t t_start = global_ns();
  const int n = (int)a.n;
  const ChainIo io = chain_io(a, c);
  const uint32_t k = (uint32_t)(st->iters - 1);
  extern __shared__ double gsm[];
  double* idiag = gsm;         // n: 1 / Abar1_jj
  double* cum = gsm + n;       // n, or the alias table (n doubles + n ints)
  double* aprob = cum;
  int32_t* aidx = reinterpret_cast<int32_t*>(gsm + 2 * n);
  __shared__ double slot[2];
  __shared__ int draw[2][2];   // (j1, j2) of the current and the next step, by parity
  __shared__ SelSmem sm;
  const double* bhat = a.bhat + (size_t)c * n;
  double bh[RPT], g[RPT], h[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int s = threadIdx.x + u * T;
    bh[u] = s < n ? bhat[s] : 0.0;
    g[u] = 0.0;
    h[u] = 0.0;
    if (s < n) {
      idiag[s] = a.inv_norms2[s];
      if (a.alias) {
        aprob[s] = a.alias_prob[s];
        aidx[s] = a.alias_idx[s];
      } else {
        cum[s] = a.cum[s];
      }
      if (!a.correction) io.xout[s] = 0.0;  // z = 0
    }
  }
  __syncthreads();
  const double target2 = a.col_target2[c];
  const int64_t check = a.check_every;
  const bool record = a.picks && c == 0 && k == 0;
  const uint32_t chain = (uint32_t)(a.chain0 + c);
  if (threadIdx.x == 0 && a.max_inner > 0) draw_columns(a, cum, aprob, aidx, n, chain, k, 0, &draw[0][0], &draw[0][1]);
  __syncthreads();
  // The columns of Abar1 a step applies depend only on its draws, which are made a step
  // ahead: each step loads the next step's two columns while it works on its own.
  double c1[RPT], c2[RPT], n1[RPT], n2[RPT];
  if (a.max_inner > 0) {
    const double* p1 = a.G1 + (size_t)draw[0][0] * n;
    const double* p2 = a.G1 + (size_t)draw[0][1] * n;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int s = threadIdx.x + u * T;
      c1[u] = s < n ? __ldg(p1 + s) : 0.0;
      c2[u] = s < n ? __ldg(p2 + s) : 0.0;
    }
  }
  int64_t t = 0;
  for (; t < a.max_inner; ++t) {
    const int par = (int)(t & 1);
    const int j1 = draw[par][0], j2 = draw[par][1];
    if (threadIdx.x == 0) {
      if (record && 2 * t + 1 < a.picks_cap) {
        a.picks[2 * t] = j1;
        a.picks[2 * t + 1] = j2;
      }
      if (t + 1 < a.max_inner) draw_columns(a, cum, aprob, aidx, n, chain, k, t + 1, &draw[par ^ 1][0], &draw[par ^ 1][1]);
    }
    if (threadIdx.x == (unsigned)(j1 % T)) {
#pragma unroll
      for (int u = 0; u < RPT; ++u)
        if (u == j1 / T) slot[0] = (bh[u] - g[u]) * idiag[j1];  // delta (step 9)
    }
    __syncthreads();
    const double delta = slot[0];
    if (t + 1 < a.max_inner) {  // the next step's columns (its draws are in place now)
      const double* p1 = a.G1 + (size_t)draw[par ^ 1][0] * n;
      const double* p2 = a.G1 + (size_t)draw[par ^ 1][1] * n;
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const int s = threadIdx.x + u * T;
        n1[u] = s < n ? __ldg(p1 + s) : 0.0;
        n2[u] = s < n ? __ldg(p2 + s) : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) g[u] = fma(delta, c1[u], g[u]);
    if (threadIdx.x == (unsigned)(j2 % T)) {
#pragma unroll
      for (int u = 0; u < RPT; ++u)
        if (u == j2 / T) {
          const double eps = (g[u] - h[u]) * idiag[j2];  // step 11
          slot[1] = eps;
          io.xout[j2] += eps;
        }
    }
    __syncthreads();
    const double eps = slot[1];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      h[u] = fma(eps, c2[u], h[u]);
      c1[u] = n1[u];
      c2[u] = n2[u];
    }
    if ((t + 1) % check == 0) {
      double part = 0.0;
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const double rv = bh[u] - h[u];
        part = fma(rv, rv, part);
      }
      block_sum_sm<T>(part, sm);
      if (threadIdx.x == 0) sm.stop = sm.rr <= target2 ? 1 : 0;
      __syncthreads();
      if (sm.stop) {
        ++t;
        break;
      }
    }
  }
  if (threadIdx.x == 0) {
    a.col_inner[c] += t;
    if (a.inner_ns && c == 0) atomicAdd(a.inner_ns, (unsigned long long)(global_ns() - t_start));
  }
}

// Vose's alias method (M. D. Vose, IEEE TSE 17(9), 1991) for the law norms2 / sum(norms2):
// q_j = n norms2_j / total; columns with q < 1 are paired with one with q >= 1, which gives
// up 1 - q_l of its mass ((q_g + q_l) - 1 keeps the arithmetic stable).  The construction
// is sequential (one thread) on shared memory; the draw is alias_pick above.
__global__ void alias_table_kernel(int n, const double* __restrict__ norms2, double* __restrict__ prob,
                                   int32_t* __restrict__ alias) {
  extern __shared__ double q[];                           // n
  int32_t* lists = reinterpret_cast<int32_t*>(q + n);     // small from the front, large from the back
  __shared__ double red[kMaxWarps];
  double part = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) part += norms2[j];
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double total = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += red[w];
  int ns = 0, nl = 0;
  for (int j = 0; j < n; ++j) {
    q[j] = (double)n * norms2[j] / total;
    if (q[j] < 1.0) lists[ns++] = j;
    else lists[n - 1 - nl++] = j;
  }
  while (ns > 0 && nl > 0) {
    const int l = lists[--ns];
    const int g = lists[n - nl];  // top of the large list
    prob[l] = q[l];
    alias[l] = g;
    q[g] = (q[g] + q[l]) - 1.0;
    if (q[g] < 1.0) {
      --nl;
      lists[ns++] = g;
    }
  }
  for (int i = 0; i < ns; ++i) {
    prob[lists[i]] = 1.0;
    alias[lists[i]] = lists[i];
  }
  for (int i = 0; i < nl; ++i) {
    prob[lists[n - 1 - i]] = 1.0;
    alias[lists[n - 1 - i]] = lists[n - 1 - i];
  }
}

// cum[j] = sum_{i <= j} norms2[i], added left to right; norms2 = diag(Abar1).  The
// diagonal is gathered in parallel; one thread then adds it in order, 32 loads at a time.
__global__ void column_cumsum_kernel(int64_t n, const double* G1, double* norms2, double* cum, double* inv_norms2) {
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = G1[j + j * n];
    norms2[j] = d;
    if (inv_norms2) inv_norms2[j] = 1.0 / d;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    double v[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = (j0 + t < n) ? norms2[j0 + t] : 0.0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (j0 + t < n) {
        s += v[t];
        cum[j0 + t] = s;
      }
    }
  }
}

template <class K>
cudaError_t launch_chain(K kernel, unsigned grid, unsigned threads, size_t smem, const RandArgs& a, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kernel<<<grid, threads, smem, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t alias_table_f64(int64_t n, const double* norms2, double* prob, int32_t* alias, cudaStream_t s) {
  const size_t smem = (size_t)n * (sizeof(double) + sizeof(int32_t));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(alias_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  alias_table_kernel<<<1, 256, smem, s>>>((int)n, norms2, prob, alias);
  note_launch();
  return cudaGetLastError();
}

cudaError_t column_cumsum_f64(int64_t n, const double* G1, double* norms2, double* cum, cudaStream_t s,
                              double* inv_norms2) {
  column_cumsum_kernel<<<1, 256, 0, s>>>(n, G1, norms2, cum, inv_norms2);
  note_launch();
  return cudaGetLastError();
}

size_t rkrgs_smem_bytes(int64_t n, int64_t p, bool vec_in_smem) {
  // z, the sampling table (cum, or the alias table's n doubles + n ints), and w, e
  return sizeof(double) * (size_t)(2 * n + (n + 1) / 2 + (vec_in_smem ? 2 * p : 0));
}

bool rkrgs_vec_fits(int64_t n, int64_t p) { return rkrgs_smem_bytes(n, p, true) <= 200 * 1024; }

// Register layouts: about eight entries of each vector per thread.  The FP64 pipe issues two
// operations a clock per SM, so every warp-wide FP64 reduction costs 80 clocks of it; fewer,
// fuller threads keep the per-step reductions cheap while the entry-wise work stays n.
cudaError_t rand_chain_f64(const RandArgs& a, int method, cudaStream_t s) {
  const unsigned grid = (unsigned)a.k;
  const int64_t n = a.n;
  if (method == ILS_SP_SCD) {
    const size_t smem = sizeof(double) * (size_t)n;
    if (n <= 256) return launch_chain(scd_chain_kernel<256, 1>, grid, 256, smem, a, s);
    if (n <= 512) return launch_chain(scd_chain_kernel<256, 2>, grid, 256, smem, a, s);
    if (n <= 1024) return launch_chain(scd_chain_kernel<256, 4>, grid, 256, smem, a, s);
    if (n <= 2048) return launch_chain(scd_chain_kernel<256, 8>, grid, 256, smem, a, s);
    if (n <= 4096) return launch_chain(scd_chain_kernel<512, 8>, grid, 512, smem, a, s);
    if (n <= 8192) return launch_chain(scd_chain_kernel<512, 16>, grid, 512, smem, a, s);
    if (n <= 16384) return launch_chain(scd_chain_kernel<512, 32>, grid, 512, smem, a, s);
    return cudaErrorInvalidValue;
  }
  if (a.gram_form) {
    const size_t smem = sizeof(double) * (size_t)(2 * n + (n + 1) / 2);
    if (n <= 256) return launch_chain(rkrgs_gram_chain_kernel<256, 1>, grid, 256, smem, a, s);
    if (n <= 512) return launch_chain(rkrgs_gram_chain_kernel<256, 2>, grid, 256, smem, a, s);
    if (n <= 1024) return launch_chain(rkrgs_gram_chain_kernel<256, 4>, grid, 256, smem, a, s);
    if (n <= 2048) return launch_chain(rkrgs_gram_chain_kernel<256, 8>, grid, 256, smem, a, s);
    if (n <= 4096) return launch_chain(rkrgs_gram_chain_kernel<512, 8>, grid, 512, smem, a, s);
    if (n <= 8192) return launch_chain(rkrgs_gram_chain_kernel<512, 16>, grid, 512, smem, a, s);
    return cudaErrorInvalidValue;
  }
  const size_t smem = rkrgs_smem_bytes(a.n, a.p, a.vec_in_smem != 0);
  return launch_chain(rkrgs_chain_kernel, grid, kChainThreads, smem, a, s);
}

}  // namespace ils
