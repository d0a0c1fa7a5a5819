// FP64-accurate Gram matrix A^T A on the tcgen05 tensor cores.
//
// GB300 issues FP64 fused multiply-adds at about 2 per clock per SM, while its BF16
// tensor cores are three orders of magnitude faster.  The Gram products of Alg. 1 step 2
// (Abar1 = A_1^T A_1) and step 3 (Abar2 = A_2^T A_2) are therefore formed from exact
// integer slice products:
//
//   1. Column j of A is scaled by 2^-e_j so that its entries lie in (-1/2, 1/2).
//   2. Each scaled entry is rounded to a multiple of 2^(-beta S) (beta = 6, S = 9: 53 bits
//      below the column's largest entry) and written in S balanced digits,
//      a = sum_{t=1..S} 2^{-beta t} d_t with |d_t| <= 2^(beta-1) = 32; every digit is exact
//      in BF16.  Rounding (not truncation) leaves the digits' signs independent of the
//      entry's sign, so the split and the omitted pairs add unbiased errors, and the error
//      of the split is at most 2^{-beta S - 1} times the column scale.
//   3. For every ordered pair (t, u) with t + u <= S + 1 (45 pairs) the tensor cores form
//      D_t^T D_u with FP32 accumulation over K chunks of at most 16384 rows.  All partial
//      sums are integers of magnitude at most 16384 * 32^2 = 2^24, so the FP32
//      accumulation is exact.  On the diagonal tiles of the Gram, D_u^T D_t is the
//      transpose of D_t^T D_u: it is not formed, the epilogue stores the transpose in its
//      place.
//   4. The epilogue stores each exact product as it stands (FP32).  A reduction adds the
//      products of equal t + u exactly as 64-bit integers, joins the 9 group sums (weight
//      2^{e_i + e_j - beta (t + u)}) in exact integer parts and the parts in FP64 with at
//      most two roundings, in a fixed order (deterministic).
//
// The tcgen05 kernel is warp-specialised: warp 0 issues TMA loads of 128 x 64 BF16 tiles
// (128B swizzle) of up to four digit slices into a 3-stage shared-memory ring, warp 1
// issues 128x128x16 MMAs of up to four digit pairs into four TMEM accumulators, warps 2-5
// drain TMEM.  Every mbarrier wait is bounded; on a timeout the kernel records an error
// flag, stops issuing work, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "ils_internal.h"

namespace ils {
namespace {

constexpr int kBeta = 6;        // bits per slice
constexpr int kSlices = 9;      // 54 bits below the column scale (53 below its largest entry)
constexpr int kBM = 128;        // output tile rows (columns of D_t)
constexpr int kBN = 128;        // output tile cols (columns of D_u)
constexpr int kBK = 64;         // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int kStages = 3;
constexpr int kKChunk = 16384;  // K rows per product at most: 16384 * 32^2 = 2^24 (exact FP32 sums)
constexpr int kThreads = 192;   // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint32_t kTileBytes = kBM * kBK * 2;  // 16 KB per operand tile
constexpr uint32_t kStageBytes = 4 * kTileBytes;  // up to four digit tiles per stage
constexpr uint64_t kWaitNs = 4000000000ull;  // bound on any mbarrier wait (4 s)

// ------------------------------- device helpers ----------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Poll an mbarrier phase for at most kWaitNs of wall time.  Returns false on timeout.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzle
// layout: 8-row x 128-byte atoms stacked every 1024 bytes (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);      // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptors: kind::f16 with BF16 A/B, FP32 D, both K-major, M = 128 and
// N = 128 or 256 (N = 256: two adjacent 128-row B tiles, i.e. two digit products that
// share their A tile, in one instruction).
constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_bf16(kBN);
constexpr uint32_t kIdesc2 = idesc_bf16(2 * kBN);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct SplitParams {
  int n;            // Gram order (columns of X)
  int n2;           // columns of Y (general product X^T Y); n for the Gram
  int K;            // rows of A (reduction length)
  int n_tiles;      // ceil(n / 128)
  int n_tiles2;     // ceil(n2 / 128)
  int n_kchunks;
  int kchunk;       // K rows per chunk (a multiple of 64, at most kKChunk)
  // Gram launches hand out their items heaviest first: the groups of each MMA cost
  // (1-4 N=128 units), diagonal (gd_*) and off-diagonal (go_*) tile pairs
  int8_t nd_c[5], no_c[5];       // groups of cost c
  int8_t gd_order[32], go_order[32];  // group ids, by cost from 4 down to 1
  const int* exps;  // per-column exponents e_j of X (device)
  const int* exps2; // of Y
  double* partial;  // [tile][product slot][K chunk][128][128] exact products, FP32 bit patterns
  int32_t* err;     // device error flag
};

// Work groups.  The digit pairs (t, u) with t + u <= S + 1 are taken in 2 x 2 blocks
// (a, b): t in {2a-1, 2a}, u in {2b-1, 2b}, a + b <= S/2 + 1.  A CTA loads the (up to)
// four digit tiles of its block once per K step and forms the block's (up to) four
// products into four TMEM accumulators: one tile load per product instead of 1.5 for
// pairs sharing only the A tile.  On a diagonal tile pair (bi = bj) the product (u, t) is
// the transpose of (t, u), so only blocks with a <= b are formed, and inside a block
// with a = b only t <= u (its two tiles serve as both operands); the epilogue stores each
// cross product a second time, transposed, as the product (u, t).
constexpr int kHalf = (kSlices + 1) / 2;  // the last block holds digit S alone when S is odd
constexpr int kMaxTiles = 4;
constexpr int kMaxProd = 4;

struct GroupDesc {
  int ntiles, nprod;
  int digit[kMaxTiles];  // 1-based digit of each loaded tile
  int side[kMaxTiles];   // 0: columns of tile bi, 1: columns of tile bj
  int ia[kMaxProd], ib[kMaxProd];  // loaded-tile index of each product's A and B operand
  int t[kMaxProd], u[kMaxProd];
  int tcol[kMaxProd];    // TMEM accumulator of each product: 2 i + j for A tile i, B tile b0 + j
  int jmask[2];          // per A tile i: bit j set when the product (i, j) is formed
  int b0;                // loaded-tile index of the first B tile (the second follows it)
  int slot0;             // product slot (within the tile) of the group's first product
};

__host__ __device__ inline bool block_valid(bool diag, int a, int b) {
  return a + b <= kHalf + 1 && (!diag || a <= b);
}

// Group g of a diagonal (diag) or off-diagonal tile pair, in row-major order of (a, b).
__host__ __device__ inline void block_desc(bool diag, int g, GroupDesc& d) {
  int slot = 0;
  for (int a = 1; a <= kHalf; ++a) {
    for (int b = 1; b <= kHalf; ++b) {
      if (!block_valid(diag, a, b)) continue;
      GroupDesc cur = {};
      cur.slot0 = slot;
      const bool same = diag && a == b;
      // stage slots 0, 1: digits 2a-1, 2a (A side); 2, 3: digits 2b-1, 2b (B side); a digit
      // past S (the odd last block) is 0: its slot is not loaded
      cur.ntiles = same ? 2 : 4;
      cur.digit[0] = 2 * a - 1;
      cur.digit[1] = 2 * a <= kSlices ? 2 * a : 0;
      cur.side[0] = cur.side[1] = 0;
      if (!same) {
        cur.digit[2] = 2 * b - 1;
        cur.digit[3] = 2 * b <= kSlices ? 2 * b : 0;
        cur.side[2] = cur.side[3] = 1;
      }
      cur.nprod = 0;
      cur.b0 = same ? 0 : 2;
      for (int i = 0; i < 2; ++i) {
        cur.jmask[i] = 0;
        for (int j = 0; j < 2; ++j) {
          const int t = 2 * a - 1 + i, u = 2 * b - 1 + j;
          if (t > kSlices || u > kSlices || t + u > kSlices + 1 || (same && t > u)) continue;
          cur.ia[cur.nprod] = i;
          cur.ib[cur.nprod] = cur.b0 + j;
          cur.t[cur.nprod] = t;
          cur.u[cur.nprod] = u;
          cur.tcol[cur.nprod] = 2 * i + j;
          cur.jmask[i] |= 1 << j;
          ++cur.nprod;
        }
      }
      if (g == 0) {
        d = cur;
        return;
      }
      --g;
      slot += cur.nprod;
    }
  }
}

__host__ __device__ inline int num_blocks(bool diag) {
  int c = 0;
  for (int a = 1; a <= kHalf; ++a)
    for (int b = 1; b <= kHalf; ++b) c += block_valid(diag, a, b) ? 1 : 0;
  return c;
}

// Product slots per tile: one per ordered pair (t, u) with t + u <= S + 1.
__host__ __device__ constexpr int slots_per_tile() {
  int c = 0;
  for (int t = 1; t <= kSlices; ++t) c += kSlices + 1 - t;
  return c;
}

// Slot of the ordered pair (t, u) (by t, then u).
__host__ __device__ inline int pair_slot(int t, int u) {
  int p = 0;
  for (int tt = 1; tt < t; ++tt) p += kSlices + 1 - tt;
  return p + (u - 1);
}

// MMA cost of a group in N = 128 units: per A tile, 2 for an N = 256 pair, 1 for one product.
__host__ __device__ inline int group_cost(bool diag, int g) {
  GroupDesc d;
  block_desc(diag, g, d);
  int c = 0;
  for (int i = 0; i < 2; ++i) c += d.jmask[i] == 3 ? 2 : (d.jmask[i] ? 1 : 0);
  return c;
}

// Work item -> (K chunk, upper tile pair, group), heaviest groups first (the block
// scheduler hands out blocks in order, so the light ones fill in at the end).  Within a
// cost class: K chunk, then the diagonal tile pairs, then the off-diagonal ones (row-major,
// bi < bj), each with its groups of that cost.
__device__ __forceinline__ void decode_item(int item, const SplitParams& P, int* bi, int* bj, int* g, int* kc,
                                            int* tile_out) {
  const int n_off = P.n_tiles * (P.n_tiles - 1) / 2;
  int rest = item, od = 0, oo = 0;
  int c = 4;
  for (; c >= 1; --c) {
    const int per_kc = P.n_tiles * P.nd_c[c] + n_off * P.no_c[c];
    if (rest < per_kc * P.n_kchunks) break;
    rest -= per_kc * P.n_kchunks;
    od += P.nd_c[c];
    oo += P.no_c[c];
  }
  const int per_kc = P.n_tiles * P.nd_c[c] + n_off * P.no_c[c];
  *kc = rest / per_kc;
  rest %= per_kc;
  if (rest < P.n_tiles * P.nd_c[c]) {
    *bi = *bj = rest / P.nd_c[c];
    *g = P.gd_order[od + rest % P.nd_c[c]];
  } else {
    rest -= P.n_tiles * P.nd_c[c];
    int off = rest / P.no_c[c];
    *g = P.go_order[oo + rest % P.no_c[c]];
    int r = 0;
    while (off >= P.n_tiles - r - 1) {
      off -= P.n_tiles - r - 1;
      ++r;
    }
    *bi = r;
    *bj = r + 1 + off;
  }
  // upper tile pairs row-major (bi <= bj)
  *tile_out = *bi * P.n_tiles - *bi * (*bi - 1) / 2 + (*bj - *bi);
}

// General product X^T Y: item -> (K chunk, tile pair (bi, bj) row-major over n_tiles x
// n_tiles2, group); every tile pair takes all ordered digit pairs.
__device__ __forceinline__ void decode_item_gen(int item, const SplitParams& P, int* bi, int* bj, int* g, int* kc,
                                                int* tile_out) {
  const int no = num_blocks(false);
  const int per_chunk = P.n_tiles * P.n_tiles2 * no;
  *kc = item / per_chunk;
  const int rest = item % per_chunk;
  const int tile = rest / no;
  *g = rest % no;
  *bi = tile / P.n_tiles2;
  *bj = tile % P.n_tiles2;
  *tile_out = tile;
}

// SYM: the Gram X^T X (upper tile pairs, transposed cross products on diagonal tiles);
// otherwise X^T Y with X's digits from tmap and Y's from tmap2.  A SYM launch may carry two
// Grams: blocks [0, items0) form the first (tmap, P0), the rest the second (tmap2, P1), so
// that the second fills the SMs the first leaves idle.
template <bool SYM>
__global__ void __launch_bounds__(kThreads, 1)
gram_split_mma_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap2,
                      SplitParams P0, SplitParams P1, int items0) {
  const bool second = SYM && (int)blockIdx.x >= items0;
  const SplitParams P = second ? P1 : P0;
  const int item = second ? (int)blockIdx.x - items0 : (int)blockIdx.x;
  const CUtensorMap* mapA = second ? &tmap2 : &tmap;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* tiles = smem;  // kStages x (up to kMaxTiles digit tiles)
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int bi, bj, g, kc, tile;
  if (SYM) decode_item(item, P, &bi, &bj, &g, &kc, &tile);
  else decode_item_gen(item, P, &bi, &bj, &g, &kc, &tile);
  const bool diag = SYM && bi == bj;
  GroupDesc gd;
  block_desc(diag, g, gd);
  const int k_begin = kc * P.kchunk;
  const int k_end = min(P.K, k_begin + P.kchunk);
  const int nk = (k_end - k_begin + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kMaxProd * kBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_acc = *tmem_slot;

  int issued = 0;  // stages handed to TMA by the producer
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int trow[kMaxTiles], tdig[kMaxTiles];
#pragma unroll
    for (int i = 0; i < kMaxTiles; ++i) {
      trow[i] = (gd.side[i] ? bj : bi) * kBM;
      tdig[i] = gd.digit[i] - 1;
    }
    const int ntiles = gd.ntiles;
    int loaded = 0;  // tiles of existing digits (a digit past S is 0: not loaded, never read)
    for (int i = 0; i < ntiles; ++i) loaded += gd.digit[i] != 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        atomicExch(P.err, 1);
        s_abort = 1;
        break;
      }
      if (*((volatile int*)&s_abort)) break;
      uint8_t* stage = tiles + (size_t)s * kStageBytes;
      mbar_expect_tx(&full[s], (uint32_t)loaded * kTileBytes);
      const int k = k_begin + kb * kBK;
#pragma unroll
      for (int i = 0; i < kMaxTiles; ++i)
        if (i < ntiles && gd.digit[i] != 0)
          tma_load_3d(stage + i * kTileBytes, SYM ? mapA : (gd.side[i] == 0 ? &tmap : &tmap2), &full[s], k,
                      trow[i], tdig[i]);
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // Per A tile i: both products -> one N = 256 MMA over B tiles b0, b0 + 1 into
    // accumulators 2i, 2i + 1; one product (i, j) -> an N = 128 MMA into accumulator 2i + j.
    const uint32_t boff0 = (uint32_t)gd.b0 * kTileBytes;
    const int jm0 = gd.jmask[0], jm1 = gd.jmask[1];
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        atomicExch(P.err, 1);
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st_addr = smem_u32(tiles + (size_t)s * kStageBytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
        for (int i = 0; i < 2; ++i) {  // A tile i: accumulators 2i (TMEM columns 2i kBN ..), 2i + 1
          const int jm = i == 0 ? jm0 : jm1;
          const uint64_t adesc = smem_desc_sw128(st_addr + (uint32_t)i * kTileBytes + kk * 32);
          if (jm == 3)
            mma_bf16(tmem_acc + (uint32_t)(2 * i * kBN), adesc, smem_desc_sw128(st_addr + boff0 + kk * 32), kIdesc2,
                     acc);
          else if (jm)
            mma_bf16(tmem_acc + (uint32_t)((2 * i + (jm >> 1)) * kBN), adesc,
                     smem_desc_sw128(st_addr + boff0 + (uint32_t)(jm >> 1) * kTileBytes + kk * 32), kIdesc, acc);
        }
      }
      mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
    }
    mma_commit(acc_full);  // arrives when every MMA issued above has completed
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> partial products (exact FP32) ----------------
    const bool ok = mbar_wait(acc_full, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp & 3;  // this warp may read TMEM lanes 32q .. 32q+31
    const int row = q * 32 + lane;
    if (!ok) {
      atomicExch(P.err, 1);
    } else if (!*((volatile int*)&s_abort)) {
      const int nslots = slots_per_tile();
      uint32_t* part = reinterpret_cast<uint32_t*>(P.partial);
      for (int p = 0; p < gd.nprod; ++p) {
        const int t = gd.t[p], u = gd.u[p];
        const size_t tile_elems = (size_t)kBM * kBN;
        // The exact integer products stay FP32 bit patterns; the reduction scales them.
        uint32_t* out = part + ((size_t)(tile * nslots + pair_slot(t, u)) * P.n_kchunks + kc) * tile_elems;
        // On a diagonal tile a cross product also stands for (u, t): its transpose goes to
        // that slot, 32 consecutive entries per thread.
        uint32_t* out_t = (diag && t != u)
                              ? part + ((size_t)(tile * nslots + pair_slot(u, t)) * P.n_kchunks + kc) * tile_elems
                              : nullptr;
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 32) {
          uint32_t v[32];
          tmem_ld_32x32b_x32(tmem_acc + ((uint32_t)(q * 32) << 16) + (uint32_t)(gd.tcol[p] * kBN + c0), v);
#pragma unroll
          for (int c = 0; c < 32; ++c) out[(size_t)(c0 + c) * kBM + row] = v[c];  // column-major 128 x 128
          if (out_t) {
            uint4* dst = reinterpret_cast<uint4*>(out_t + (size_t)row * kBM + c0);
#pragma unroll
            for (int c = 0; c < 32; c += 4) dst[c / 4] = make_uint4(v[c], v[c + 1], v[c + 2], v[c + 3]);
          }
        }
      }
    }
  }
  // Producer: on an abort, wait (bounded) for the copies it issued before leaving.
  if (warp == 0 && lane == 0 && *((volatile int*)&s_abort)) {
    for (int kb = 0; kb < issued; ++kb) mbar_wait(&full[kb % kStages], (uint32_t)(kb / kStages) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_acc), "r"(kMaxProd * kBN));
  }
}

__device__ __forceinline__ int exponent_of_field(int m) {
  // A normal value with exponent field f lies in [2^(f-1023), 2^(f-1022)): with e = f - 1021
  // the column scaled by 2^-e lies in (-1/2, 1/2), which keeps the top digit within 32.
  return (m == 0 || m == 0x7FF) ? 0 : m - 1021;
}

// Per-column exponent e_j with max_r |A(r,j)| < 2^(e_j - 1) (0 for a zero column), read from the
// exponent fields of the FP64 bit patterns (integer work only).
__global__ void column_exponent_kernel(int K, int n, const double* __restrict__ A, int64_t lda, int* __restrict__ exps) {
  const int j = blockIdx.x;
  int mx = 0;
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    const long long bits = __double_as_longlong(A[r + (int64_t)j * lda]);
    mx = max(mx, (int)((bits >> 52) & 0x7FF));
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    exps[j] = exponent_of_field(m);
  }
}

// Digits of column j: D[t][j][r] (K-contiguous, leading dimension ldk).  The scaled entry
// a 2^-e_j is rounded to the 50-bit fixed-point integer V = rint(a 2^(50 - e_j)) straight
// from its bit pattern, and V is written in balanced base 32: five-bit digits in
// [-16, 15] from the least significant end, the top digit taking the rest (|d_1| <= 32).
// This equals the digit expansion by repeated rounding to nearest, using integer work
// only (GB300's FP64 pipe is the scarce unit).
// Rows r >= sign_split are split negated (J's sign for a product A^T J B).
// A thread takes four consecutive rows r0 .. r0 + 3 of column j (one 8-byte store per
// slice); rows in [K, ldk) get zero digits (the padding TMA reads).  The optional copy of
// A is written on the way.  Grid: (ceil(ldk / 1024), n) blocks of 256 threads.
__device__ __forceinline__ long long split_value(long long bits, int ej, bool negate, int32_t* err) {
  const int f = (int)((bits >> 52) & 0x7FF);
  if (f == 0x7FF) {
    atomicExch(err, 2);
    return 0;
  }
  if (f == 0) return 0;  // subnormals are below 2^-1022 and round to 0 at 50 bits
  const unsigned long long mant = (unsigned long long)(bits & 0xFFFFFFFFFFFFFll) | (1ull << 52);
  // value = mant 2^(f - 1075); V = mant 2^(f - 1075 + kBeta*kSlices - e_j), rounded, with
  // |V| <= 2^(kBeta*kSlices - 1) as |a| < 2^(e_j - 1)
  const int sh = 1075 - f - kBeta * kSlices + ej;
  if (sh >= 64) return 0;
  const unsigned long long half = (sh > 0) ? (1ull << (sh - 1)) : 0ull;
  const unsigned long long mag = (sh > 0) ? ((mant + half) >> sh) : (mant << (-sh));
  return ((bits < 0) != negate) ? -(long long)mag : (long long)mag;
}

// The digits of four consecutive rows r0 .. r0 + 3 of column j: one 8-byte store per slice.
// Adding C = 32 (1 + 64 + ... + 64^(S-2)) turns the balanced digits d_t in [-32, 31] of
// V into the plain base-64 digits d_t + 32 of W = V + C, and W >> 6 (S - 1) is the top
// digit; so each digit is one 6-bit field of W.  A small integer u becomes its FP32 value
// by one integer and one FP32 addition (the bit pattern of 1.5 2^23 + u, minus 1.5 2^23),
// and, having at most 7 significant bits, its BF16 pattern is the float's upper half.
// This keeps the split off the conversion pipe (a quarter of the ALU rate).
__device__ __forceinline__ uint32_t small_int_bf16_bits(int u, float bias) {
  return __float_as_uint(__int_as_float(0x4B400000 + u) - bias) >> 16;
}

__device__ __forceinline__ void store_digits4(const long long (&V)[4], __nv_bfloat16* __restrict__ D, int64_t ldk,
                                              int n, int j, int64_t r0) {
  constexpr int kHalfBase = 1 << (kBeta - 1);  // 32: balanced digits lie in [-32, 31]
  constexpr long long kC = kHalfBase * ((1ll << (kBeta * (kSlices - 1))) - 1) / ((1ll << kBeta) - 1);
  long long W[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) W[i] = V[i] + kC;
#pragma unroll
  for (int t = 0; t < kSlices; ++t) {
    const int slice = kSlices - 1 - t;  // slice 0 holds the top digit
    uint32_t h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (t < kSlices - 1) {
        const int u = (int)((unsigned long long)W[i] >> (kBeta * t)) & ((1 << kBeta) - 1);  // d_t + 32
        h[i] = small_int_bf16_bits(u, 12582912.0f + (float)kHalfBase);
      } else {
        const int top = (int)(W[i] >> (kBeta * t));  // |top| <= 32
        h[i] = small_int_bf16_bits(top + 64, 12582912.0f + 64.0f);
      }
    }
    *reinterpret_cast<uint2*>(D + ((int64_t)slice * n + j) * ldk + r0) =
        make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
  }
}

__global__ void split_rows4_kernel(int K, int64_t ldk, int n, const double* __restrict__ A, int64_t lda,
                                   const int* __restrict__ exps, __nv_bfloat16* __restrict__ D, int32_t* err,
                                   double* __restrict__ Acopy, int64_t ldcopy, int sign_split) {
  const int j = blockIdx.y;
  const int64_t r0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (r0 >= ldk) return;
  const int ej = exps[j];
  long long V[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + i;
    V[i] = 0;
    if (r >= K) continue;
    const long long bits = __double_as_longlong(__ldg(A + r + (int64_t)j * lda));
    if (Acopy) Acopy[r + (int64_t)j * ldcopy] = __longlong_as_double(bits);
    V[i] = split_value(bits, ej, r >= sign_split, err);
  }
  store_digits4(V, D, ldk, n, j, r0);
}

// Exponent and digits in one pass: column j is taken by a cluster of C CTAs (grid (C, n),
// cluster (C, 1, 1)), CTA c holding rows [4096 c, 4096 (c + 1)) in registers, 4
// consecutive rows per thread and group of 1024.  The column's largest exponent field is
// the maximum of the C CTAs' maxima, read through distributed shared memory; then every
// CTA splits its rows.  Rows in [K, ldk) get zero digits.  Used for ldk <= 8 * 4096.
constexpr int kClusterRows = 4096;
constexpr int kClusterMax = 8;

__global__ void __launch_bounds__(256) exponent_split_cluster_kernel(int K, int64_t ldk, int n,
                                                                     const double* __restrict__ A, int64_t lda,
                                                                     int* __restrict__ exps,
                                                                     __nv_bfloat16* __restrict__ D, int32_t* err,
                                                                     double* __restrict__ Acopy, int64_t ldcopy,
                                                                     int sign_split) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ int s_red[8];
  __shared__ int s_max;
  __shared__ int s_e;
  const int j = blockIdx.y;
  const int64_t base = (int64_t)blockIdx.x * kClusterRows;
  constexpr int kGroups = kClusterRows / 1024;
  long long bits[kGroups][4];
  int mx = 0;
#pragma unroll
  for (int g = 0; g < kGroups; ++g) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = base + g * 1024 + 4 * threadIdx.x + i;
      bits[g][i] = r < K ? __double_as_longlong(__ldg(A + r + (int64_t)j * lda)) : 0ll;
      mx = max(mx, (int)((bits[g][i] >> 52) & 0x7FF));
    }
  }
  if (Acopy) {
#pragma unroll
    for (int g = 0; g < kGroups; ++g)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t r = base + g * 1024 + 4 * threadIdx.x + i;
        if (r < K) Acopy[r + (int64_t)j * ldcopy] = __longlong_as_double(bits[g][i]);
      }
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < 8; ++w) m = max(m, s_red[w]);
    s_max = m;
  }
  cl.sync();  // every CTA's s_max is written
  if (threadIdx.x == 0) {
    int m = 0;
    for (unsigned r = 0; r < cl.num_blocks(); ++r) m = max(m, *cl.map_shared_rank(&s_max, r));
    s_e = exponent_of_field(m);
    if (blockIdx.x == 0) exps[j] = s_e;
  }
  cl.sync();  // s_e is set, and no CTA leaves while another may still read its s_max
  const int ej = s_e;
#pragma unroll
  for (int g = 0; g < kGroups; ++g) {
    const int64_t r0 = base + g * 1024 + 4 * threadIdx.x;
    if (r0 >= ldk) break;
    long long V[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) V[i] = split_value(bits[g][i], ej, base + g * 1024 + 4 * threadIdx.x + i >= sign_split, err);
    store_digits4(V, D, ldk, n, j, r0);
  }
}

// C(i,j) for the upper tiles.  Every stored product is an exact integer held in FP32.
// The products of equal t + u carry the same scale 2^{e_i + e_j - beta (t + u)}, so they
// are added exactly in integers first (at most 9 terms of magnitude at most 2^24 each per K chunk), and
// the 9 group sums are joined by combine_groups (below).  Then the tile is mirrored.  Every
// tile has all its ordered-pair slots (a diagonal tile's transposed slots were written by
// the epilogue).  A thread takes one entry.
constexpr int kScales = kSlices;  // t + u = 2 .. S + 1

// Sum_g V[g] 2^(e - beta (g + 2)) for the exact integer group sums V[g] (g = t + u - 2).
// Groups are joined three at a time by exact int64 Horner steps (each part stays below 2^53
// for up to 8192 K chunks, so its conversion to FP64 is exact), then the parts by two
// FMAs and one ldexp: at most two roundings, and a handful of FP64 instructions instead of
// one conversion, scaling and addition per group (the FP64 pipe is GB300's scarce unit).
constexpr int kPartLen = 3;
constexpr int kParts = (kScales + kPartLen - 1) / kPartLen;

__device__ __forceinline__ double combine_groups(const long long (&V)[kScales], int e) {
  double acc = 0.0;
  int prev_last = -1;
#pragma unroll
  for (int p = 0; p < kParts; ++p) {
    const int g0 = p * kPartLen;
    const int g1 = (g0 + kPartLen < kScales ? g0 + kPartLen : kScales) - 1;  // last group of part p
    long long part = 0;
#pragma unroll
    for (int g = g0; g <= g1; ++g) part = part * (1ll << kBeta) + V[g];
    acc = p == 0 ? (double)part : fma(acc, (double)(1ll << (kBeta * (g1 - prev_last))), (double)part);
    prev_last = g1;
  }
  return ldexp(acc, e - kBeta * (kScales + 1));
}

// Group sums of one entry: every K chunk's exact products (FP32 integers), added by t + u.
__device__ __forceinline__ void group_sums(const uint32_t* __restrict__ base, int n_kchunks, size_t tile_elems,
                                           long long (&V)[kScales]) {
#pragma unroll
  for (int g = 0; g < kScales; ++g) V[g] = 0;
  for (int kc = 0; kc < n_kchunks; ++kc) {
    float w[slots_per_tile()];
#pragma unroll
    for (int slot = 0; slot < slots_per_tile(); ++slot)  // every load in flight before the sums
      w[slot] = __uint_as_float(__ldcg(base + ((size_t)slot * n_kchunks + kc) * tile_elems));
    int slot = 0;
#pragma unroll
    for (int t = 1; t <= kSlices; ++t)
#pragma unroll
      for (int u = 1; u <= kSlices + 1 - t; ++u, ++slot) V[t + u - 2] += (long long)__float2int_rz(w[slot]);
  }
}

__global__ void split_reduce_kernel(SplitParams P, double* __restrict__ C, int64_t ldc) {
  const int items_per_tile = slots_per_tile() * P.n_kchunks;
  const int n_upper = P.n_tiles * (P.n_tiles + 1) / 2;
  const size_t tile_elems = (size_t)kBM * kBN;
  const int64_t total = (int64_t)n_upper * tile_elems;
  const uint32_t* part = reinterpret_cast<const uint32_t*>(P.partial);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int tile = (int)(e / tile_elems);
    const int local = (int)(e % tile_elems);
    const int row = local % kBM, col = local / kBM;
    int r = 0;
    int tt = tile;
    while (tt >= P.n_tiles - r) {
      tt -= P.n_tiles - r;
      ++r;
    }
    const int bi = r, bj = r + tt;
    const int gi = bi * kBM + row, gj = bj * kBN + col;
    if (gj >= P.n || gi >= P.n || (bi == bj && gi > gj)) continue;
    long long V[kScales];
    group_sums(part + (size_t)tile * items_per_tile * tile_elems + local, P.n_kchunks, tile_elems, V);
    const double s = combine_groups(V, P.exps[gi] + P.exps[gj]);
    C[gi + (int64_t)gj * ldc] = s;
    C[gj + (int64_t)gi * ldc] = s;
  }
}

// The general product X^T Y (n x n2 output, every tile pair with all 45 ordered digit pairs):
// the same exact grouping by t + u.  With C0, C = C0 - X^T Y (the FP64 residual
// bbar - H X of a refinement step); C and C0 may be the same array.
__global__ void gemm_reduce_kernel(SplitParams P, double* __restrict__ C, int64_t ldc, const double* C0,
                                   int64_t ldc0) {
  const int items_per_tile = slots_per_tile() * P.n_kchunks;
  const size_t tile_elems = (size_t)kBM * kBN;
  const int64_t total = (int64_t)P.n_tiles * P.n_tiles2 * tile_elems;
  const uint32_t* part = reinterpret_cast<const uint32_t*>(P.partial);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int tile = (int)(e / tile_elems);
    const int local = (int)(e % tile_elems);
    const int row = local % kBM, col = local / kBM;
    const int bi = tile / P.n_tiles2, bj = tile % P.n_tiles2;
    const int gi = bi * kBM + row, gj = bj * kBN + col;
    if (gj >= P.n2 || gi >= P.n) continue;
    long long V[kScales];
    group_sums(part + (size_t)tile * items_per_tile * tile_elems + local, P.n_kchunks, tile_elems, V);
    const double v = combine_groups(V, P.exps[gi] + P.exps2[gj]);
    C[gi + (int64_t)gj * ldc] = C0 ? C0[gi + (int64_t)gj * ldc0] - v : v;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

size_t smem_bytes() { return 1024 + (size_t)kStages * kStageBytes + (2 * kStages + 2) * sizeof(uint64_t) + 16; }

}  // namespace

namespace {

// Heaviest-first tables of the Gram launches (group ids by MMA cost).
void fill_item_order(SplitParams& P) {
  for (int c = 0; c < 5; ++c) P.nd_c[c] = P.no_c[c] = 0;
  int od = 0, oo = 0;
  for (int c = 4; c >= 1; --c) {
    for (int g = 0; g < num_blocks(true); ++g)
      if (group_cost(true, g) == c) {
        P.gd_order[od++] = (int8_t)g;
        ++P.nd_c[c];
      }
    for (int g = 0; g < num_blocks(false); ++g)
      if (group_cost(false, g) == c) {
        P.go_order[oo++] = (int8_t)g;
        ++P.no_c[c];
      }
  }
}

constexpr bool kGramBalanceChunks = false;  // measured: the extra chunks' fill and drain cost more than they save

int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 148;
    }
  }
  return sms;
}

// K chunks of a Gram launch: at least ceil(K / 16384) (exact FP32 sums), and more where the
// heaviest items (the groups of the largest MMA cost) would not cover the SMs: each chunk
// then splits them, so the launch's length is set by items of about half the work, while
// every chunk keeps at least 4096 rows (fill and drain of an item stay small beside it).
// Returns the chunk count; *rows gets the rows per chunk (a multiple of 64).
int gram_kchunks(int64_t K, int64_t n, int* rows) {
  const int64_t nt = (n + kBM - 1) / kBM;
  int heavy_d = 0, heavy_o = 0, top = 0;
  for (int g = 0; g < num_blocks(true); ++g) top = std::max(top, group_cost(true, g));
  for (int g = 0; g < num_blocks(false); ++g) top = std::max(top, group_cost(false, g));
  for (int g = 0; g < num_blocks(true); ++g) heavy_d += group_cost(true, g) == top;
  for (int g = 0; g < num_blocks(false); ++g) heavy_o += group_cost(false, g) == top;
  const int64_t heavy = nt * heavy_d + nt * (nt - 1) / 2 * heavy_o;
  const int64_t base = std::max<int64_t>(1, (K + kKChunk - 1) / kKChunk);
  const int64_t want = kGramBalanceChunks ? (device_sms() + heavy - 1) / heavy : 1;
  const int64_t kc = std::max<int64_t>(base, std::min<int64_t>(want, K / 4096));
  int64_t r = (K + kc - 1) / kc;
  r = (r + kBK - 1) / kBK * kBK;
  if (r > kKChunk) r = kKChunk;
  *rows = (int)r;
  return (int)((K + r - 1) / r);
}

}  // namespace

GramSplitWork gram_split_work(int64_t K, int64_t n) {
  GramSplitWork w;
  const int64_t ldk = ((K + 7) / 8) * 8;
  const int64_t n_tiles = (n + kBM - 1) / kBM;
  const int64_t n_upper = n_tiles * (n_tiles + 1) / 2;
  int rows = 0;
  const int64_t n_kchunks = K > 0 ? gram_kchunks(K, n, &rows) : 1;
  w.slice_elems = (size_t)kSlices * (size_t)n * (size_t)ldk;
  w.partial_elems = (size_t)n_upper * slots_per_tile() * n_kchunks * kBM * kBN;
  w.exps = (size_t)n;
  return w;
}

namespace {

int64_t slice_ld(int64_t K) { return ((K + 7) / 8) * 8; }

// Digits of the K x n matrix A (rows >= sign_split negated) into slices (kSlices x n x ldk BF16)
// and the column exponents into exps; with a_copy, A is copied there on the way.
cudaError_t split_into(int64_t K, int64_t n, const double* A, int64_t lda, int64_t sign_split, void* slices, int* exps,
                       int32_t* err, cudaStream_t s, double* a_copy = nullptr, int64_t ld_copy = 0) {
  const int64_t ldk = slice_ld(K);
  __nv_bfloat16* D = static_cast<__nv_bfloat16*>(slices);
  const int ss = (int)std::min<int64_t>(sign_split, K);
  cudaError_t e;
  const int64_t C = (ldk + kClusterRows - 1) / kClusterRows;
  if (C <= kClusterMax) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, (unsigned)n);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, exponent_split_cluster_kernel, (int)K, ldk, (int)n, A, lda, exps, D, err, a_copy,
                           ld_copy, ss);
    note_launch();
    return e;
  }
  column_exponent_kernel<<<(unsigned)n, 1024, 0, s>>>((int)K, (int)n, A, lda, exps);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // ldk is a multiple of 8, so the threads' 4-row groups cover [0, ldk) exactly
  split_rows4_kernel<<<dim3((unsigned)((ldk + 1023) / 1024), (unsigned)n), 256, 0, s>>>(
      (int)K, ldk, (int)n, A, lda, exps, D, err, a_copy, ld_copy, ss);
  note_launch();
  return cudaGetLastError();
}

// TMA map over the slices: (K, n, digit) BF16, 128 x 64 boxes, 128-byte swizzle.
cudaError_t slices_map(const void* slices, int64_t K, int64_t n, CUtensorMap* map) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode_fn();
  if (!encode) return cudaErrorNotSupported;
  const int64_t ldk = slice_ld(K);
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)n, (cuuint64_t)kSlices};
  const cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)ldk * 2 * (cuuint64_t)n};
  const cuuint32_t box[3] = {kBK, kBM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(slices), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

}  // namespace

namespace {

SplitParams gram_params(int64_t K, int64_t n, int* exps, double* partial, int32_t* err) {
  SplitParams P;
  P.n = P.n2 = (int)n;
  P.K = (int)K;
  P.n_tiles = P.n_tiles2 = (int)((n + kBM - 1) / kBM);
  P.n_kchunks = gram_kchunks(K, n, &P.kchunk);
  fill_item_order(P);
  P.exps = P.exps2 = exps;
  P.partial = partial;
  P.err = err;
  return P;
}

int gram_items(const SplitParams& P) {
  const int n_upper = P.n_tiles * (P.n_tiles + 1) / 2;
  return (P.n_tiles * num_blocks(true) + (n_upper - P.n_tiles) * num_blocks(false)) * P.n_kchunks;
}

cudaError_t gram_reduce(const SplitParams& P, double* C, int64_t ldc, cudaStream_t s) {
  const int n_upper = P.n_tiles * (P.n_tiles + 1) / 2;
  split_reduce_kernel<<<(unsigned)std::min<int64_t>(((int64_t)n_upper * kBM * kBN + 255) / 256, 4096), 256, 0, s>>>(
      P, C, ldc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t gram_split_tc(int64_t K, int64_t n, const double* A, int64_t lda, double* C, int64_t ldc, void* slices,
                          double* partial, int* exps, int32_t* err, cudaStream_t s, cudaEvent_t mma_begin,
                          cudaEvent_t mma_end, double* a_copy, int64_t ld_copy, cudaEvent_t copied) {
  if (n <= 0) return cudaSuccess;
  if (K <= 0) return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * n, n, s);
  if (K > (int64_t)1 << 30 || n > 65535) return cudaErrorInvalidValue;
  cudaError_t e = split_into(K, n, A, lda, K, slices, exps, err, s, a_copy, ld_copy);
  if (e != cudaSuccess) return e;
  if (copied && (e = cudaEventRecord(copied, s)) != cudaSuccess) return e;
  CUtensorMap map;
  if ((e = slices_map(slices, K, n, &map)) != cudaSuccess) return e;
  const SplitParams P = gram_params(K, n, exps, partial, err);
  const int n_upper = P.n_tiles * (P.n_tiles + 1) / 2;
  const int items = gram_items(P);
  const size_t smem = smem_bytes();
  e = cudaFuncSetAttribute(gram_split_mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (mma_begin && (e = cudaEventRecord(mma_begin, s)) != cudaSuccess) return e;
  gram_split_mma_kernel<true><<<items, kThreads, smem, s>>>(map, map, P, P, items);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mma_end && (e = cudaEventRecord(mma_end, s)) != cudaSuccess) return e;
  split_reduce_kernel<<<(unsigned)std::min<int64_t>(((int64_t)n_upper * kBM * kBN + 255) / 256, 4096), 256, 0, s>>>(
      P, C, ldc);
  note_launch();
  return cudaGetLastError();
}


cudaError_t gram_split_pair_tc(int64_t K1, int64_t K2, int64_t n, const double* A1, int64_t lda1, const double* A2,
                               int64_t lda2, double* C1, double* C2, int64_t ldc, void* slices1, void* slices2,
                               double* partial1, double* partial2, int* exps1, int* exps2, int32_t* err,
                               cudaStream_t s1, cudaStream_t s2, cudaEvent_t ev_split2, cudaEvent_t ev_mma,
                               cudaEvent_t mma_begin, cudaEvent_t mma_end, double* copy1, double* copy2,
                               int64_t ld_copy, cudaEvent_t copied1) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e;
  if (K1 <= 0 || K2 <= 0) {  // a Gram of nothing is zero: no shared launch
    if ((e = gram_split_tc(K1, n, A1, lda1, C1, ldc, slices1, partial1, exps1, err, s1, mma_begin, mma_end, copy1,
                           ld_copy, copied1)) != cudaSuccess)
      return e;
    return gram_split_tc(K2, n, A2, lda2, C2, ldc, slices2, partial2, exps2, err, s2, nullptr, nullptr, copy2, ld_copy,
                         nullptr);
  }
  if (K1 > (int64_t)1 << 30 || K2 > (int64_t)1 << 30 || n > 65535) return cudaErrorInvalidValue;
  if ((e = split_into(K2, n, A2, lda2, K2, slices2, exps2, err, s2, copy2, ld_copy)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(ev_split2, s2)) != cudaSuccess) return e;
  if ((e = split_into(K1, n, A1, lda1, K1, slices1, exps1, err, s1, copy1, ld_copy)) != cudaSuccess) return e;
  if (copied1 && (e = cudaEventRecord(copied1, s1)) != cudaSuccess) return e;
  CUtensorMap map1, map2;
  if ((e = slices_map(slices1, K1, n, &map1)) != cudaSuccess) return e;
  if ((e = slices_map(slices2, K2, n, &map2)) != cudaSuccess) return e;
  const SplitParams P1 = gram_params(K1, n, exps1, partial1, err), P2 = gram_params(K2, n, exps2, partial2, err);
  // the longer Gram's items first: the block scheduler hands out blocks in order, so the
  // shorter one fills the SMs the longer one leaves
  const bool first1 = K1 >= K2;
  const SplitParams& Pa = first1 ? P1 : P2;
  const SplitParams& Pb = first1 ? P2 : P1;
  const int items_a = gram_items(Pa), items_b = gram_items(Pb);
  const size_t smem = smem_bytes();
  e = cudaFuncSetAttribute(gram_split_mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s1, ev_split2, 0)) != cudaSuccess) return e;
  if (mma_begin && (e = cudaEventRecord(mma_begin, s1)) != cudaSuccess) return e;
  gram_split_mma_kernel<true><<<items_a + items_b, kThreads, smem, s1>>>(first1 ? map1 : map2, first1 ? map2 : map1,
                                                                         Pa, Pb, items_a);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mma_end && (e = cudaEventRecord(mma_end, s1)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(ev_mma, s1)) != cudaSuccess) return e;
  if ((e = gram_reduce(P1, C1, ldc, s1)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s2, ev_mma, 0)) != cudaSuccess) return e;
  return gram_reduce(P2, C2, ldc, s2);
}

size_t digit_slice_elems(int64_t K, int64_t n) { return (size_t)kSlices * (size_t)n * (size_t)slice_ld(K); }

size_t gemm_partial_elems(int64_t K, int64_t n1, int64_t n2) {
  const int64_t t1 = (n1 + kBM - 1) / kBM, t2 = (n2 + kBN - 1) / kBN;
  const int64_t kc = std::max<int64_t>(1, (K + kKChunk - 1) / kKChunk);
  return (size_t)(t1 * t2) * slots_per_tile() * kc * kBM * kBN / 2;  // FP32 values in a double buffer
}

cudaError_t split_digits(int64_t K, int64_t n, const double* A, int64_t lda, int64_t sign_split, void* slices,
                         int* exps, int32_t* err, cudaStream_t s) {
  if (n <= 0 || K <= 0) return cudaSuccess;
  if (K > (int64_t)1 << 30 || n > 65535) return cudaErrorInvalidValue;
  return split_into(K, n, A, lda, sign_split, slices, exps, err, s);
}

cudaError_t gemm_split_tc(int64_t K, int64_t n1, int64_t n2, const void* slicesX, const int* expsX,
                          const void* slicesY, const int* expsY, double* C, int64_t ldc, const double* C0,
                          int64_t ldc0, double* partial, int32_t* err, cudaStream_t s) {
  if (n1 <= 0 || n2 <= 0) return cudaSuccess;
  if (K <= 0 || K > (int64_t)1 << 30 || n1 > 65535 || n2 > 65535) return cudaErrorInvalidValue;
  CUtensorMap mx, my;
  cudaError_t e;
  if ((e = slices_map(slicesX, K, n1, &mx)) != cudaSuccess) return e;
  if ((e = slices_map(slicesY, K, n2, &my)) != cudaSuccess) return e;
  SplitParams P;
  P.n = (int)n1;
  P.n2 = (int)n2;
  P.K = (int)K;
  P.n_tiles = (int)((n1 + kBM - 1) / kBM);
  P.n_tiles2 = (int)((n2 + kBN - 1) / kBN);
  P.n_kchunks = (int)std::max<int64_t>(1, (K + kKChunk - 1) / kKChunk);
  P.kchunk = kKChunk;
  fill_item_order(P);  // unused by the general product's items
  P.exps = expsX;
  P.exps2 = expsY;
  P.partial = partial;
  P.err = err;
  const int items = P.n_tiles * P.n_tiles2 * num_blocks(false) * P.n_kchunks;
  const size_t smem = smem_bytes();
  e = cudaFuncSetAttribute(gram_split_mma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  gram_split_mma_kernel<false><<<items, kThreads, smem, s>>>(mx, my, P, P, items);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  gemm_reduce_kernel<<<(unsigned)std::min<int64_t>(((int64_t)P.n_tiles * P.n_tiles2 * kBM * kBN + 255) / 256, 4096),
                       256, 0, s>>>(P, C, ldc, C0, ldc0);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ils
