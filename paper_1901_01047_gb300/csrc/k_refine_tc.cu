// k_refine_tc.cu -- the residual of the periodic recompute (mixed precision),
//     R = I - A N0,   A = e^V - g0 (e^V - 1) (Eq. Zk, formed in FP64 by
//                     k_build_A and held as FP32 pairs), N0 the FP32 N,
// on the 5th-generation tensor cores by exponent-aligned digit slicing
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)): every row of A and every
// column of N0 is written as a short sum of signed 9-bit integer digits
// times powers of two sharing one exponent per row (column),
//     A[i, k]  = 2^ea_i  sum_s  a_s[i, k] 2^(-9 (s + 1)),   s < 5,
//     N0[k, j] = 2^eb_j  sum_t  b_t[k, j] 2^(-9 (t + 1)),   t < 4,
// |a_s|, |b_t| <= 256, each exact in FP16.  A product of two digit planes is
// then a matrix of integers: with |a b| <= 2^16, the 128 terms of one chunk
// of K sum to at most 2^23 for one plane pair and 2^24 for two, so they
// accumulate without rounding in the FP32 accumulators of tcgen05.mma
// kind::f16.  The pairs (s, t) with
// s + t = g share the scale 2^(ea_i + eb_j - 9 (g + 2)) and one accumulator;
// groups 0 and 1 (the leading 2^-18 and 2^-27 parts) are read out exactly
// every 128 K and summed in double-float, groups 2 .. 5 (2^-36 and below)
// accumulate over all K in FP32, whose rounding stays below 2^-60 of the
// scale.  Pairs with s + t > 5 are dropped (17 products in all): the
// truncation of the digit expansions and the dropped pairs leave R within
// ~2^-40 of max|A_i.| max|N0_.j| per term, enough for the Newton step
// N1 = N0 + N0 R to bring an FP32 N back to its rounding level.
//
// Kernels:
//   k_oz_exp      exponents: ea_i from max_k |A[i, k]|, eb_j from max_k |N0[k, j]|
//   k_oz_slice_a  digit planes of A, row-major [5][cap][cap] (FP16)
//   k_oz_slice_n  digit planes of N0 transposed, [4][cap][cap]: row j holds column j
//   k_refine_oz   the 17 plane products, D^T[j, i] = sum_k b_t[k, j] a_s[i, k]
//                 (M = 128 columns j, N = 64 rows i, K = 64 per stage), and R
// The digit planes are zero for k in [n, roundup(n, 64)) (the last K stage);
// rows past n are never stored.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "device_util.cuh"
#include "item_plan.cuh"
#include "kernels.h"
#include "state.h"
#include "tc_ptx.cuh"

namespace dca {

constexpr int OZ_BETA = 9;    // bits per digit
constexpr int OZ_SA = 5;      // digit planes of A
constexpr int OZ_SB = 4;      // digit planes of N0
constexpr int OZ_T = 5;       // plane pairs with s + t <= OZ_T
constexpr int OZ_BM = 128;    // output columns j per tile (MMA M)
constexpr int OZ_BN = 64;     // output rows i per tile (MMA N)
constexpr int OZ_BK = 64;     // K per stage: one 128-byte row of FP16
constexpr int OZ_CH = 2;      // stages per exact chunk of groups 0 and 1 (K = 128)

__device__ __forceinline__ bool oz_wants(const WalkerDev& w) {
  return w.active && w.recompute_pending && w.status == ST_OK && w.n > 0;
}

// K extent of the digit planes that the stages read: n rounded up to the
// stage (within the buffer; the TMA fills columns past cap with zeros).
__device__ __forceinline__ int oz_kpad(const WalkerDev& w) {
  const int k = (w.n + OZ_BK - 1) / OZ_BK * OZ_BK;
  return k < w.cap ? k : w.cap;
}

// Exponent e with |x| < 2^e for every x of a row (column) whose largest
// magnitude is m, plus one: the scaled entries are below 1/2 in magnitude, so
// every rounded digit is at most 2^(OZ_BETA - 1).
__device__ __forceinline__ int oz_exponent(float m) {
  if (!(m > 0.0f)) return 0;
  int e;
  frexpf(m, &e);  // m = f 2^e, 1/2 <= f < 1
  return e + 1;
}

// Items per walker-spin: blocks of 8 rows of A (a warp per row), then
// strips of 32 columns of N0 (8 row groups of 32 threads, one thread per
// column and group, the group maxima combined in shared memory).
__global__ void __launch_bounds__(256) k_oz_exp(Config cfg) {
  __shared__ float s_m[8][32];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return oz_wants(w) ? blocks_of(w.n, 8) + blocks_of(w.n, 32) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap;
        const int rb = (int)blocks_of(n, 8);
        const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
        if (item < rb) {
          const int i = item * 8 + grp;
          if (i >= n) return;
          const float2* A = reinterpret_cast<const float2*>(w.Ascr[sp]) + (size_t)i * ld;
          float m = 0.0f;
          for (int k = lane; k < n; k += 32) m = fmaxf(m, fabsf(A[k].x));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (lane == 0) w.OzE[sp][i] = oz_exponent(m);
        } else {
          // block-uniform branch: the strip's barrier is reached by every thread
          const int j = (item - rb) * 32 + lane;
          const float* N0 = (const float*)w.N[w.parity][sp];
          float m = 0.0f;
          if (j < n)
#pragma unroll 4
            for (int k = grp; k < n; k += 8) m = fmaxf(m, fabsf(N0[(size_t)k * ld + j]));
          __syncthreads();  // the previous strip's reads of s_m are done
          s_m[grp][lane] = m;
          __syncthreads();
          if (grp == 0 && j < n) {
#pragma unroll
            for (int g = 1; g < 8; ++g) m = fmaxf(m, s_m[g][lane]);
            w.OzE[sp][ld + j] = oz_exponent(m);
          }
        }
      });
}

// Error-free sum of two FP32 values (Knuth): s + e = a + b exactly.
__device__ __forceinline__ void oz_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Digit planes of A: element (i, k) of row block i < n, k < kpad (zero for
// k >= n).  The value hi + lo scaled by 2^-ea_i is kept as a double-float
// remainder; each digit is the remainder times 2^9 rounded to an integer.
__global__ void __launch_bounds__(256) k_oz_slice_a(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return oz_wants(w) ? blocks_of((long long)w.n * oz_kpad(w), 256) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap, kp = oz_kpad(w);
        const long long e = (long long)item * 256 + threadIdx.x;
        if (e >= (long long)n * kp) return;
        const int i = (int)(e / kp), k = (int)(e - (long long)i * kp);
        __half* out = reinterpret_cast<__half*>(w.OzA[sp]) + (size_t)i * ld + k;
        const size_t plane = (size_t)ld * ld;
        if (k >= n) {
#pragma unroll
          for (int d = 0; d < OZ_SA; ++d) out[d * plane] = __float2half_rn(0.0f);
          return;
        }
        const float2 a = reinterpret_cast<const float2*>(w.Ascr[sp])[(size_t)i * ld + k];
        const int ea = w.OzE[sp][i];
        float xh = ldexpf(a.x, -ea), xl = ldexpf(a.y, -ea);  // exact: powers of two
#pragma unroll
        for (int d = 0; d < OZ_SA; ++d) {
          const float yh = xh * (float)(1 << OZ_BETA), yl = xl * (float)(1 << OZ_BETA);
          const float q = rintf(yh);
          out[d * plane] = __float2half_rn(q);  // |q| <= 256: exact
          oz_two_sum(__fsub_rn(yh, q), yl, xh, xl);
        }
      });
}

// Digit planes of N0, transposed: plane t, row j, column k = digit t of
// N0[k, j] scaled by 2^-eb_j.  Item = 32 x 32 tile (k0, j0) of N0 over
// k < kpad, j < n, staged through shared memory for the transposition.
__global__ void __launch_bounds__(256) k_oz_slice_n(Config cfg) {
  __shared__ __half ts[OZ_SB][32][34];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return oz_wants(w) ? blocks_of(oz_kpad(w), 32) * blocks_of(w.n, 32) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap, kp = oz_kpad(w);
        const int tj = (int)blocks_of(n, 32);
        const int k0 = (item / tj) * 32, j0 = (item - (item / tj) * tj) * 32;
        const float* N0 = (const float*)w.N[w.parity][sp];
        const int c = threadIdx.x & 31, r8 = threadIdx.x >> 5;
        __syncthreads();  // the previous item's reads of the tile are done
        const int j = j0 + c;
        const int eb = j < n ? w.OzE[sp][ld + j] : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = r8 + 8 * q, k = k0 + r;
          float x = (k < n && j < n) ? ldexpf(N0[(size_t)k * ld + j], -eb) : 0.0f;
#pragma unroll
          for (int d = 0; d < OZ_SB; ++d) {
            const float y = x * (float)(1 << OZ_BETA);
            const float qd = rintf(y);
            ts[d][c][r] = __float2half_rn(qd);
            x = __fsub_rn(y, qd);  // exact
          }
        }
        __syncthreads();
        __half* out = reinterpret_cast<__half*>(w.OzN[sp]);
        const size_t plane = (size_t)ld * ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rj = r8 + 8 * q, jj = j0 + rj, k = k0 + c;
          if (jj < n && k < kp)
#pragma unroll
            for (int d = 0; d < OZ_SB; ++d) out[d * plane + (size_t)jj * ld + k] = ts[d][rj][c];
        }
      });
}

// ---------------------------------------------------------------------------
// The plane products.  Work item = one tile of 128 columns j x 64 rows i of
// one walker-spin; a CTA (one per SM) streams the K extent in stages of 64:
//   warp 4 (TMA producer)  per stage the four N0 planes (128 rows j) and the
//                          five A planes (64 rows i), 104 KB, two stages;
//   warp 5 (MMA issuer)    17 products x 4 K steps of tcgen05.mma kind::f16
//                          (M = 128, N = 64) into six accumulators: groups
//                          0 and 1 in two alternating buffers (one per exact
//                          chunk of 128 K), groups 2 .. 5 for the whole item;
//   warps 0-3 (epilogue)   per chunk the exact groups into double-float
//                          registers, at the end of the item the rest, then
//                          R[i, j] = delta_ij - 2^(ea_i + eb_j - 18) sum.
// Tensor memory: 512 columns (groups 0 / 1 of buffer b at 128 b, 128 b + 64;
// group g >= 2 at 256 + 64 (g - 2)).  Every wait is bounded; a timeout sets
// the walker's status to ST_ERR_TIMEOUT, lets the copies in flight land,
// frees the tensor memory and returns.
struct OzLayout {
  static constexpr int N_TILE = OZ_BM * 128;                   // one N0 plane: 128 rows x 128 B
  static constexpr int A_TILE = OZ_BN * 128;                   // one A plane: 64 rows x 128 B
  static constexpr int STAGE = OZ_SB * N_TILE + OZ_SA * A_TILE;  // 106496
  static constexpr int OFF_BAR = 2 * STAGE;
  static constexpr int SMEM = OFF_BAR + 128 + 1024;            // barriers, TMEM slot, flag; alignment slack
  static constexpr uint32_t TMEM_COLS = 512;
  static_assert(SMEM + sizeof(ItemPlan) <= 232448, "shared memory (dynamic + the static item plan)");
};

__device__ __forceinline__ long long oz_items(const Config& cfg, int s) {
  const WalkerDev& w = cfg.W[s >> 1];
  return oz_wants(w) ? blocks_of(w.n, OZ_BM) * blocks_of(w.n, OZ_BN) : 0;
}

struct OzIter {
  PlanWalk<ItemPlan> pw;
  __device__ void start(const ItemPlan& plan) { pw.start(plan); }
  __device__ bool next(const Config& cfg, int& set, int& sub) {
    return pw.next(2 * cfg.n_walkers, [&](int s) { return oz_items(cfg, s); }, set, sub);
  }
};

__device__ __forceinline__ const void* oz_map(const Config& cfg, int wi, int sp, int kind) {
  return (const void*)(cfg.tmaps + ((size_t)wi * 2 + sp) * TMAPS_PER_SPIN + kind);
}

// Instruction descriptor of kind::f16 with FP16 operands and FP32
// accumulation, both operands K-major: D format bits 4-5 (1 = F32), A and B
// formats bits 7-9 / 10-12 (0 = F16), N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t oz_idesc() {
  return (1u << 4) | ((uint32_t)(OZ_BN >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ uint32_t oz_col(int g, int b) {
  return g < 2 ? (uint32_t)(128 * b + 64 * g) : (uint32_t)(256 + 64 * (g - 2));
}

__global__ void __launch_bounds__(192, 1) k_refine_oz(Config cfg) {
  using L = OzLayout;
  extern __shared__ uint8_t oz_raw[];
  const uint32_t raw = tc::smem_u32(oz_raw);
  const uint32_t sb = (raw + 1023u) & ~1023u;  // 1024-byte aligned base (128-byte swizzle atoms)
  uint8_t* gb = oz_raw + (sb - raw);
  const uint32_t bar = sb + L::OFF_BAR;
  // [2] each, 8 bytes apart: stage full / empty, accumulator buffer full / empty
  const uint32_t full0 = bar, empty0 = bar + 16, afull0 = bar + 32, aempty0 = bar + 48;
  const uint32_t gfree = bar + 64, fin = bar + 72;
  uint32_t* tmem_slot = (uint32_t*)(gb + L::OFF_BAR + 80);
  volatile int* abort_flag = (volatile int*)(gb + L::OFF_BAR + 84);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(full0 + 8 * s, 1);
      tc::mbar_init(empty0 + 8 * s, 1);
      tc::mbar_init(afull0 + 8 * s, 1);
      tc::mbar_init(aempty0 + 8 * s, 1);
    }
    tc::mbar_init(gfree, 1);
    tc::mbar_init(fin, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 5) {
    tc::tmem_alloc(tc::smem_u32(tmem_slot), L::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  __shared__ ItemPlan plan;
  plan_items(plan, 2 * cfg.n_walkers, [&](int s) { return oz_items(cfg, s); });

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      OzIter it;
      it.start(plan);
      uint32_t g = 0;
      uint32_t armed[2] = {0u, 0u};  // uses of each stage armed so far
      int set = 0, sub = 0;
      bool ok = true;
      while (ok && it.next(cfg, set, sub)) {
        const WalkerDev& w = cfg.W[set >> 1];
        const int wi = set >> 1, sp = set & 1, n = w.n, cap = w.cap;
        const int ti = (int)blocks_of(n, OZ_BN);
        const int j0 = (sub / ti) * OZ_BM, i0 = (sub - (sub / ti) * ti) * OZ_BN;
        const void* mN = oz_map(cfg, wi, sp, 8);
        const void* mA = oz_map(cfg, wi, sp, 9);
        const int nst = (n + OZ_BK - 1) / OZ_BK;
        for (int q = 0; q < nst; ++q, ++g) {
          const int st = (int)(g & 1u);
          const uint32_t u = g >> 1;
          if (u > 0 && !tc::mbar_wait(empty0 + 8 * st, (u - 1) & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          const uint32_t sS = sb + st * L::STAGE;
          tc::mbar_expect_tx(full0 + 8 * st, (uint32_t)L::STAGE);
          armed[st] = u + 1;
          const int k0 = q * OZ_BK;
          for (int t = 0; t < OZ_SB; ++t) tc::tma_load_2d(sS + t * L::N_TILE, mN, k0, t * cap + j0, full0 + 8 * st);
          for (int s = 0; s < OZ_SA; ++s)
            tc::tma_load_2d(sS + OZ_SB * L::N_TILE + s * L::A_TILE, mA, k0, s * cap + i0, full0 + 8 * st);
        }
      }
      if (!ok) {
        set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
        // the loads already issued land before the CTA exits
        for (int st = 0; st < 2; ++st)
          if (armed[st] > 0) tc::mbar_wait(full0 + 8 * st, (armed[st] - 1) & 1u, nullptr, 400000000LL);
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      OzIter it;
      it.start(plan);
      uint32_t g = 0, c = 0, items = 0;
      int set = 0, sub = 0;
      bool ok = true;
      constexpr uint32_t idesc = oz_idesc();
      while (ok && it.next(cfg, set, sub)) {
        const int n = cfg.W[set >> 1].n;
        const int nst = (n + OZ_BK - 1) / OZ_BK;
        // groups 2 .. 5 of the previous item have been read out
        if (items > 0 && !tc::mbar_wait(gfree, (items - 1) & 1u, abort_flag, cfg.wait_cycles)) {
          ok = false;
          break;
        }
        uint32_t started = 0;  // accumulators written in this item (groups >= 2) or chunk (0, 1)
        for (int q = 0; q < nst && ok; ++q, ++g) {
          const int st = (int)(g & 1u);
          const uint32_t u = g >> 1;
          const int b = (int)(c & 1u);
          if (q % OZ_CH == 0) {
            started &= ~3u;
            // buffer b of groups 0 / 1 has been read out (its use two chunks ago)
            if (c >= 2 && !tc::mbar_wait(aempty0 + 8 * b, ((c >> 1) - 1) & 1u, abort_flag, cfg.wait_cycles)) {
              ok = false;
              break;
            }
          }
          if (!tc::mbar_wait(full0 + 8 * st, u & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sS = sb + st * L::STAGE;
          for (int kk = 0; kk < OZ_BK / 16; ++kk) {
            // K step kk: 32-byte offset inside the 128-byte swizzle row
            for (int gg = 0; gg <= OZ_T; ++gg) {
              const uint32_t d = tmem + oz_col(gg, b);
              for (int s = 0; s < OZ_SA; ++s) {
                const int t = gg - s;
                if (t < 0 || t >= OZ_SB) continue;
                const uint64_t ad = tc::sdesc_k_sw128(sS + t * L::N_TILE + kk * 32);
                const uint64_t bd = tc::sdesc_k_sw128(sS + OZ_SB * L::N_TILE + s * L::A_TILE + kk * 32);
                mma_f16(d, ad, bd, idesc, (started >> gg) & 1u);
                started |= 1u << gg;
              }
            }
          }
          tc::mma_commit(empty0 + 8 * st);  // the stage's shared memory is free once these MMAs are done
          if (q % OZ_CH == OZ_CH - 1 || q == nst - 1) {
            tc::mma_commit(afull0 + 8 * b);  // the chunk (and, at the item's end, every group) is complete
            ++c;
          }
        }
        ++items;
      }
      if (!ok) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
      // every MMA of this CTA has completed before the tensor memory is freed
      tc::mma_commit(fin);
      tc::mbar_wait(fin, 0u, nullptr, 400000000LL);
    }
  } else {
    // ---------------- epilogue: warps 0-3, TMEM lanes 32 warp .. +31 ----------------
    OzIter it;
    it.start(plan);
    uint32_t c = 0;
    int set = 0, sub = 0;
    bool stop = false;
    const int r = 32 * warp + lane;  // column j of the tile = TMEM lane
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    while (!stop && it.next(cfg, set, sub)) {
      const WalkerDev& w = cfg.W[set >> 1];
      const int sp = set & 1, n = w.n, ld = w.cap;
      const int ti = (int)blocks_of(n, OZ_BN);
      const int j0 = (sub / ti) * OZ_BM, i0 = (sub - (sub / ti) * ti) * OZ_BN;
      const int nst = (n + OZ_BK - 1) / OZ_BK, nch = (nst + OZ_CH - 1) / OZ_CH;
      float h[OZ_BN], l[OZ_BN];  // sum of the groups in units of 2^(ea + eb - 18), double-float
#pragma unroll
      for (int x = 0; x < OZ_BN; ++x) h[x] = l[x] = 0.0f;
      for (int ch = 0; ch < nch && !stop; ++ch, ++c) {
        const int b = (int)(c & 1u);
        const bool mine = tc::mbar_wait(afull0 + 8 * b, (c >> 1) & 1u, abort_flag, cfg.wait_cycles);
        const bool okw = __all_sync(0xffffffffu, mine);
        if (okw) {
          tc::fence_after_sync();
          const bool last = ch == nch - 1;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            float v0[32], v1[32];
            tc::tmem_ld32(tmem + lane_base + oz_col(0, b) + 32 * half, v0);
            tc::tmem_ld32(tmem + lane_base + oz_col(1, b) + 32 * half, v1);
#pragma unroll
            for (int x = 0; x < 32; ++x) {
              float s, e;
              oz_two_sum(h[32 * half + x], v0[x], s, e);  // integers below 2^24: exact values
              l[32 * half + x] = __fadd_rn(l[32 * half + x], e);
              oz_two_sum(s, v1[x] * (1.0f / (float)(1 << OZ_BETA)), h[32 * half + x], e);
              l[32 * half + x] = __fadd_rn(l[32 * half + x], e);
            }
            if (last) {
#pragma unroll 1
              for (int gg = 2; gg <= OZ_T; ++gg) {
                const float sc = ldexpf(1.0f, -OZ_BETA * gg);
                tc::tmem_ld32(tmem + lane_base + oz_col(gg, b) + 32 * half, v0);
#pragma unroll
                for (int x = 0; x < 32; ++x) {
                  float s, e;
                  oz_two_sum(h[32 * half + x], v0[x] * sc, s, e);
                  h[32 * half + x] = s;
                  l[32 * half + x] = __fadd_rn(l[32 * half + x], e);
                }
              }
            }
          }
          tc::fence_before_sync();
        }
        // uniform decision of the 128 epilogue threads; then the buffer (and at
        // the item's end groups 2 .. 5) may be overwritten
        stop = tc::named_bar_or(1, 128, !okw || *abort_flag != 0);
        if (stop) break;
        if (threadIdx.x == 0) {
          tc::mbar_arrive(aempty0 + 8 * b);
          if (ch == nch - 1) tc::mbar_arrive(gfree);
        }
      }
      if (stop) break;
      // R[i, j] = delta_ij - 2^(ea_i + eb_j - 18) (h + l), FP32
      const int j = j0 + r;
      if (j < n) {
        const int eb = w.OzE[sp][ld + j];
        float* R = (float*)w.N[w.parity ^ 1][sp];
#pragma unroll
        for (int x = 0; x < OZ_BN; ++x) {
          const int i = i0 + x;
          if (i < n) {
            const int e = w.OzE[sp][i] + eb - 2 * OZ_BETA;
            const float d = __fsub_rn(i == j ? 1.0f : 0.0f, ldexpf(h[x], e));
            R[(size_t)i * ld + j] = __fsub_rn(d, ldexpf(l[x], e));
          }
        }
      }
    }
    if (stop && threadIdx.x == 0) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // an aborted CTA may have left any of its items undone: stop every walker it served
    OzIter it;
    it.start(plan);
    int set = 0, sub = 0;
    while (it.next(cfg, set, sub)) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
  }
  if (warp == 5) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, L::TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
cudaError_t setup_refine_tc() {
  return cudaFuncSetAttribute(k_refine_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, OzLayout::SMEM);
}

void launch_refine_oz(const Config& cfg, int max_cap, cudaStream_t st) {
  const long long S = 2LL * cfg.n_walkers;
  k_oz_exp<<<persist_grid((const void*)k_oz_exp, S * (blocks_of(max_cap, 8) + blocks_of(max_cap, 32)), 256), 256,
             0, st>>>(cfg);
  k_oz_slice_a<<<persist_grid((const void*)k_oz_slice_a, S * blocks_of((long long)max_cap * max_cap, 256), 256), 256,
                 0, st>>>(cfg);
  k_oz_slice_n<<<persist_grid((const void*)k_oz_slice_n, S * blocks_of(max_cap, 32) * blocks_of(max_cap, 32), 256),
                 256, 0, st>>>(cfg);
  k_refine_oz<<<device_sm_count(), 192, OzLayout::SMEM, st>>>(cfg);
}

}  // namespace dca
