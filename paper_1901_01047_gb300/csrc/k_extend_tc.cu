// k_extend_tc.cu -- candidate products of the extension on the 5th
// generation tensor cores (mixed precision), Sec. 2.3 "Submatrix updates":
//     G_ext[i, n + c] = sum_j N[i, j] V[c, j],   V[c, j] = g0(r_j - r_c, tau_j - tau_c)   (k_ext_g_tc)
//     X[c, j]         = sum_i U[c, i] N[i, j],   U[c, i] = g0(r_c - r_i, tau_c - tau_i) (e^{V_i} - 1)   (k_ext_x_tc)
// 3xTF32 as in the N update: every operand x is split into two TF32 values,
// hi = tf32(x) and lo = tf32(x - hi); hi*hi + hi*lo + lo*hi accumulate in
// FP32 in tensor memory.  V arrives pre-split from k_cand_zero ([hi | lo]
// planes x KS_MAX rows x cap columns, in the update-operand buffer that is
// free during the extension); N tiles are split in shared memory.
//
// Work item = one 128-row block of one walker-spin N.  The CTA streams the
// block's columns 32 at a time through a ring of stages (CN = 64: two CTAs
// per SM with two stages each; CN = 128: one CTA with three):
//   warp 4 (TMA producer)   N box (128 rows x 32 columns) and the V boxes;
//   warps 0-3 (converters)  split the N box in place into hi and a lo plane,
//                           zero the columns >= n; at the end of the item they
//                           read the accumulator and store G_ext;
//   warp 5 (MMA issuer)     4 K steps x 3 tcgen05.mma kind::tf32 (M = 128,
//                           N = CN candidates) into one TMEM accumulator.
// Every wait is bounded; a timeout sets the walker's status to
// ST_ERR_TIMEOUT, lets the copies in flight land, frees the tensor memory and
// returns.
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"
#include "item_plan.cuh"
#include "tc_ptx.cuh"

namespace dca {

constexpr int XT_BM = 128;    // rows per item

// CTAS CTAs per SM: one with a ring of as many stages as fit, or (CN = 64)
// two with two stages each, so that one CTA's epilogue overlaps the other's
// loads and products.
template <int CN, int CTAS = 1>
struct XtLayout {
  static constexpr int N_BOX = XT_BM * 128;     // 128 rows x 32 FP32 columns
  static constexpr int V_BOX = CN * 128;        // CN rows x 32 columns
  static constexpr int STAGE = 2 * N_BOX + 2 * V_BOX;  // N (hi), N lo, V hi, V lo
  static constexpr int STAGES = CTAS == 2 ? 2 : (CN <= 64 ? 4 : 3);  // ring depth
  static constexpr int OFF_BAR = STAGES * STAGE;
  static constexpr int SMEM = OFF_BAR + 256 + 1024;
  static constexpr uint32_t TMEM_COLS = CN < 32 ? 32 : CN;
  static_assert(CTAS * (SMEM + sizeof(ItemPlan) + 1024) <= 233472, "shared memory of the CTAs of one SM");
};

__device__ __forceinline__ long long xt_items(const Config& cfg, int s) {
  const WalkerDev& w = cfg.W[s >> 1];
  return (w.active && w.n_cand > 0 && w.n > 0) ? (long long)((w.n + XT_BM - 1) / XT_BM) : 0;
}

struct XtIter {
  PlanWalk<ItemPlan> pw;
  __device__ void start(const Config&, const ItemPlan& plan) { pw.start(plan); }
  __device__ bool next(const Config& cfg, int& set, int& rb) {
    return pw.next(2 * cfg.n_walkers, [&](int s) { return xt_items(cfg, s); }, set, rb);
  }
};

__device__ __forceinline__ const void* xt_map(const Config& cfg, int wi, int sp, int kind) {
  return (const void*)(cfg.tmaps + ((size_t)wi * 2 + sp) * TMAPS_PER_SPIN + kind);
}

template <int CN, int CTAS>
__global__ void __launch_bounds__(192, CTAS) k_ext_g_tc(Config cfg) {
  using L = XtLayout<CN, CTAS>;
  extern __shared__ uint8_t xt_raw[];
  const uint32_t raw = tc::smem_u32(xt_raw);
  const uint32_t sb = (raw + 1023u) & ~1023u;
  uint8_t* gb = xt_raw + (sb - raw);
  const uint32_t bar = sb + L::OFF_BAR;
  // barriers: full[S], conv[S], empty[S], dg_full, dg_empty, fin (S = L::STAGES)
  constexpr int S = L::STAGES;
  auto full = [&](int st) { return bar + 8 * st; };
  auto conv = [&](int st) { return bar + 8 * (S + st); };
  auto empty = [&](int st) { return bar + 8 * (2 * S + st); };
  const uint32_t dg_full = bar + 8 * (3 * S), dg_empty = dg_full + 8, fin = dg_full + 16;
  uint32_t* tmem_slot = (uint32_t*)(gb + L::OFF_BAR + 8 * (3 * S + 3));
  volatile int* abort_flag = (volatile int*)(gb + L::OFF_BAR + 8 * (3 * S + 3) + 4);
  static_assert(8 * (3 * S + 3) + 8 <= 256, "barrier area");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      tc::mbar_init(full(st), 1);
      tc::mbar_init(conv(st), 4);
      tc::mbar_init(empty(st), 1);
    }
    tc::mbar_init(dg_full, 1);
    tc::mbar_init(dg_empty, 4);
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
  plan_items(plan, 2 * cfg.n_walkers, [&](int s) { return xt_items(cfg, s); });

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      XtIter it;
      it.start(cfg, plan);
      uint32_t g = 0;
      uint32_t armed[S] = {};
      int set = 0, rb = 0;
      bool ok = true;
      while (ok && it.next(cfg, set, rb)) {
        const WalkerDev& w = cfg.W[set >> 1];
        const int wi = set >> 1, sp = set & 1, n = w.n, i0 = rb * XT_BM;
        const void* mN = xt_map(cfg, wi, sp, 2 + w.parity);
        const void* mN32 = xt_map(cfg, wi, sp, 6 + w.parity);  // 32-row boxes: the last, partial row block
        const int nsub = n - i0 >= XT_BM ? 4 : (n - i0 + 31) / 32;  // 32-row boxes that start below n
        const void* mV = xt_map(cfg, wi, sp, 4);
        for (int j0 = 0; j0 < n; j0 += 32, ++g) {
          const int st = (int)(g % S);
          const uint32_t u = g / S;
          if (u > 0 && !tc::mbar_wait(empty(st), (u - 1) & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          const uint32_t s0 = sb + st * L::STAGE;
          tc::mbar_expect_tx(full(st), (uint32_t)(nsub * (L::N_BOX / 4) + 2 * L::V_BOX));
          armed[st] = u + 1;
          if (nsub == 4) {
            tc::tma_load_2d(s0, mN, j0, i0, full(st));
          } else {
            for (int q = 0; q < nsub; ++q) tc::tma_load_2d(s0 + q * (L::N_BOX / 4), mN32, j0, i0 + 32 * q, full(st));
          }
          tc::tma_load_2d(s0 + 2 * L::N_BOX, mV, j0, 0, full(st));
          tc::tma_load_2d(s0 + 2 * L::N_BOX + L::V_BOX, mV, j0, KS_MAX, full(st));
        }
      }
      if (!ok) {
        set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
        for (int st = 0; st < S; ++st)
          if (armed[st] > 0) tc::mbar_wait(full(st), (armed[st] - 1) & 1u, nullptr, 400000000LL);
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      XtIter it;
      it.start(cfg, plan);
      uint32_t g = 0, k = 0;
      int set = 0, rb = 0;
      bool ok = true;
      const bool three = cfg.tf32_terms != 1;
      const uint32_t idesc = tc::idesc_tf32(XT_BM, CN);
      while (ok && it.next(cfg, set, rb)) {
        const int n = cfg.W[set >> 1].n;
        if (k > 0 && !tc::mbar_wait(dg_empty, (k - 1) & 1u, abort_flag, cfg.wait_cycles)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        bool first = true;
        for (int j0 = 0; j0 < n; j0 += 32, ++g) {
          const int st = (int)(g % S);
          const uint32_t u = g / S;
          if (!tc::mbar_wait(conv(st), u & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t s0 = sb + st * L::STAGE;
          const uint32_t nH = s0, nL = s0 + L::N_BOX, vH = s0 + 2 * L::N_BOX, vL = vH + L::V_BOX;
#pragma unroll
          for (int q = 0; q < 4; ++q) {  // K step of 8 columns: 32 bytes inside the 128-byte swizzle row
            const uint64_t ah = tc::sdesc_k_sw128(nH + 32 * q), al = tc::sdesc_k_sw128(nL + 32 * q);
            const uint64_t bh = tc::sdesc_k_sw128(vH + 32 * q), bl = tc::sdesc_k_sw128(vL + 32 * q);
            tc::mma_tf32(tmem, ah, bh, idesc, first ? 0u : 1u);
            if (three) {  // 3xTF32: the two correction products
              tc::mma_tf32(tmem, ah, bl, idesc, 1u);
              tc::mma_tf32(tmem, al, bh, idesc, 1u);
            }
            first = false;
          }
          tc::mma_commit(empty(st));
        }
        if (!ok) break;
        tc::mma_commit(dg_full);
        ++k;
      }
      if (!ok) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
      tc::mma_commit(fin);
      tc::mbar_wait(fin, 0u, nullptr, 400000000LL);
    }
  } else {
    // ---------------- converters / epilogue: warps 0-3 ----------------
    XtIter it;
    it.start(cfg, plan);
    uint32_t g = 0, k = 0;
    int set = 0, rb = 0;
    bool stop = false;
    const int r = 32 * warp + lane;  // row of the block = TMEM lane
    while (!stop && it.next(cfg, set, rb)) {
      WalkerDev& w = cfg.W[set >> 1];
      const int sp = set & 1, n = w.n, nc_ = w.n_cand, ld = w.cap, i0 = rb * XT_BM;
      for (int j0 = 0; j0 < n; j0 += 32, ++g) {
        const int st = (int)(g % S);
        const uint32_t u = g / S;
        const bool mine = tc::mbar_wait(full(st), u & 1u, abort_flag, cfg.wait_cycles);
        if (!__all_sync(0xffffffffu, mine)) {
          stop = true;
          break;
        }
        // split this thread's row of the N box: hi in place, lo in the lo plane.
        // Logical 16-byte chunk lc of row r sits at physical chunk lc ^ (r & 7)
        // (128-byte swizzle): walking logical chunks spreads the lanes of a warp
        // over all banks (walking physical chunks put all 32 lanes on 4 banks).
        // Rows >= n are zeroed: in the last row block their 32-row boxes are not loaded.
        uint8_t* nrow = gb + st * L::STAGE + r * 128;
        const bool row_ok = i0 + r < n;
#pragma unroll
        for (int lc = 0; lc < 8; ++lc) {
          const int pc = lc ^ (r & 7);
          float4* ph = (float4*)(nrow + pc * 16);
          float4* pl = (float4*)(nrow + L::N_BOX + pc * 16);
          float4 x = *ph;
          const int jc = j0 + 4 * lc;
          float xv[4] = {x.x, x.y, x.z, x.w}, hv[4], lv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) tc::tf32_split(row_ok && jc + q < n ? xv[q] : 0.f, hv[q], lv[q]);
          *ph = make_float4(hv[0], hv[1], hv[2], hv[3]);
          *pl = make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(conv(st));
      }
      if (stop) break;
      // accumulator of the item: row i0 + r, candidates 0 .. CN - 1
      const bool mine = tc::mbar_wait(dg_full, k & 1u, abort_flag, cfg.wait_cycles);
      if (!__all_sync(0xffffffffu, mine)) {
        stop = true;
        break;
      }
      tc::fence_after_sync();
      const int i = i0 + r;
#pragma unroll 1
      for (int cb = 0; cb < CN; cb += 32) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
        if (i < n)
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (cb + c < nc_) w.Gc[sp][(size_t)(cb + c) * ld + i] = (double)v[c];
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(dg_empty);
      ++k;
    }
    if (stop && lane == 0) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
    if (stop) *abort_flag = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // an aborted CTA may have left any of its items undone: stop every walker it served
    XtIter it;
    it.start(cfg, plan);
    int set = 0, rb = 0;
    while (it.next(cfg, set, rb)) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
  }
  if (warp == 5) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, L::TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// X[c, j] = sum_i U[c, i] N[i, j] (the candidates' rows of N), same 3xTF32
// scheme.  Work item = one 128-column block of one walker-spin N; the CTA
// streams the rows 32 at a time.  Operands per stage: U (A, K-major: 128
// candidate rows x 32 rows of N, [hi | lo] from k_cand_zero) and N^T (B,
// K-major: 128 columns of N x 32 rows), which the converter warps write
// transposed, split and swizzled from the four 32 x 32 boxes the TMA loads.
// Accumulator: 128 lanes (candidates) x 128 columns.
constexpr int XX2_BJ = 128;  // columns per item

// Stage: U hi | U lo (CN candidate rows each) | N boxes | N^T hi | N^T lo.
// The MMA has M = 128: with CN = 64 its rows 64 .. 127 read the next planes
// of the same stage (accumulator lanes that are never stored).
template <int CN>
struct Xx2Layout {
  static constexpr int U_TILE = CN * 128;              // CN candidates x 32 rows
  static constexpr int N_BOX = 32 * 128;               // 32 rows x 32 columns (TMA)
  static constexpr int N_TILE = 4 * N_BOX;             // 32 rows x 128 columns
  static constexpr int T_TILE = 128 * 128;             // N^T: 128 columns x 32 rows, one plane
  static constexpr int OFF_U = 0, OFF_N = 2 * U_TILE, OFF_T = OFF_N + N_TILE;
  static constexpr int STAGE = OFF_T + 2 * T_TILE;
  static constexpr int STAGES = CN <= 64 ? 3 : 2;      // ring depth: as many stages as fit
  static constexpr int OFF_BAR = STAGES * STAGE;
  static constexpr int SMEM = OFF_BAR + 256 + 1024;
  static constexpr uint32_t TMEM_COLS = XX2_BJ;
  static_assert(2 * U_TILE + N_TILE >= 128 * 128, "the M = 128 rows of the lo plane stay inside the stage");
  static_assert(SMEM + sizeof(ItemPlan) <= 232448, "shared memory (dynamic + the static item plan)");
};

__device__ __forceinline__ long long xx2_items(const Config& cfg, int s) {
  const WalkerDev& w = cfg.W[s >> 1];
  return (w.active && w.n_cand > 0 && w.n > 0) ? (long long)((w.n + XX2_BJ - 1) / XX2_BJ) : 0;
}

struct Xx2Iter {
  PlanWalk<ItemPlan> pw;
  __device__ void start(const Config&, const ItemPlan& plan) { pw.start(plan); }
  __device__ bool next(const Config& cfg, int& set, int& jb) {
    return pw.next(2 * cfg.n_walkers, [&](int s) { return xx2_items(cfg, s); }, set, jb);
  }
};

template <int CN>
__global__ void __launch_bounds__(192, 1) k_ext_x_tc(Config cfg) {
  using L = Xx2Layout<CN>;
  extern __shared__ uint8_t xx_raw[];
  const uint32_t raw = tc::smem_u32(xx_raw);
  const uint32_t sb = (raw + 1023u) & ~1023u;
  uint8_t* gb = xx_raw + (sb - raw);
  const uint32_t bar = sb + L::OFF_BAR;
  constexpr int S = L::STAGES;
  auto full = [&](int st) { return bar + 8 * st; };
  auto conv = [&](int st) { return bar + 8 * (S + st); };
  auto empty = [&](int st) { return bar + 8 * (2 * S + st); };
  const uint32_t dx_full = bar + 8 * (3 * S), dx_empty = dx_full + 8, fin = dx_full + 16;
  uint32_t* tmem_slot = (uint32_t*)(gb + L::OFF_BAR + 8 * (3 * S + 3));
  volatile int* abort_flag = (volatile int*)(gb + L::OFF_BAR + 8 * (3 * S + 3) + 4);
  static_assert(8 * (3 * S + 3) + 8 <= 256, "barrier area");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) {
      tc::mbar_init(full(st), 1);
      tc::mbar_init(conv(st), 4);
      tc::mbar_init(empty(st), 1);
    }
    tc::mbar_init(dx_full, 1);
    tc::mbar_init(dx_empty, 4);
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
  plan_items(plan, 2 * cfg.n_walkers, [&](int s) { return xx2_items(cfg, s); });

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      Xx2Iter it;
      it.start(cfg, plan);
      uint32_t g = 0;
      uint32_t armed[S] = {};
      int set = 0, jb = 0;
      bool ok = true;
      while (ok && it.next(cfg, set, jb)) {
        const WalkerDev& w = cfg.W[set >> 1];
        const int wi = set >> 1, sp = set & 1, n = w.n, j0 = jb * XX2_BJ;
        const void* mN = xt_map(cfg, wi, sp, 6 + w.parity);
        const void* mU = xt_map(cfg, wi, sp, 5);
        for (int i0 = 0; i0 < n; i0 += 32, ++g) {
          const int st = (int)(g % S);
          const uint32_t u = g / S;
          if (u > 0 && !tc::mbar_wait(empty(st), (u - 1) & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          const uint32_t s0 = sb + st * L::STAGE;
          // the 32-column boxes that start below n (the others are not loaded)
          const int ncb = (n - j0 + 31) / 32 < 4 ? (n - j0 + 31) / 32 : 4;
          tc::mbar_expect_tx(full(st), (uint32_t)(ncb * L::N_BOX + 2 * L::U_TILE));
          armed[st] = u + 1;
          for (int b = 0; b < ncb; ++b) tc::tma_load_2d(s0 + L::OFF_N + b * L::N_BOX, mN, j0 + 32 * b, i0, full(st));
          tc::tma_load_2d(s0 + L::OFF_U, mU, i0, 0, full(st));
          tc::tma_load_2d(s0 + L::OFF_U + L::U_TILE, mU, i0, KS_MAX, full(st));
        }
      }
      if (!ok) {
        set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
        for (int st = 0; st < S; ++st)
          if (armed[st] > 0) tc::mbar_wait(full(st), (armed[st] - 1) & 1u, nullptr, 400000000LL);
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      Xx2Iter it;
      it.start(cfg, plan);
      uint32_t g = 0, k = 0;
      int set = 0, jb = 0;
      bool ok = true;
      const bool three = cfg.tf32_terms != 1;
      const uint32_t idesc = tc::idesc_tf32(128, XX2_BJ);
      while (ok && it.next(cfg, set, jb)) {
        const int n = cfg.W[set >> 1].n;
        if (k > 0 && !tc::mbar_wait(dx_empty, (k - 1) & 1u, abort_flag, cfg.wait_cycles)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        bool first = true;
        for (int i0 = 0; i0 < n; i0 += 32, ++g) {
          const int st = (int)(g % S);
          const uint32_t u = g / S;
          if (!tc::mbar_wait(conv(st), u & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t s0 = sb + st * L::STAGE;
          const uint32_t tH = s0 + L::OFF_T, tL = tH + L::T_TILE, uH = s0 + L::OFF_U, uL = uH + L::U_TILE;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            // K step of 8 rows of N: 32 bytes inside the 128-byte swizzle rows of U and N^T
            const uint64_t ah = tc::sdesc_k_sw128(uH + 32 * q), al = tc::sdesc_k_sw128(uL + 32 * q);
            const uint64_t bh = tc::sdesc_k_sw128(tH + 32 * q), bl = tc::sdesc_k_sw128(tL + 32 * q);
            tc::mma_tf32(tmem, ah, bh, idesc, first ? 0u : 1u);
            if (three) {  // 3xTF32: the two correction products
              tc::mma_tf32(tmem, ah, bl, idesc, 1u);
              tc::mma_tf32(tmem, al, bh, idesc, 1u);
            }
            first = false;
          }
          tc::mma_commit(empty(st));
        }
        if (!ok) break;
        tc::mma_commit(dx_full);
        ++k;
      }
      if (!ok) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
      tc::mma_commit(fin);
      tc::mbar_wait(fin, 0u, nullptr, 400000000LL);
    }
  } else {
    // ---------------- converters / epilogue: warps 0-3 ----------------
    Xx2Iter it;
    it.start(cfg, plan);
    uint32_t g = 0, k = 0;
    int set = 0, jb = 0;
    bool stop = false;
    const int bx = warp, r = lane;  // converter: box bx, row r of the box
    while (!stop && it.next(cfg, set, jb)) {
      WalkerDev& w = cfg.W[set >> 1];
      const int sp = set & 1, n = w.n, nc_ = w.n_cand, ld = w.cap, j0 = jb * XX2_BJ;
      for (int i0 = 0; i0 < n; i0 += 32, ++g) {
        const int st = (int)(g % S);
        const uint32_t u = g / S;
        const bool mine = tc::mbar_wait(full(st), u & 1u, abort_flag, cfg.wait_cycles);
        if (!__all_sync(0xffffffffu, mine)) {
          stop = true;
          break;
        }
        // row i = i0 + r of box bx (columns j = 32 bx + 4 lc + q of the item):
        // split, and write N^T[j][i] into the K-major planes (row j, 128-byte
        // swizzle: 16-byte chunk (r >> 2) ^ (j & 7), word r & 3).  The 32 lanes
        // of a warp write the 32 words of one 128-byte row: no bank conflicts.
        // Rows >= n (K padding) and the boxes of columns >= n (not loaded) are
        // zeroed; the logical chunk lc of the box row sits at physical chunk
        // lc ^ (r & 7).
        const bool row_ok = i0 + r < n && j0 + 32 * bx < n;  // and the box was loaded
        const uint8_t* nrow = gb + st * L::STAGE + L::OFF_N + bx * L::N_BOX + r * 128;
        uint8_t* tH = gb + st * L::STAGE + L::OFF_T;
        uint8_t* tL = tH + L::T_TILE;
#pragma unroll
        for (int lc = 0; lc < 8; ++lc) {
          const float4 x = *(const float4*)(nrow + ((lc ^ (r & 7)) << 4));
          const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float hv, lv;
            tc::tf32_split(row_ok ? xv[q] : 0.f, hv, lv);
            const int j = 32 * bx + 4 * lc + q;
            const int off = j * 128 + ((((r >> 2) ^ (j & 7)) << 4) | ((r & 3) << 2));
            *(float*)(tH + off) = hv;
            *(float*)(tL + off) = lv;
          }
        }
        tc::fence_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(conv(st));
      }
      if (stop) break;
      const bool mine = tc::mbar_wait(dx_full, k & 1u, abort_flag, cfg.wait_cycles);
      if (!__all_sync(0xffffffffu, mine)) {
        stop = true;
        break;
      }
      tc::fence_after_sync();
      // accumulator lane = candidate 32 warp + lane, columns j0 .. j0 + 127
      if (32 * warp < nc_) {
        const int c = 32 * warp + lane;
        float* xrow = reinterpret_cast<float*>(w.Xr[sp]) + (size_t)c * ld;
#pragma unroll 1
        for (int cb = 0; cb < XX2_BJ; cb += 32) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
          if (c < nc_)
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (j0 + cb + q < n) xrow[j0 + cb + q] = v[q];
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(dx_empty);
      ++k;
    }
    if (stop && lane == 0) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
    if (stop) *abort_flag = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // an aborted CTA may have left any of its items undone: stop every walker it served
    Xx2Iter it;
    it.start(cfg, plan);
    int set = 0, rb = 0;
    while (it.next(cfg, set, rb)) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
  }
  if (warp == 5) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, L::TMEM_COLS);
  }
}

cudaError_t setup_ext_tc() {
  cudaError_t e = cudaFuncSetAttribute(k_ext_g_tc<64, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       XtLayout<64, 2>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ext_g_tc<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, XtLayout<128>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ext_x_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, Xx2Layout<64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ext_x_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Xx2Layout<128>::SMEM);
  return e;
}

void launch_ext_g_tc(const Config& cfg, cudaStream_t st) {
  const int sms = device_sm_count();
  if (ext_tile_c(cfg.ks) <= 64) k_ext_g_tc<64, 2><<<2 * sms, 192, XtLayout<64, 2>::SMEM, st>>>(cfg);
  else k_ext_g_tc<128, 1><<<sms, 192, XtLayout<128>::SMEM, st>>>(cfg);
}

void launch_ext_x_tc(const Config& cfg, cudaStream_t st) {
  const int sms = device_sm_count();
  if (ext_tile_c(cfg.ks) <= 64) k_ext_x_tc<64><<<sms, 192, Xx2Layout<64>::SMEM, st>>>(cfg);
  else k_ext_x_tc<128><<<sms, 192, Xx2Layout<128>::SMEM, st>>>(cfg);
}

}  // namespace dca
