// k_update_tc.cu -- the rank-l update of the FP32 N matrices (mixed
// precision) on the 5th-generation tensor cores:
//     N[0:n, 0:n) += L' R,   L' = (G[:,P] - E_P) diag(a_P) B^-1  (n x l),
//                             R  = N_ext[P, 0:n)                  (l x n),
// the submatrix update of the DCA++ paper (Sec. 2.3, "Submatrix updates").
//
// Precision (3xTF32).  Every FP32 operand x is split into two TF32 values,
// hi = x rounded to TF32 and lo = x - hi rounded to TF32 (the tensor core
// would otherwise truncate the remainder's low bits); the MMA chain
// accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor memory, each product
// exact, the split carrying x to about 2^-22 of |x|.  The split operands are written by k_upd_factors in the
// layout the TMA loads: planes [hi | lo] x rows x 128 K-columns (512 B rows).
//
// Work item = one 128-row block of one walker-spin N.  A CTA (one per SM)
// loads the block's L' rows (hi, lo; K = l rounded up to 32) once, then walks
// the 128 x BN column tiles of those rows through a two-stage pipeline:
//   warp 4 (TMA producer)  B operand rows (R^T hi, lo) and the N tile;
//   warp 5 (MMA issuer)    3 l/8 tcgen05.mma kind::tf32 into one of two TMEM
//                          accumulators (M = 128, N = BN);
//   warps 0-3 (epilogue)   TMEM -> registers, add into the N tile held in
//                          shared memory (128-byte swizzle), TMA store.
// Only the 32-column boxes, and in the last row block the 32-row boxes, that
// start below n are loaded and stored; inside them, rows or columns >= n are
// stored back unchanged.
#include <cuda.h>

#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"
#include "item_plan.cuh"
#include "tc_ptx.cuh"

namespace dca {

constexpr int TC_BM = 128;
constexpr int TC_KS = 128;  // K columns per operand row in global memory (KS_MAX)

template <int BN, int KP>
struct TcLayout {
  static constexpr int KCH = KP / 32;                 // 32-column (128-byte) K chunks
  static constexpr int A_CHUNK = TC_BM * 128;         // one chunk of one plane
  static constexpr int A_PLANE = KCH * A_CHUNK;
  static constexpr int B_CHUNK = BN * 128;
  static constexpr int B_PLANE = KCH * B_CHUNK;
  static constexpr int B_STAGE = 2 * B_PLANE;
  static constexpr int N_BOX = TC_BM * 128;           // 128 rows x 32 columns
  static constexpr int N_STAGE = (BN / 32) * N_BOX;
  static constexpr int OFF_A = 0;
  static constexpr int OFF_B = 2 * A_PLANE;
  static constexpr int OFF_N = OFF_B + 2 * B_STAGE;
  static constexpr int OFF_BAR = OFF_N + 2 * N_STAGE;
  static constexpr int SMEM = OFF_BAR + 128 + 1024;   // barriers, TMEM slot, flag; 1 KB alignment slack
  static constexpr uint32_t TMEM_COLS = 2 * BN;
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 128, "tile width");
  using Plan = typename std::conditional<SMEM + sizeof(ItemPlan) <= 232448, ItemPlan, ItemPlanSmall>::type;
  static_assert(SMEM + sizeof(Plan) <= 232448, "shared memory (dynamic + the static item plan)");
};

// Work items: (walker-spin s, 128-row block) for walkers with an update.
__device__ __forceinline__ long long tc_items(const Config& cfg, int s) {
  const WalkerDev& w = cfg.W[s >> 1];
  return (w.active && w.n_acc > 0) ? (long long)((w.n + TC_BM - 1) / TC_BM) : 0;
}

// Walk over the items of this CTA (the same in every role), from its plan.
template <typename Plan>
struct TcIter {
  PlanWalk<Plan> pw;
  __device__ void start(const Config&, const Plan& plan) { pw.start(plan); }
  __device__ bool next(const Config& cfg, int& set, int& rb) {
    return pw.next(2 * cfg.n_walkers, [&](int s) { return tc_items(cfg, s); }, set, rb);
  }
};

// 32-row boxes of the row block at i0 that start below n (4: the whole block),
// and 32-column boxes of the tile at j0 (BN columns) that start below n.
__device__ __forceinline__ int tc_row_boxes(int n, int i0) {
  const int r = n - i0;
  return r >= TC_BM ? 4 : (r + 31) / 32;
}
__device__ __forceinline__ int tc_col_boxes(int n, int j0, int bn) {
  const int c = (n - j0 + 31) / 32;
  return c < bn / 32 ? c : bn / 32;
}

__device__ __forceinline__ const void* tc_map(const Config& cfg, int wi, int sp, int kind) {
  return (const void*)(cfg.tmaps + ((size_t)wi * 2 + sp) * TMAPS_PER_SPIN + kind);
}

template <int BN, int KP>
__global__ void __launch_bounds__(192, 1) k_upd_tc(Config cfg) {
  using L = TcLayout<BN, KP>;
  extern __shared__ uint8_t tc_raw[];
  const uint32_t raw = tc::smem_u32(tc_raw);
  const uint32_t sb = (raw + 1023u) & ~1023u;  // 1024-byte aligned base (128-byte swizzle atoms)
  uint8_t* gb = tc_raw + (sb - raw);
  const uint32_t bar = sb + L::OFF_BAR;
  const uint32_t a_full = bar, a_empty = bar + 8, fin = bar + 16;
  const uint32_t full0 = bar + 24, mdone0 = bar + 40, empty0 = bar + 56;  // [2] each, 8 bytes apart
  uint32_t* tmem_slot = (uint32_t*)(gb + L::OFF_BAR + 72);
  volatile int* abort_flag = (volatile int*)(gb + L::OFF_BAR + 76);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    tc::mbar_init(a_full, 1);
    tc::mbar_init(a_empty, 1);
    tc::mbar_init(fin, 1);
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(full0 + 8 * s, 1);
      tc::mbar_init(mdone0 + 8 * s, 1);
      tc::mbar_init(empty0 + 8 * s, 1);
    }
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
  __shared__ typename L::Plan plan;
  plan_items(plan, 2 * cfg.n_walkers, [&](int s) { return tc_items(cfg, s); });

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      TcIter<typename L::Plan> it;
      it.start(cfg, plan);
      uint32_t g = 0, k = 0;
      uint32_t armed[2] = {0u, 0u};  // uses of each stage armed so far
      int set = 0, rb = 0;
      bool ok = true;
      while (ok && it.next(cfg, set, rb)) {
        const WalkerDev& w = cfg.W[set >> 1];
        const int wi = set >> 1, sp = set & 1;
        const int n = w.n, l = w.n_acc, kch = (l + 31) >> 5, i0 = rb * TC_BM, cap = w.cap;
        const void* mA = tc_map(cfg, wi, sp, 0);
        const void* mB = tc_map(cfg, wi, sp, 1);
        const void* mN = tc_map(cfg, wi, sp, 2 + w.parity);
        const void* mN32 = tc_map(cfg, wi, sp, 6 + w.parity);  // 32-row boxes: the last, partial row block
        const int nsub = tc_row_boxes(n, i0);
        if (k > 0 && !tc::mbar_wait(a_empty, (k - 1) & 1u, abort_flag, cfg.wait_cycles)) {
          ok = false;
          break;
        }
        tc::mbar_expect_tx(a_full, (uint32_t)(kch * 2 * L::A_CHUNK));
        for (int c = 0; c < kch; ++c)
          for (int h = 0; h < 2; ++h)
            tc::tma_load_2d(sb + L::OFF_A + h * L::A_PLANE + c * L::A_CHUNK, mA, 32 * c, h * cap + i0, a_full);
        ++k;
        const int ntiles = (n + BN - 1) / BN;
        for (int t = 0; t < ntiles; ++t, ++g) {
          const int st = (int)(g & 1u);
          const uint32_t u = g >> 1;
          if (u > 0 && !tc::mbar_wait(empty0 + 8 * st, (u - 1) & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          const int j0 = t * BN;
          const uint32_t sB = sb + L::OFF_B + st * L::B_STAGE, sN = sb + L::OFF_N + st * L::N_STAGE;
          // the N tile: 32-column boxes that start below n, and in the last row
          // block only the 32-row boxes that start below n (the rest of the
          // tile is neither read nor stored)
          const int ncb = tc_col_boxes(n, j0, BN);
          tc::mbar_expect_tx(full0 + 8 * st, (uint32_t)(kch * 2 * L::B_CHUNK + ncb * nsub * (L::N_BOX / 4)));
          armed[st] = u + 1;
          for (int c = 0; c < kch; ++c)
            for (int h = 0; h < 2; ++h)
              tc::tma_load_2d(sB + h * L::B_PLANE + c * L::B_CHUNK, mB, 32 * c, h * cap + j0, full0 + 8 * st);
          for (int b = 0; b < ncb; ++b) {
            if (nsub == 4) {
              tc::tma_load_2d(sN + b * L::N_BOX, mN, j0 + 32 * b, i0, full0 + 8 * st);
            } else {
              for (int q = 0; q < nsub; ++q)
                tc::tma_load_2d(sN + b * L::N_BOX + q * (L::N_BOX / 4), mN32, j0 + 32 * b, i0 + 32 * q, full0 + 8 * st);
            }
          }
        }
      }
      if (!ok) {
        set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
        // the loads already issued land before the CTA exits
        if (k > 0) tc::mbar_wait(a_full, (k - 1) & 1u, nullptr, 400000000LL);
        for (int st = 0; st < 2; ++st)
          if (armed[st] > 0) tc::mbar_wait(full0 + 8 * st, (armed[st] - 1) & 1u, nullptr, 400000000LL);
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      TcIter<typename L::Plan> it;
      it.start(cfg, plan);
      uint32_t g = 0, k = 0;
      int set = 0, rb = 0;
      bool ok = true;
      const bool three = cfg.tf32_terms != 1;
      const uint32_t idesc = tc::idesc_tf32(TC_BM, BN);
      while (ok && it.next(cfg, set, rb)) {
        const WalkerDev& w = cfg.W[set >> 1];
        const int n = w.n, steps = (w.n_acc + 7) >> 3;
        if (!tc::mbar_wait(a_full, k & 1u, abort_flag, cfg.wait_cycles)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t aH = sb + L::OFF_A, aL = aH + L::A_PLANE;
        const int ntiles = (n + BN - 1) / BN;
        for (int t = 0; t < ntiles; ++t, ++g) {
          const int st = (int)(g & 1u);
          const uint32_t u = g >> 1;
          if ((u > 0 && !tc::mbar_wait(empty0 + 8 * st, (u - 1) & 1u, abort_flag, cfg.wait_cycles)) ||
              !tc::mbar_wait(full0 + 8 * st, u & 1u, abort_flag, cfg.wait_cycles)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t d = tmem + (uint32_t)(st * BN);
          const uint32_t bH = sb + L::OFF_B + st * L::B_STAGE, bL = bH + L::B_PLANE;
          for (int q = 0; q < steps; ++q) {
            // K step q: chunk q / 4, 32-byte offset (q % 4) inside the 128-byte swizzle row
            const uint32_t ao = (uint32_t)((q >> 2) * L::A_CHUNK + (q & 3) * 32);
            const uint32_t bo = (uint32_t)((q >> 2) * L::B_CHUNK + (q & 3) * 32);
            const uint64_t ah = tc::sdesc_k_sw128(aH + ao), al = tc::sdesc_k_sw128(aL + ao);
            const uint64_t bh = tc::sdesc_k_sw128(bH + bo), bl = tc::sdesc_k_sw128(bL + bo);
            tc::mma_tf32(d, ah, bh, idesc, q > 0 ? 1u : 0u);
            if (three) {  // 3xTF32: the two correction products
              tc::mma_tf32(d, ah, bl, idesc, 1u);
              tc::mma_tf32(d, al, bh, idesc, 1u);
            }
          }
          tc::mma_commit(mdone0 + 8 * st);
        }
        if (!ok) break;
        tc::mma_commit(a_empty);
        ++k;
      }
      if (!ok) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
      // every MMA of this CTA has completed before the tensor memory is freed
      tc::mma_commit(fin);
      tc::mbar_wait(fin, 0u, nullptr, 400000000LL);
    }
  } else {
    // ---------------- epilogue: warps 0-3, TMEM lanes 32 warp .. +31 ----------------
    TcIter<typename L::Plan> it;
    it.start(cfg, plan);
    uint32_t g = 0;
    int set = 0, rb = 0;
    bool stop = false;
    const int r = 32 * warp + lane;  // row of the block = TMEM lane
    while (!stop && it.next(cfg, set, rb)) {
      const WalkerDev& w = cfg.W[set >> 1];
      const int wi = set >> 1, sp = set & 1, n = w.n, i0 = rb * TC_BM;
      const void* mN = tc_map(cfg, wi, sp, 2 + w.parity);
      const void* mN32 = tc_map(cfg, wi, sp, 6 + w.parity);
      const int nsub = tc_row_boxes(n, i0);
      const bool row_ok = i0 + r < n;
      const int ntiles = (n + BN - 1) / BN;
      for (int t = 0; t < ntiles; ++t, ++g) {
        const int st = (int)(g & 1u);
        const uint32_t u = g >> 1;
        const int j0 = t * BN;
        // every lane waits; the warp proceeds only if all lanes saw both phases
        // complete (tcgen05.ld is warp-wide)
        const bool mine =
            tc::mbar_wait(full0 + 8 * st, u & 1u, abort_flag, cfg.wait_cycles) && tc::mbar_wait(mdone0 + 8 * st, u & 1u, abort_flag, cfg.wait_cycles);
        const bool okw = __all_sync(0xffffffffu, mine);
        if (okw) {
          tc::fence_after_sync();
          uint8_t* tile = gb + L::OFF_N + st * L::N_STAGE;
#pragma unroll 1
          for (int b = 0; b < BN / 32; ++b) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(st * BN + 32 * b), v);
            uint8_t* rowp = tile + b * L::N_BOX + r * 128;
            const int cb = j0 + 32 * b;
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) {
              float4* p = (float4*)(rowp + ((ch ^ (r & 7)) << 4));
              float4 x = *p;
              const int c = cb + 4 * ch;
              if (row_ok) {
                if (c < n) x.x += v[4 * ch];
                if (c + 1 < n) x.y += v[4 * ch + 1];
                if (c + 2 < n) x.z += v[4 * ch + 2];
                if (c + 3 < n) x.w += v[4 * ch + 3];
              }
              *p = x;
            }
          }
          tc::fence_before_sync();
          tc::fence_async_smem();
        }
        // uniform decision of the 128 epilogue threads
        stop = tc::named_bar_or(1, 128, !okw || *abort_flag != 0);
        if (stop) break;
        if (threadIdx.x == 0) {
          const int ncb = tc_col_boxes(n, j0, BN);
          for (int b = 0; b < ncb; ++b) {
            const uint32_t box = sb + L::OFF_N + st * L::N_STAGE + b * L::N_BOX;
            if (nsub == 4) {
              tc::tma_store_2d(mN, j0 + 32 * b, i0, box);
            } else {
              for (int q = 0; q < nsub; ++q)
                tc::tma_store_2d(mN32, j0 + 32 * b, i0 + 32 * q, box + q * (L::N_BOX / 4));
            }
          }
          tc::bulk_commit();
          tc::bulk_wait_read0();
          tc::mbar_arrive(empty0 + 8 * st);
        }
      }
    }
    if (stop && threadIdx.x == 0) set_status(cfg.W[set >> 1], ST_ERR_TIMEOUT);
    if (threadIdx.x == 0) tc::bulk_wait0();
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // an aborted CTA may have left any of its items undone: stop every walker it served
    TcIter<typename L::Plan> it;
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

// The update factors of the tensor-core path in one pass (replaces the three
// kernels of the other paths, L -> L' -> split operands):
//   L[x, p]  = (G_ext[x, P_p] - delta_{x P_p}) a_p   for the rows x of the block,
//   L'[x, :] = L[x, :] B^-1                           (double-float, stored in Lp),
//   A rows x < n of the operand: TF32 split of L'[x, p], zero for l <= p < lpad;
// and per 32-column block of R = N_ext[P, :] (stored in Rr for the border
// update) its transposed TF32 split into the B operand.
// L is formed in double-float on the FP32 pipes for the rows x < n (N and
// the candidate columns G_ext[x < n, c] are FP32 products, so exact in FP32;
// the per-column factors e^{V} / (e^{V} - 1) a_p are formed once per item in
// FP64 and split), in FP64 for the rows of accepted insertions (X is FP64).
// Items per walker-spin: ceil(rows / 32) row blocks (rows = n + n_ins), then
// ceil(n / 32) column blocks.  Dynamic shared memory: the L rows of a row
// block [32][ld], ld = 65 with k_s <= 64 (then also B^-1, [64][64]) or 129
// (odd strides: the rows a warp reads at one p fall in different banks); a
// column block reuses it as the transposition tile [128][33].
constexpr int FACT_RB = 32, FACT_BS = 64, FACT_PB = 8;

__host__ __device__ constexpr size_t fact_smem(bool bs) {
  return bs ? sizeof(float2) * (FACT_RB * (FACT_BS + 1) + FACT_BS * FACT_BS) : sizeof(float2) * FACT_RB * (KS_MAX + 1);
}

__global__ void __launch_bounds__(256) k_upd_factors(Config cfg) {
  constexpr int RB = FACT_RB;
  static_assert(KS_MAX * 33 * sizeof(float) <= fact_smem(false) && fact_smem(false) <= fact_smem(true), "tiles");
  __shared__ float2 s_c1[KS_MAX];
  __shared__ int s_pp[KS_MAX], s_ok[KS_MAX], s_xr[FACT_RB];
  extern __shared__ __align__(16) float2 s_dyn[];
  const bool bs = cfg.ks <= FACT_BS;
  const int lds = bs ? FACT_BS + 1 : KS_MAX + 1;  // row stride of the L rows
  float2* s_Lb = s_dyn;                           // [RB][lds]
  float2* s_binv = s_dyn + RB * (FACT_BS + 1);    // [FACT_BS][FACT_BS] (bs only)
  float(*s_t)[33] = reinterpret_cast<float(*)[33]>(s_dyn);  // [KS_MAX][33]
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        if (!(w.active && w.n_acc > 0)) return 0;
        return blocks_of(w.n + w.n_ins, RB) + blocks_of(w.n, RB);
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, l = w.n_acc, cap = w.cap, ld = w.cap;
        const int rows = n + w.n_ins, lpad = (l + 31) & ~31;
        const int ra = (int)blocks_of(rows, RB);
        const ProblemDev& pb = cfg.P[w.problem];
        const float* N = (const float*)w.N[w.parity][sp];
        const int* vs = w.vs[w.parity];
        __syncthreads();  // the previous item is done with the shared tiles
        if (item < ra) {
          const int t0 = item * RB;
          for (int r = threadIdx.x; r < RB; r += blockDim.x) {
            const int t = t0 + r;
            int x = -1;
            if (t < rows) {
              x = t < n ? t : n + w.acc_slot[t - n];
              if (x < n && vs[x] == 0) x = -1;  // dead row: its L row is zero
            }
            s_xr[r] = x;
          }
          for (int p = threadIdx.x; p < l; p += blockDim.x) {
            const int P = w.P[p];
            const double a = w.aP[sp][p];
            s_pp[p] = P;
            s_ok[p] = a != 0.0;
            if (P < n) {
              const int sy = vs[P];
              s_c1[p] = df_split(expV(pb, sp, sy) * pb.rexpVm1[sp][sy > 0 ? 1 : 0] * a);
            } else {
              s_c1[p] = df_split(a);
            }
          }
          const float2* Bi = reinterpret_cast<const float2*>(w.Binv[sp]);
          if (bs)
            for (int e = threadIdx.x; e < l * lpad; e += blockDim.x) {
              const int p = e / lpad, q = e - p * lpad;
              s_binv[p * FACT_BS + q] = q < l ? Bi[(size_t)p * KS_MAX + q] : make_float2(0.f, 0.f);
            }
          __syncthreads();
          // L in batches of FACT_PB entries per thread: the loads of a batch are all
          // issued before the arithmetic (they are scattered columns of N)
          for (int e0 = 0; e0 < RB * l; e0 += FACT_PB * 256) {
            float gv[FACT_PB];
#pragma unroll
            for (int k = 0; k < FACT_PB; ++k) {
              const int e = e0 + k * 256 + threadIdx.x;
              gv[k] = 0.f;
              if (e < RB * l) {
                const int r = e / l, p = e - r * l;
                const int x = s_xr[r], P = s_pp[p];
                if (x >= 0 && x < n && s_ok[p])
                  gv[k] = P < n ? N[(size_t)x * ld + P] : (float)w.Gc[sp][(size_t)(P - n) * ld + x];
              }
            }
#pragma unroll
            for (int k = 0; k < FACT_PB; ++k) {
              const int e = e0 + k * 256 + threadIdx.x;
              if (e >= RB * l) break;
              const int r = e / l, p = e - r * l;
              const int x = s_xr[r], P = s_pp[p];
              float2 v = make_float2(0.f, 0.f);
              if (x >= 0 && s_ok[p]) {
                if (x < n) {
                  // FP32-exact entry times the column factor, in double-float.  An
                  // existing column y = P: G_ext[x, y] = (N_xy e^{V_y} - delta) / (e^{V_y} - 1),
                  // so (G_ext - delta) a = (N_xy - delta) e^{V_y} a / (e^{V_y} - 1) = (N_xy - delta) c1;
                  // a candidate column: (G_ext[x, c] - 0) a with c1 = a (x < n is never the candidate)
                  float hi = 0.f, lo = 0.f;
                  df_fma(hi, lo, gv[k], 0.f, s_c1[p].x, s_c1[p].y);
                  if (x == P) df_fma(hi, lo, -1.f, 0.f, s_c1[p].x, s_c1[p].y);
                  v = df_norm(hi, lo);
                } else {
                  const double a = w.aP[sp][p];
                  double val;
                  if (P < n) {
                    const int sy = vs[P];
                    val = ((double)reinterpret_cast<const float*>(w.Xr[sp])[(size_t)(x - n) * ld + P] * expV(pb, sp, sy)) *
                          pb.rexpVm1[sp][sy > 0 ? 1 : 0] * a;
                  } else {
                    val = (w.Gc[sp][(size_t)(P - n) * ld + x] - (x == P ? 1.0 : 0.0)) * a;
                  }
                  v = df_split(val);
                }
              }
              s_Lb[r * lds + p] = v;
            }
          }
          __syncthreads();
          // L' = L B^-1: four consecutive outputs of a row per thread (four
          // independent double-float chains sharing the loads of L)
          const int lq = lpad / 4;
          for (int e = threadIdx.x; e < RB * lq; e += blockDim.x) {
            const int r = e / lq, q = (e - r * lq) * 4;
            const int t = t0 + r;
            if (t >= rows) continue;
            const int x = t < n ? t : n + w.acc_slot[t - n];
            float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
            if (q < l) {
              for (int p = 0; p < l; ++p) {
                const float2 a = s_Lb[r * lds + p];
                const float2* brow = bs ? s_binv + p * FACT_BS + q : Bi + (size_t)p * KS_MAX + q;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const float2 b = brow[u];  // columns >= l of B^-1 are never read back
                  df_fma(hi[u], lo[u], a.x, a.y, b.x, b.y);
                }
              }
            }
            float2* lp = reinterpret_cast<float2*>(w.Lp[sp]) + (size_t)x * KS_MAX + q;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float2 o = df_norm(hi[u], lo[u]);
              if (q + u < l) lp[u] = o;
              if (x < n) {
                float th, tl;
                tc::tf32_split(q + u < l ? o.x : 0.0f, th, tl);
                w.Aop[sp][(size_t)x * TC_KS + q + u] = th;
                w.Aop[sp][((size_t)cap + x) * TC_KS + q + u] = tl;
              }
            }
          }
        } else {
          // R rows (Rr, for the border update) and the transposed split B operand
          const int j0 = (item - ra) * RB;
          const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, j = j0 + lane;
          float* Rr = (float*)w.Rr[sp];
          float rv[KS_MAX / 8];  // this lane's entries of rows p = warp + 8 k, loads issued together
#pragma unroll
          for (int k = 0; k < KS_MAX / 8; ++k) {
            const int p = warp + 8 * k;
            rv[k] = 0.0f;
            if (p < l && j < n) {
              const int P = w.P[p];
              rv[k] = P < n ? N[(size_t)P * ld + j] : reinterpret_cast<const float*>(w.Xr[sp])[(size_t)(P - n) * ld + j];
            }
          }
#pragma unroll
          for (int k = 0; k < KS_MAX / 8; ++k) {
            const int p = warp + 8 * k;
            if (p < lpad) {
              if (p < l && j < n) Rr[(size_t)p * cap + j] = rv[k];
              s_t[p][lane] = rv[k];
            }
          }
          __syncthreads();
          for (int jj = warp; jj < RB; jj += 8) {
            const int jr = j0 + jj;
            if (jr < n)
              for (int p = lane; p < lpad; p += 32) {
                float hi, lo;
                tc::tf32_split(s_t[p][jj], hi, lo);
                w.Bop[sp][(size_t)jr * TC_KS + p] = hi;
                w.Bop[sp][((size_t)cap + jr) * TC_KS + p] = lo;
              }
          }
        }
      });
}

void launch_upd_factors(const Config& cfg, int max_cap, cudaStream_t st) {
  const long long items = 2LL * cfg.n_walkers * (blocks_of(max_cap, 32) + blocks_of(max_cap, 32));
  const size_t smem = fact_smem(cfg.ks <= FACT_BS);
  k_upd_factors<<<persist_grid((const void*)k_upd_factors, items, 256, smem), 256, smem, st>>>(cfg);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int BN, int KP>
static cudaError_t tc_setup_one() {
  return cudaFuncSetAttribute(k_upd_tc<BN, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcLayout<BN, KP>::SMEM);
}

cudaError_t setup_update_tc() {
  cudaError_t e = cudaFuncSetAttribute(k_upd_factors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fact_smem(true));
  if (e == cudaSuccess) e = tc_setup_one<64, 32>();
  if (e == cudaSuccess) e = tc_setup_one<32, 32>();
  if (e == cudaSuccess) e = tc_setup_one<32, 64>();
  if (e == cudaSuccess) e = tc_setup_one<64, 64>();
  if (e == cudaSuccess) e = tc_setup_one<32, 128>();
  return e;
}

int tc_tile_n(int ks, int bn) {
  if (ks > 64) return 32;           // the K extent of 128 leaves room for BN = 32 only
  return bn == 32 ? 32 : 64;        // default 64
}


void launch_upd_tc(const Config& cfg, cudaStream_t st) {
  const int grid = device_sm_count();
  const bool wide = tc_tile_n(cfg.ks, cfg.upd_bn) == 64;
  if (cfg.ks <= 32) {
    if (wide) k_upd_tc<64, 32><<<grid, 192, TcLayout<64, 32>::SMEM, st>>>(cfg);
    else k_upd_tc<32, 32><<<grid, 192, TcLayout<32, 32>::SMEM, st>>>(cfg);
  } else if (cfg.ks <= 64) {
    if (wide) k_upd_tc<64, 64><<<grid, 192, TcLayout<64, 64>::SMEM, st>>>(cfg);
    else k_upd_tc<32, 64><<<grid, 192, TcLayout<32, 64>::SMEM, st>>>(cfg);
  } else {
    k_upd_tc<32, 128><<<grid, 192, TcLayout<32, 128>::SMEM, st>>>(cfg);
  }
}

// Tensor maps of walker wi, spin sp: A operand, B operand, N of parity 0 and
// 1 (FP32, 128-byte swizzle, boxes of 32 columns).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

static bool encode_2d(TmapDev* out, void* base, uint64_t cols, uint64_t rows, uint64_t row_bytes, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {32u, box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  static_assert(sizeof(TmapDev) == sizeof(CUtensorMap), "tensor map size");
  return fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP16 digit planes of the sliced recompute residual: `rows` rows of `cols`
// FP16 values (row pitch cols * 2 bytes), boxes of 64 values (128 bytes) x
// box_rows.
static bool encode_2d_f16(TmapDev* out, void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {64u, box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int ext_tile_c(int ks) { return ks <= 64 ? 64 : 128; }

bool encode_update_maps(const WalkerDev& w, int ks, int upd_bn, TmapDev* out) {
  const uint64_t C = (uint64_t)w.cap;
  const uint32_t bn = (uint32_t)tc_tile_n(ks, upd_bn);
  for (int sp = 0; sp < 2; ++sp) {
    TmapDev* m = out + TMAPS_PER_SPIN * sp;
    if (!encode_2d(m + 0, w.Aop[sp], TC_KS, 2 * C, TC_KS * 4, TC_BM)) return false;
    if (!encode_2d(m + 1, w.Bop[sp], TC_KS, 2 * C, TC_KS * 4, bn)) return false;
    for (int par = 0; par < 2; ++par)
      if (!encode_2d(m + 2 + par, w.N[par][sp], C, C, C * 4, TC_BM)) return false;
    // candidate table V of the tensor-core extension: [hi | lo] x KS_MAX rows x C columns,
    // in the update-operand buffer (free during the extension)
    if (!encode_2d(m + 4, w.Aop[sp], C, 2 * (uint64_t)KS_MAX, C * 4, (uint32_t)ext_tile_c(ks))) return false;
    // candidate table U ([hi | lo] x KS_MAX rows x C columns, in the other
    // operand buffer), boxes of the candidate tile's rows
    if (!encode_2d(m + 5, w.Bop[sp], C, 2 * (uint64_t)KS_MAX, C * 4, (uint32_t)ext_tile_c(ks))) return false;
    for (int par = 0; par < 2; ++par)
      if (!encode_2d(m + 6 + par, w.N[par][sp], C, C, C * 4, 32u)) return false;
    // digit planes of the sliced recompute residual: N (4 planes, 128-row
    // boxes, the MMA's M side) and A (5 planes, 64-row boxes)
    if (w.OzN[sp] && !encode_2d_f16(m + 8, w.OzN[sp], C, 4 * C, 128u)) return false;
    if (w.OzA[sp] && !encode_2d_f16(m + 9, w.OzA[sp], C, 5 * C, 64u)) return false;
  }
  return true;
}

}  // namespace dca
