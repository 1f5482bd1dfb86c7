// k_aux.cu -- initial configuration, from-scratch recomputation of N,
// measurement of G(tau), and the isolated-cluster G0 builder.
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace dca {

// ---------------------------------------------------------------------------
// Initial configuration: n0 random interacting vertices (App. B,
// "initial-configuration-size"), counter tag 2, vertex i <- counter (i, 0, 2, 0).
// ---------------------------------------------------------------------------
__global__ void k_init_vertices(Config cfg, int n0) {
  WalkerDev& w = cfg.W[blockIdx.x];
  const ProblemDev& pb = cfg.P[w.problem];
  for (int i = threadIdx.x; i < n0; i += blockDim.x) {
    const Philox4 r = draw(w, (uint64_t)i, TAG_INIT);
    w.vs[0][i] = (r.v[0] & 2u) ? 1 : -1;
    w.vsite[0][i] = (int)scaled_index(r.v[1], (uint32_t)pb.nc);
    w.vtau[0][i] = pb.beta * uniform53(r.v[2], r.v[3]);
  }
  for (int i = threadIdx.x; i < n0; i += blockDim.x) w.live_idx[i] = i;
  if (threadIdx.x == 0) {
    w.n = n0;
    w.n_live = n0;
    w.n_dead = 0;
    w.compact_pending = 0;
    w.parity = 0;
  }
}

// A = e^V - g0 (e^V - 1) for the current vertex list (all live: the
// recompute runs right after a compaction), in FP64.  The FP64 work matrix
// is N[dst][sp] itself for FP64 storage and Ascr[sp] for FP32 storage.
// mode 0: dst = current parity (initial build); mode 1: dst = other parity
// (periodic recompute, only walkers with recompute_pending).
// mode 0: every walker (initial build, rebuild after a checkpoint load);
// mode 1: walkers with a periodic recompute in this window (into the other
// buffer); mode 2: walkers whose bare propagator changed (in place).
__device__ __forceinline__ bool wants_build(const WalkerDev& w, int mode) {
  if (mode == 0) return true;
  if (mode == 2) return w.rebuild_pending && w.status == ST_OK;
  return w.active && w.recompute_pending && w.status == ST_OK;
}

__device__ __forceinline__ double* work_matrix(const Config& cfg, const WalkerDev& w, int mode, int sp) {
  if (cfg.prec == PREC_MIXED) return w.Ascr[sp];
  return (double*)w.N[mode == 1 ? w.parity ^ 1 : w.parity][sp];
}

// Persistent grid; one item = 256 entries of one walker-spin's A.
__global__ void __launch_bounds__(256) k_build_A(Config cfg, int mode) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *cfg.gj_next = 0;  // work queue of the inverse that follows
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return wants_build(w, mode) ? blocks_of((long long)w.n * w.n, 256) : 0;
      },
      [&](int s, int item) {
  const WalkerDev& w = cfg.W[s >> 1];
  const int sp = s & 1;
  const int n = w.n, ld = w.cap, par = w.parity;
  const ProblemDev& pb = cfg.P[w.problem];
  double* A = work_matrix(cfg, w, mode, sp);
  const int* vsite = w.vsite[par];
  const double* vtau = w.vtau[par];
  const int* vs = w.vs[par];
  const long long idx = (long long)item * 256 + threadIdx.x;
  if (idx < (long long)n * n) {
    const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
    const double ej = expV(pb, sp, vs[j]);
    const double g = (i == j) ? g0_diag(pb, sp, vsite[i]) : g0_pair(pb, sp, vsite[i], vtau[i], vsite[j], vtau[j]);
    const double a = (i == j ? ej : 0.0) - g * (ej - 1.0);
    if (mode == 1 && cfg.prec == PREC_MIXED && !cfg.recompute_gj) {
      // Newton recompute: A as an unevaluated FP32 pair hi + lo (~48 bits)
      const float hi = (float)a;
      reinterpret_cast<float2*>(A)[(size_t)i * ld + j] = make_float2(hi, (float)(a - (double)hi));
    } else {
      A[(size_t)i * ld + j] = a;
    }
  }
      });
}

static int grid_for(long long items) { return sm_grid(items, 4); }

// Initial build finish: sign of prod_sigma det N_sigma^-1.
__global__ void k_init_finish(Config cfg, const int* sgn) {
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= cfg.n_walkers) return;
  WalkerDev& w = cfg.W[wi];
  if (w.n == 0) {
    w.sign = 1.0;
    return;
  }
  const int s = sgn[2 * wi] * sgn[2 * wi + 1];
  if (s == 0) set_status(w, ST_ERR_NUMERIC);
  w.sign = s < 0 ? -1.0 : 1.0;
}

// FP32 storage: round the FP64 inverse into the destination buffer.
// grid = (blocks, walkers*2)
__global__ void __launch_bounds__(256) k_store_fp32(Config cfg, int mode) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return (wants_build(w, mode) && w.status == ST_OK) ? blocks_of((long long)w.n * w.n, 256) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap;
        const double* A = w.Ascr[sp];
        float* N = (float*)w.N[mode == 1 ? w.parity ^ 1 : w.parity][sp];
        const long long idx = (long long)item * 256 + threadIdx.x;
        if (idx < (long long)n * n) {
          const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
          N[(size_t)i * ld + j] = (float)A[(size_t)i * ld + j];
        }
      });
}

// Drift of the updated N against the fresh inverse: max |N_old - N_new| and
// max |N_new| over both spins, reduced per block and folded in with atomicMax
// on the bit patterns (non-negative doubles order like their bits).
// Persistent grid over walker-spin pairs, 2048 entries per item.
template <typename T>
__global__ void __launch_bounds__(256) k_recompute_drift(Config cfg) {
  __shared__ double s_d[8], s_n[8];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return (w.active && w.recompute_pending && w.status == ST_OK) ? blocks_of((long long)w.n * w.n, 2048) : 0;
      },
      [&](int s, int item) {
        WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap, par = w.parity;
        const T* Nold = (const T*)w.N[par][sp];
        const T* Nnew = (const T*)w.N[par ^ 1][sp];
        double dmax = 0.0, nmax = 0.0;
        const long long e0 = (long long)item * 2048, e1 = min(e0 + 2048, (long long)n * n);
        for (long long idx = e0 + threadIdx.x; idx < e1; idx += 256) {
          const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
          const double a = ldN(Nold, (size_t)i * ld + j), b = ldN(Nnew, (size_t)i * ld + j);
          dmax = fmax(dmax, fabs(a - b));
          nmax = fmax(nmax, fabs(b));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
          nmax = fmax(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
          s_d[threadIdx.x >> 5] = dmax;
          s_n[threadIdx.x >> 5] = nmax;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double d = 0.0, m = 0.0;
          for (int k = 0; k < 8; ++k) {
            d = fmax(d, s_d[k]);
            m = fmax(m, s_n[k]);
          }
          atomicMax(&w.drift_bits[0], (unsigned long long)__double_as_longlong(d));
          atomicMax(&w.drift_bits[1], (unsigned long long)__double_as_longlong(m));
        }
        __syncthreads();
      });
}

// Adopt the fresh inverse: copy the vertex list to the other buffer, switch
// the parity, log the relative drift.  grid = walkers, block 256.
__global__ void __launch_bounds__(256) k_recompute_adopt(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  if (!(w.active && w.recompute_pending && w.status == ST_OK)) return;
  const int n = w.n, par = w.parity;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    w.vsite[par ^ 1][i] = w.vsite[par][i];
    w.vtau[par ^ 1][i] = w.vtau[par][i];
    w.vs[par ^ 1][i] = w.vs[par][i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double d = __longlong_as_double((long long)w.drift_bits[0]);
    const double m = __longlong_as_double((long long)w.drift_bits[1]);
    const double rel = m > 0.0 ? d / m : 0.0;
    if (rel > w.max_drift) w.max_drift = rel;
    w.drift_bits[0] = 0ull;
    w.drift_bits[1] = 0ull;
    w.parity = par ^ 1;
    w.n_recomputes++;
    w.rec_flops += 2.0 * 2.0 * (double)n * (double)n * (double)n;
    w.recompute_pending = 0;
  }
}

// ---------------------------------------------------------------------------
// Measurement on the tau grid (after a post-warm-up sweep):
//   G(dr, tau_a) = g0(dr, tau_a) + (1/Nc) sum_{r'} sum_i g0(r'+dr - r_i, tau_a - tau_i) b_i(r'),
//   b_i(r') = (e^{V_i} - 1) sum_j N_ij g0(r_j - r', tau_j),
// accumulated as sign * (-G) in the paper's convention.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool wants_measure(const WalkerDev& w) { return w.active && w.measure_pending; }

// gR[sp][r'][j] = g0_sp(r_j - r', tau_j - 0+) ; grid = (blocks, walkers*2)
__global__ void __launch_bounds__(256) k_meas_gr(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return wants_measure(w) ? blocks_of((long long)cfg.P[w.problem].nc * w.n, 256) : 0;
      },
      [&](int s, int item) {
  const WalkerDev& w = cfg.W[s >> 1];
  const int sp = s & 1;
  const ProblemDev& pb = cfg.P[w.problem];
  const int n = w.n, par = w.parity, nc = pb.nc;
  const int total = nc * n;
  const int idx = item * 256 + threadIdx.x;
  if (idx < total) {
    const int rp = idx / n, j = idx - rp * n;
    const bool live = w.vs[par][j] != 0;  // a dead column of N is e_j: no contribution
    const size_t o = ((size_t)sp * nc + rp) * w.cap + j;
    if (cfg.prec == PREC_MIXED) {
      float g = 0.0f;
      if (live) {
        const int d = __ldg(pb.site_sub + w.vsite[par][j] * nc + rp);
        g = g0_interp_grid(g0f_row(pb, sp, d), pb.n_tau, grid_time(w.vtau[par][j], pb.tau_scale), GridTime{0, 0.0f});
      }
      reinterpret_cast<float*>(w.gR)[o] = g;
    } else {
      w.gR[o] = live ? g0_pair(pb, sp, w.vsite[par][j], w.vtau[par][j], rp, 0.0) : 0.0;
    }
  }
      });
}

// bvec[sp][r'][i] = (e^{V_i} - 1) sum_j N[i][j] gR[sp][r'][j]; one warp per (i, r').
// b[r'][i] = (e^{V_i} - 1) sum_j N[i][j] gR[r'][j] as a tiled product:
// a warp owns R rows of N (R = 4 for nc <= 8, 2 for nc <= 16, else 1), each
// row on 32 / R lanes that own the reference sites r' (and r' + 32 for
// nc > 32); one item = the 8 R rows of the block's warps; chunks of 32 columns
// of N and gR are staged in shared memory.
__device__ __forceinline__ int meas_b_rows(int nc) { return nc <= 8 ? 4 : (nc <= 16 ? 2 : 1); }

template <typename T, typename A>
__global__ void __launch_bounds__(256) k_meas_b(Config cfg) {
  __shared__ A sN[32][33];
  __shared__ A sG[64][33];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return wants_measure(w) ? blocks_of(w.n, 8 * meas_b_rows(cfg.P[w.problem].nc)) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1;
        const ProblemDev& pb = cfg.P[w.problem];
        const int n = w.n, par = w.parity, nc = pb.nc, ld = w.cap;
        const T* N = (const T*)w.N[par][sp];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int R = meas_b_rows(nc), lw = 32 / R;
        const int sub = lane / lw, rp = lane - sub * lw;  // row of the warp, reference site
        const int i0 = item * 8 * R + warp * R;           // first row of the warp
        const int i = i0 + sub;
        // products summed in A within a chunk of 32 columns, chunk sums in FP64
        // (the rounding of a long FP32 sum would otherwise grow with n)
        double tot0 = 0.0, tot1 = 0.0;
        const bool two = nc > 32;  // uniform: the second reference-site half exists (R = 1)
        for (int j0 = 0; j0 < n; j0 += 32) {
          A acc0 = (A)0, acc1 = (A)0;
          __syncthreads();
          {
            const int j = j0 + lane;
            for (int r = 0; r < R; ++r)
              sN[warp * R + r][lane] = (i0 + r < n && j < n) ? ldA<A>(N, (size_t)(i0 + r) * ld + j) : (A)0;
          }
          for (int e = threadIdx.x; e < (two ? 64 : lw) * 32; e += 256) {
            const int q = e >> 5, jl = e & 31, j = j0 + jl;
            sG[q][jl] = (q < nc && j < n) ? reinterpret_cast<const A*>(w.gR)[((size_t)sp * nc + q) * ld + j] : (A)0;
          }
          __syncthreads();
          if (two) {
#pragma unroll 8
            for (int jl = 0; jl < 32; ++jl) {
              const A nij = sN[warp][jl];
              acc0 += nij * sG[lane][jl];
              acc1 += nij * sG[lane + 32][jl];
            }
          } else {
            const int row = warp * R + sub;
#pragma unroll 8
            for (int jl = 0; jl < 32; ++jl) acc0 += sN[row][jl] * sG[rp][jl];
          }
          tot0 += (double)acc0;
          tot1 += (double)acc1;
        }
        if (i < n) {
          const double f = expV(pb, sp, w.vs[par][i]) - 1.0;
          A* bv = reinterpret_cast<A*>(w.bvec);
          if (rp < nc) bv[((size_t)sp * nc + rp) * ld + i] = (A)(f * tot0);
          if (two && rp + 32 < nc) bv[((size_t)sp * nc + rp + 32) * ld + i] = (A)(f * tot1);
        }
      });
}

// Correction term as a product: rows (x, tau_a), inner index the vertex i,
// columns the reference site r':
//   C[(x, a), r'] = sum_i g0(x - r_i, tau_a - tau_i) b_i(r'),
// scattered to Gtmp[sp][x - r'][a] (FP64 atomics).  The g0 factor is
// interpolated on the fly (FP64 path: FP64; mixed path: FP32 on the split
// grid time, with the tau_a and tau_i grid times formed once per tile).  A is
// the arithmetic type of the products, MR >= nc the reference-site tile.
// Item = (site x, block of MT tau points) of one walker-spin, block 256.
constexpr int MT = 64;   // tau points per item
constexpr int MK = 32;   // vertices per step

template <typename A, int MR>
__device__ __forceinline__ void meas_gemm_item(const Config& cfg, int wi, int sp, int item);

// One kernel per reference-site tile MR, each taking the walkers whose
// cluster falls in its class (MR / 2 < nc <= MR; nc <= 16 for MR = 16): the
// register allocation of each follows its own tile.
template <typename A, int MR>
__global__ void __launch_bounds__(256) k_meas_gemm(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        const int nc = cfg.P[w.problem].nc;
        const bool mine = MR == 16 ? nc <= 16 : (nc > MR / 2 && nc <= MR);
        return (wants_measure(w) && mine) ? (long long)nc * blocks_of(cfg.n_tau_meas, MT) : 0;
      },
      [&](int s, int item) { meas_gemm_item<A, MR>(cfg, s >> 1, s & 1, item); });
}

// Item = (reference site x, MT tau points): the tiles of MK vertices pass
// through shared memory.  On the FP32 path in two stages: while the tile t
// is multiplied, the table values of tile t + 1 are filled in and the vertex
// records of tile t + 2 prepared, one barrier per tile; the FP64 path keeps
// one stage (its tiles would not fit twice in static shared memory).
template <typename A, int MR>
__device__ __forceinline__ void meas_gemm_item(const Config& cfg, int wi, int sp, int item) {
  constexpr bool kGrid = sizeof(A) == 4;
  constexpr int NS = kGrid ? 2 : 1;  // stages
  const WalkerDev& w = cfg.W[wi];
  const ProblemDev& pb = cfg.P[w.problem];
  const int nc = pb.nc, ntm = cfg.n_tau_meas, n = w.n, par = w.parity, ld = w.cap;
  const int tblocks = (ntm + MT - 1) / MT;
  const int x = item / tblocks, a0 = (item - x * tblocks) * MT;
  __shared__ A As[NS][MT][MK + 1];
  __shared__ __align__(16) A Bs[NS][MK][MR];  // rows of MR values: a thread's MR / 4 sites are contiguous
  __shared__ GridTime s_ga[MT], s_gi[NS][MK];
  __shared__ int s_row[NS][MK];               // table row of g0(x - r_i, .), -1 for a dead vertex
  __shared__ int s_ph[NS][MK], s_mb[NS][MK];  // phase-table path: phase p_i and m offset of vertex i
  __shared__ float s_fw[NS][MK];              // and its interpolation weight
  const int q = kGrid ? pb.meas_q : 0;
  const int tid = threadIdx.x;
  const int ta = tid & (MT - 1), tr = tid >> 6;  // 4 groups of reference sites
  // products summed in A within a tile of MK vertices; the tile sums in FP64
  // (FP64 path) or in double-float (FP32 path: an error-free FP32 two-sum per
  // tile instead of a conversion and an add on GB300's scarce FP64 units)
  double tot[MR / 4];
  float th[MR / 4], tl[MR / 4];
#pragma unroll
  for (int m = 0; m < MR / 4; ++m) {
    tot[m] = 0.0;
    th[m] = tl[m] = 0.0f;
  }
  const int* vsite = w.vsite[par];
  const double* vtau = w.vtau[par];
  const int* vs = w.vs[par];
  const int np1 = pb.n_tau + 1;
  const double* row_base = pb.g0 + (size_t)sp * nc * np1;

  // vertex records of the tile at i0 into stage b (threads tid < MK)
  auto prep = [&](int i0, int b) {
    if (tid < MK) {
      const int i = i0 + tid;
      const bool live = i < n && vs[i] != 0;
      s_row[b][tid] = live ? __ldg(pb.site_sub + x * nc + vsite[i]) : -1;
      if (kGrid && live) {
        const GridTime gi = grid_time(vtau[i], pb.tau_scale);
        s_gi[b][tid] = gi;
        if (q > 0) {
          // grid offset of tau_a - tau_i: l = q a + c, c = q/2 - gi.i - (gi.f > 0), weight 1 - gi.f
          const int c = q / 2 - gi.i - (gi.f > 0.0f ? 1 : 0);
          const int p = ((c % q) + q) % q;
          s_ph[b][tid] = p;
          s_mb[b][tid] = (c - p) / q;
          s_fw[b][tid] = gi.f > 0.0f ? 1.0f - gi.f : 0.0f;
        }
      }
    }
  };
  // table values g0(x - r_i, tau_a - tau_i) and the rows b_i of the tile at i0 into stage b
  auto fill = [&](int i0, int b) {
    if (q > 0) {
      // phase table: consecutive threads take consecutive tau points of one
      // vertex, i.e. consecutive entries of one phase row
      const size_t mrow = (size_t)ntm + 1;
      const float* gm = pb.g0m + (size_t)sp * q * nc * mrow;
      for (int e = tid; e < MT * MK; e += 256) {
        const int il = e / MT, al = e - il * MT;
        const int a = a0 + al, d = s_row[b][il];
        A v = (A)0;
        if (a < ntm && d >= 0) {
          const int p = s_ph[b][il];
          int m = a + s_mb[b][il];
          float sgn = 1.0f;
          if (m < 0) {  // tau_a - tau_i < 0: antiperiodic continuation
            m += ntm;
            sgn = -1.0f;
          }
          const float lo = __ldg(gm + ((size_t)p * nc + d) * mrow + m);
          const float hi = p + 1 < q ? __ldg(gm + ((size_t)(p + 1) * nc + d) * mrow + m)
                                     : __ldg(gm + (size_t)d * mrow + m + 1);
          v = (A)(sgn * (lo + s_fw[b][il] * (hi - lo)));
        }
        As[b][al][il] = v;
      }
    } else {
      for (int e = tid; e < MT * MK; e += 256) {
        const int al = e / MK, il = e - al * MK;
        const int a = a0 + al, d = s_row[b][il];
        A v = (A)0;
        if (a < ntm && d >= 0) {
          const double* row = row_base + (size_t)d * np1;
          if (kGrid) {
            v = (A)g0_interp_grid(g0f_row(pb, sp, d), pb.n_tau, s_ga[al], s_gi[b][il]);
          } else {
            const double ta_ = ((double)a + 0.5) * pb.beta / (double)ntm;
            v = (A)g0_interp(row, pb.n_tau, pb.beta, pb.tau_scale, ta_ - vtau[i0 + il]);
          }
        }
        As[b][al][il] = v;
      }
    }
    for (int e = tid; e < MK * MR; e += 256) {
      const int il = e / MR, rp = e - il * MR;
      const int i = i0 + il;
      Bs[b][il][rp] = (i < n && rp < nc) ? reinterpret_cast<const A*>(w.bvec)[((size_t)sp * nc + rp) * ld + i] : (A)0;
    }
  };
  // products of stage b, added to the tile sums
  auto compute = [&](int b) {
    A acc[MR / 4];
#pragma unroll
    for (int m = 0; m < MR / 4; ++m) acc[m] = (A)0;
#pragma unroll 4
    for (int k = 0; k < MK; ++k) {
      const A g = As[b][ta][k];
      // sites MR/4 tr .. MR/4 tr + MR/4 - 1: the same row segment for the whole
      // warp (a broadcast), read as 16-byte vectors on the FP32 path
      if constexpr (sizeof(A) == 4) {
#pragma unroll
        for (int m4 = 0; m4 < MR / 16; ++m4) {
          const float4 bv = *reinterpret_cast<const float4*>(&Bs[b][k][tr * (MR / 4) + 4 * m4]);
          acc[4 * m4] += g * bv.x;
          acc[4 * m4 + 1] += g * bv.y;
          acc[4 * m4 + 2] += g * bv.z;
          acc[4 * m4 + 3] += g * bv.w;
        }
      } else {
#pragma unroll
        for (int m = 0; m < MR / 4; ++m) acc[m] += g * Bs[b][k][tr * (MR / 4) + m];
      }
    }
    if constexpr (sizeof(A) == 4) {
#pragma unroll
      for (int m = 0; m < MR / 4; ++m) {
        const float s1 = __fadd_rn(th[m], (float)acc[m]);
        const float bb = __fsub_rn(s1, th[m]);
        tl[m] += __fadd_rn(__fsub_rn(th[m], __fsub_rn(s1, bb)), __fsub_rn((float)acc[m], bb));
        th[m] = s1;
      }
    } else {
#pragma unroll
      for (int m = 0; m < MR / 4; ++m) tot[m] += (double)acc[m];
    }
  };

  __syncthreads();  // the previous item of this block is done with the shared tiles
  if (kGrid && tid < MT) s_ga[tid] = grid_time(((double)(a0 + tid) + 0.5) * pb.beta / (double)ntm, pb.tau_scale);
  if constexpr (NS == 2) {
    if (n > 0) {
      prep(0, 0);
      if (MK < n) prep(MK, 1);
      __syncthreads();
      fill(0, 0);
      __syncthreads();
      for (int i0 = 0, t = 0; i0 < n; i0 += MK, ++t) {
        const int b = t & 1;
        if (i0 + MK < n) fill(i0 + MK, b ^ 1);     // reads the records of stage b ^ 1
        compute(b);
        if (i0 + 2 * MK < n) prep(i0 + 2 * MK, b);  // stage b's records were read one tile ago
        __syncthreads();
      }
    }
  } else {
    for (int i0 = 0; i0 < n; i0 += MK) {
      __syncthreads();
      prep(i0, 0);
      __syncthreads();
      fill(i0, 0);
      __syncthreads();
      compute(0);
    }
  }
  const int a = a0 + ta;
  if (a < ntm) {
#pragma unroll
    for (int m = 0; m < MR / 4; ++m) {
      const int rp = tr * (MR / 4) + m;
      if (rp < nc) {
        const int d = __ldg(pb.site_sub + x * nc + rp);
        const double v = sizeof(A) == 4 ? (double)th[m] + (double)tl[m] : tot[m];
        atomicAdd(&w.Gtmp[((size_t)sp * nc + d) * ntm + a], v);
      }
    }
  }
}

// Gacc[sp][dr][a] += sign * (-G), G = g0(dr, tau_a) + Gtmp / Nc; Gtmp cleared.
// grid = (blocks, walkers), thread per (sp, dr, a).
__global__ void __launch_bounds__(256) k_meas_acc(Config cfg) {
  for_each_item(
      cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s];
        return wants_measure(w) ? blocks_of(2LL * cfg.P[w.problem].nc * cfg.n_tau_meas, 256) : 0;
      },
      [&](int s, int item) {
  WalkerDev& w = cfg.W[s];
  const ProblemDev& pb = cfg.P[w.problem];
  const int nc = pb.nc, ntm = cfg.n_tau_meas;
  const int total = 2 * nc * ntm;
  const double sign = w.sign;
  const int idx = item * 256 + threadIdx.x;
  if (idx < total) {
    const int sp = idx / (nc * ntm);
    const int rem = idx - sp * nc * ntm;
    const int d = rem / ntm, a = rem - d * ntm;
    const double ta = ((double)a + 0.5) * pb.beta / (double)ntm;
    const double* row = pb.g0 + ((size_t)sp * nc + d) * (size_t)(pb.n_tau + 1);
    const double G = g0_interp(row, pb.n_tau, pb.beta, pb.tau_scale, ta) + w.Gtmp[idx] / (double)nc;
    w.Gtmp[idx] = 0.0;
    w.Gacc[idx] += sign * (-G);
  }
      });
}

__global__ void k_meas_finish(Config cfg) {
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= cfg.n_walkers) return;
  WalkerDev& w = cfg.W[wi];
  if (!wants_measure(w)) return;
  w.sign_sum += w.sign;
  w.n_meas++;
  w.k_sum += w.sign * (double)w.n_live;
  w.measure_pending = 0;
}

// ---------------------------------------------------------------------------
// Isolated-cluster G0 (paper convention) on the tau grid:
//   G0(r, tau_l) = -(1/Nc) sum_K cos(K.r) e^{-tau xi_K} / (1 + e^{-beta xi_K})
// ---------------------------------------------------------------------------
__global__ void k_g0_isolated(int nc, const double* eps, const double* kr, double mu_eff, double beta, int n_tau,
                              double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = nc * (n_tau + 1);
  if (idx >= m) return;
  const int r = idx / (n_tau + 1), l = idx - r * (n_tau + 1);
  const double tau = (double)l * beta / (double)n_tau;
  double acc = 0.0;
  for (int k = 0; k < nc; ++k) {
    const double xi = eps[k] - mu_eff;
    double f;
    if (xi >= 0.0) f = exp(-tau * xi) / (1.0 + exp(-beta * xi));
    else f = exp((beta - tau) * xi) / (exp(beta * xi) + 1.0);
    acc += cos(kr[(size_t)k * nc + r]) * f;
  }
  const double v = -acc / (double)nc;
  out[idx] = v;
  out[m + idx] = v;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
void launch_init(const Config& cfg, int n0, int max_cap, int* d_sgn, cudaStream_t st) {
  const int W = cfg.n_walkers;
  k_init_vertices<<<W, 256, 0, st>>>(cfg, n0);
  if (n0 > 0) {
    const long long g = grid_for(2LL * W * blocks_of((long long)n0 * n0, 256));
    k_build_A<<<g, 256, 0, st>>>(cfg, 0);
    launch_gj(cfg, 0, n0, d_sgn, st);
    if (cfg.prec == PREC_MIXED) k_store_fp32<<<g, 256, 0, st>>>(cfg, 0);
  }
  k_init_finish<<<(W + 127) / 128, 128, 0, st>>>(cfg, d_sgn);
  (void)max_cap;
}

int launch_recompute(int part, const Config& cfg, int max_cap, int* d_sgn, cudaStream_t st) {
  const int W = cfg.n_walkers;
  const int g = grid_for(2LL * W * blocks_of((long long)max_cap * max_cap, 256));
  const int gd = grid_for(2LL * W * blocks_of((long long)max_cap * max_cap, 2048));
  switch (part) {
    case GROUP_RECOMPUTE_PRE:
      k_build_A<<<g, 256, 0, st>>>(cfg, 1);
      return 1;
    case GROUP_RECOMPUTE:
      if (cfg.prec == PREC_MIXED && !cfg.recompute_gj) {
        if (cfg.recompute_oz) {
          launch_refine_oz(cfg, max_cap, st);
          launch_refine_correct(cfg, max_cap, st);
          return 5;
        }
        launch_refine_gemms(cfg, max_cap, st);
        return 2;
      }
      launch_gj(cfg, 1, max_cap, d_sgn, st);
      return 1;
    case GROUP_RECOMPUTE_POST:
      if (cfg.prec == PREC_MIXED && !cfg.recompute_gj) {
        launch_refine_adopt(cfg, max_cap, st);
        k_recompute_adopt<<<W, 256, 0, st>>>(cfg);
        return 2;
      }
      if (cfg.prec == PREC_MIXED) {
        k_store_fp32<<<g, 256, 0, st>>>(cfg, 1);
        k_recompute_drift<float><<<gd, 256, 0, st>>>(cfg);
        k_recompute_adopt<<<W, 256, 0, st>>>(cfg);
        return 3;
      }
      k_recompute_drift<double><<<gd, 256, 0, st>>>(cfg);
      k_recompute_adopt<<<W, 256, 0, st>>>(cfg);
      return 2;
    default:
      return 0;
  }
}

// Rebuild every walker's N from scratch for the vertex list in its current
// buffer (after a checkpoint load), with the configuration sign from the
// determinants, exactly as the initial build does.
void launch_rebuild(const Config& cfg, int max_n, int* d_sgn, cudaStream_t st) {
  const int W = cfg.n_walkers;
  if (max_n > 0) {
    const long long g = grid_for(2LL * W * blocks_of((long long)max_n * max_n, 256));
    k_build_A<<<g, 256, 0, st>>>(cfg, 0);
    launch_gj(cfg, 0, max_n, d_sgn, st);
    if (cfg.prec == PREC_MIXED) k_store_fp32<<<g, 256, 0, st>>>(cfg, 0);
  }
  k_init_finish<<<(W + 127) / 128, 128, 0, st>>>(cfg, d_sgn);
}

// From-scratch N for the vertex list held in the current buffer of every walker
// of cfg (used by the standalone fresh-N operations): build A, invert in place.
void launch_fresh_inverse(const Config& cfg, int max_n, int* d_sgn, cudaStream_t st) {
  const int W = cfg.n_walkers;
  if (max_n <= 0) return;
  k_build_A<<<grid_for(2LL * W * blocks_of((long long)max_n * max_n, 256)), 256, 0, st>>>(cfg, 0);
  launch_gj(cfg, 0, max_n, d_sgn, st);
}

// g0 = -G0 in FP64 and its FP32 copy, from a staged table, committed only if
// every staged entry is finite (else *bad is set and the old table stays);
// *changed is set if the committed table differs from the old one.
// One block: the check and the commit need one barrier between them.
__global__ void __launch_bounds__(1024) k_negate(const double* src, double* dst, float* dstf, size_t n, int* bad,
                                                 int* changed) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  int b = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) b |= isfinite(src[i]) ? 0 : 1;
  if (b) s_bad = 1;
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) *bad = 1;
    return;
  }
  int c = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    c |= dst[i] != -src[i] ? 1 : 0;
    dst[i] = -src[i];
    dstf[i] = (float)(-src[i]);
  }
  if (__syncthreads_or(c) && threadIdx.x == 0) *changed = 1;
}

void launch_negate(const double* src, double* dst, float* dstf, size_t n, int* bad, int* changed, cudaStream_t st) {
  k_negate<<<1, 1024, 0, st>>>(src, dst, dstf, n, bad, changed);
}

// Walkers of a problem whose table changed: N rebuilt from scratch in place
// (the inverse of e^V - g0 (e^V - 1) for the new g0), with the configuration
// sign from the determinants.
__global__ void k_mark_rebuild(Config cfg, const int* changed) {
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= cfg.n_walkers) return;
  WalkerDev& w = cfg.W[wi];
  w.rebuild_pending = (changed[w.problem] && w.n > 0 && w.status == ST_OK) ? 1 : 0;
}

__global__ void k_rebuild_finish(Config cfg, const int* sgn) {
  const int wi = blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= cfg.n_walkers) return;
  WalkerDev& w = cfg.W[wi];
  if (!w.rebuild_pending) return;
  w.rebuild_pending = 0;
  const int s = sgn[2 * wi] * sgn[2 * wi + 1];
  if (s == 0) set_status(w, ST_ERR_NUMERIC);
  w.sign = s < 0 ? -1.0 : 1.0;
}

int launch_rebuild_changed(const Config& cfg, int max_cap, const int* changed, int* d_sgn, cudaStream_t st) {
  const int W = cfg.n_walkers;
  k_mark_rebuild<<<(W + 127) / 128, 128, 0, st>>>(cfg, changed);
  const long long g = grid_for(2LL * W * blocks_of((long long)max_cap * max_cap, 256));
  k_build_A<<<g, 256, 0, st>>>(cfg, 2);
  launch_gj(cfg, 2, max_cap, d_sgn, st);
  if (cfg.prec == PREC_MIXED) k_store_fp32<<<g, 256, 0, st>>>(cfg, 2);
  k_rebuild_finish<<<(W + 127) / 128, 128, 0, st>>>(cfg, d_sgn);
  return cfg.prec == PREC_MIXED ? 5 : 4;
}

// g0m[sp][p][d][m] = g0f[sp][d][q m + p] for q m + p <= n_tau, else 0.
__device__ __forceinline__ float meas_table_entry(const float* g0f, int nc, int n_tau, int q, int ntm, size_t e) {
  const int m = (int)(e % (ntm + 1));
  size_t r = e / (ntm + 1);
  const int d = (int)(r % nc);
  r /= nc;
  const int p = (int)(r % q), sp = (int)(r / q);
  const int l = q * m + p;
  return l <= n_tau ? g0f[((size_t)sp * nc + d) * (n_tau + 1) + l] : 0.0f;
}

__global__ void k_meas_table(const float* g0f, float* g0m, int nc, int n_tau, int q, int ntm) {
  const size_t total = (size_t)2 * q * nc * (ntm + 1);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    g0m[e] = meas_table_entry(g0f, nc, n_tau, q, ntm, e);
}

void launch_meas_table(const ProblemDev& pd, int n_tau_meas, cudaStream_t st) {
  const size_t total = (size_t)2 * pd.meas_q * pd.nc * (n_tau_meas + 1);
  const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 4096);
  k_meas_table<<<blocks, 256, 0, st>>>(pd.g0f, const_cast<float*>(pd.g0m), pd.nc, pd.n_tau, pd.meas_q, n_tau_meas);
}

// All problems at once: the staged tables lie back to back (problem p at
// off[p], 2 nc (n_tau + 1) entries).  Check: bad[p] = 1 (and *bad_any = 1) if a
// staged entry of problem p is not finite; commit: g0 = -G0 and its FP32
// copy for every problem with bad[p] == 0; then the measurement phase tables.
__global__ void k_g0_check_all(const ProblemDev* P, int np, const double* stage, const long long* off, int* bad,
                               int* bad_any) {
  const int p = blockIdx.y;
  if (p >= np) return;
  const long long n = 2LL * P[p].nc * (P[p].n_tau + 1);
  const double* src = stage + off[p];
  int b = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b |= isfinite(src[i]) ? 0 : 1;
  if (__syncthreads_or(b) && threadIdx.x == 0) {
    bad[p] = 1;
    *bad_any = 1;
  }
}

__global__ void k_g0_commit_all(const ProblemDev* P, int np, const double* stage, const long long* off,
                                const int* bad, int* changed) {
  const int p = blockIdx.y;
  if (p >= np || bad[p]) return;
  const long long n = 2LL * P[p].nc * (P[p].n_tau + 1);
  const double* src = stage + off[p];
  double* dst = const_cast<double*>(P[p].g0);
  float* dstf = const_cast<float*>(P[p].g0f);
  int c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    c |= dst[i] != -src[i] ? 1 : 0;
    dst[i] = -src[i];
    dstf[i] = (float)(-src[i]);
  }
  if (__syncthreads_or(c) && threadIdx.x == 0) changed[p] = 1;
}

__global__ void k_meas_table_all(const ProblemDev* P, int np, int ntm, const int* bad) {
  const int p = blockIdx.y;
  if (p >= np || bad[p] || P[p].meas_q <= 0) return;
  const int q = P[p].meas_q, nc = P[p].nc;
  float* g0m = const_cast<float*>(P[p].g0m);
  const size_t total = (size_t)2 * q * nc * (ntm + 1);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    g0m[e] = meas_table_entry(P[p].g0f, nc, P[p].n_tau, q, ntm, e);
}

void launch_g0_update_all(const ProblemDev* d_P, int np, int ntm, const double* stage, const long long* off, int* bad,
                          int* bad_any, int* changed, cudaStream_t st) {
  const dim3 grid(16, np);
  k_g0_check_all<<<grid, 256, 0, st>>>(d_P, np, stage, off, bad, bad_any);
  k_g0_commit_all<<<grid, 256, 0, st>>>(d_P, np, stage, off, bad, changed);
  k_meas_table_all<<<grid, 256, 0, st>>>(d_P, np, ntm, bad);
}


int launch_measure(const Config& cfg, int max_cap, int max_nc, cudaStream_t st) {
  const int W = cfg.n_walkers;
  const long long S = 2LL * W;
  k_meas_gr<<<persist_grid((const void*)k_meas_gr, S * blocks_of((long long)max_nc * max_cap, 256), 256), 256, 0,
              st>>>(cfg);
  const long long ib = S * blocks_of(max_cap, 8);
  if (cfg.prec == PREC_MIXED)
    k_meas_b<float, float><<<persist_grid((const void*)k_meas_b<float, float>, ib, 256), 256, 0, st>>>(cfg);
  else
    k_meas_b<double, double><<<persist_grid((const void*)k_meas_b<double, double>, ib, 256), 256, 0, st>>>(cfg);
  const long long ig = S * max_nc * blocks_of(cfg.n_tau_meas, MT);
#define DCA_MEAS_GEMM(A, MR) k_meas_gemm<A, MR><<<persist_grid((const void*)k_meas_gemm<A, MR>, ig, 256), 256, 0, st>>>(cfg)
  if (cfg.prec == PREC_MIXED) {
    DCA_MEAS_GEMM(float, 16);
    if (max_nc > 16) DCA_MEAS_GEMM(float, 32);
    if (max_nc > 32) DCA_MEAS_GEMM(float, 64);
  } else {
    DCA_MEAS_GEMM(double, 16);
    if (max_nc > 16) DCA_MEAS_GEMM(double, 32);
    if (max_nc > 32) DCA_MEAS_GEMM(double, 64);
  }
#undef DCA_MEAS_GEMM
  k_meas_acc<<<grid_for((long long)W * blocks_of(2LL * max_nc * cfg.n_tau_meas, 256)), 256, 0, st>>>(cfg);
  const int nf = launch_meas_nfft(cfg, max_cap, max_nc, st) + launch_meas_g4(cfg, max_cap, max_nc, st);
  k_meas_finish<<<(W + 127) / 128, 128, 0, st>>>(cfg);
  return 5 + (max_nc > 16) + (max_nc > 32) + nf;
}

// Read-out of the tau-grid measurement: every walker's accumulator Gacc
// [2][nc][n_tau_meas] to out + base[walker].  grid = (chunks, walkers).
__global__ void k_gather_G(Config cfg, const long long* base, double* out) {
  const int wi = blockIdx.y;
  const WalkerDev& w = cfg.W[wi];
  const long long total = 2LL * cfg.P[w.problem].nc * cfg.n_tau_meas;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    out[base[wi] + e] = w.Gacc[e];
}

void launch_gather_G(const Config& cfg, int max_nc, const long long* d_base, double* d_out, cudaStream_t st) {
  const long long per = 2LL * max_nc * cfg.n_tau_meas;
  const int bx = (int)((per + 255) / 256 < 64 ? (per + 255) / 256 : 64);
  k_gather_G<<<dim3(bx, cfg.n_walkers), 256, 0, st>>>(cfg, d_base, d_out);
}

void launch_g0_isolated(int nc, const double* d_eps, const double* d_kr, double mu_eff, double beta, int n_tau,
                        double* d_out, cudaStream_t st) {
  const int m = nc * (n_tau + 1);
  k_g0_isolated<<<(m + 255) / 256, 256, 0, st>>>(nc, d_eps, d_kr, mu_eff, beta, n_tau, d_out);
}

}  // namespace dca
