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
__device__ __forceinline__ bool wants_build(const WalkerDev& w, int mode) {
  return mode == 0 ? true : (w.active && w.recompute_pending && w.status == ST_OK);
}

__device__ __forceinline__ double* work_matrix(const Config& cfg, const WalkerDev& w, int mode, int sp) {
  if (cfg.prec == PREC_MIXED) return w.Ascr[sp];
  return (double*)w.N[mode == 0 ? w.parity : w.parity ^ 1][sp];
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

constexpr int PERSIST = 4 * 152;

static int grid_for(long long items) { return (int)(items < 1 ? 1 : (items < PERSIST ? items : PERSIST)); }

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
  if (s == 0) w.status = ST_ERR_NUMERIC;
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
        float* N = (float*)w.N[mode == 0 ? w.parity : w.parity ^ 1][sp];
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
// one item = 8 rows of N (one warp each); lanes own reference sites r' and
// r' + 32; chunks of 32 columns of N and gR are staged in shared memory.
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_meas_b(Config cfg) {
  __shared__ A sN[8][33];
  __shared__ A sG[64][33];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return wants_measure(w) ? blocks_of(w.n, 8) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1;
        const ProblemDev& pb = cfg.P[w.problem];
        const int n = w.n, par = w.parity, nc = pb.nc, ld = w.cap;
        const T* N = (const T*)w.N[par][sp];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int i = item * 8 + warp;
        A acc0 = (A)0, acc1 = (A)0;
        const bool two = nc > 32;  // uniform: the second reference-site half exists
        for (int j0 = 0; j0 < n; j0 += 32) {
          __syncthreads();
          {
            const int j = j0 + lane;
            sN[warp][lane] = (i < n && j < n) ? ldA<A>(N, (size_t)i * ld + j) : (A)0;
          }
          for (int e = threadIdx.x; e < (two ? 64 : 32) * 32; e += 256) {
            const int rp = e >> 5, jl = e & 31, j = j0 + jl;
            sG[rp][jl] = (rp < nc && j < n) ? reinterpret_cast<const A*>(w.gR)[((size_t)sp * nc + rp) * ld + j] : (A)0;
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
#pragma unroll 8
            for (int jl = 0; jl < 32; ++jl) acc0 += sN[warp][jl] * sG[lane][jl];
          }
        }
        if (i < n) {
          const A f = (A)(expV(pb, sp, w.vs[par][i]) - 1.0);
          A* bv = reinterpret_cast<A*>(w.bvec);
          if (lane < nc) bv[((size_t)sp * nc + lane) * ld + i] = f * acc0;
          if (lane + 32 < nc) bv[((size_t)sp * nc + lane + 32) * ld + i] = f * acc1;
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

template <typename A, int MR>
__device__ __forceinline__ void meas_gemm_item(const Config& cfg, int wi, int sp, int item) {
  const WalkerDev& w = cfg.W[wi];
  const ProblemDev& pb = cfg.P[w.problem];
  const int nc = pb.nc, ntm = cfg.n_tau_meas, n = w.n, par = w.parity, ld = w.cap;
  const int tblocks = (ntm + MT - 1) / MT;
  const int x = item / tblocks, a0 = (item - x * tblocks) * MT;
  constexpr bool kGrid = sizeof(A) == 4;
  __shared__ A As[MT][MK + 1];
  __shared__ A Bs[MK][MR + 1];
  __shared__ GridTime s_ga[MT], s_gi[MK];
  __shared__ int s_row[MK];  // table row of g0(x - r_i, .), -1 for a dead vertex
  const int tid = threadIdx.x;
  const int ta = tid & (MT - 1), tr = tid >> 6;  // 4 groups of reference sites
  A acc[MR / 4];
#pragma unroll
  for (int m = 0; m < MR / 4; ++m) acc[m] = (A)0;
  const int* vsite = w.vsite[par];
  const double* vtau = w.vtau[par];
  const int* vs = w.vs[par];
  const int np1 = pb.n_tau + 1;
  const double* row_base = pb.g0 + (size_t)sp * nc * np1;
  __syncthreads();  // the previous item of this block is done with the shared tiles
  if (kGrid && tid < MT) s_ga[tid] = grid_time(((double)(a0 + tid) + 0.5) * pb.beta / (double)ntm, pb.tau_scale);
  for (int i0 = 0; i0 < n; i0 += MK) {
    __syncthreads();
    if (tid < MK) {
      const int i = i0 + tid;
      const bool live = i < n && vs[i] != 0;
      s_row[tid] = live ? __ldg(pb.site_sub + x * nc + vsite[i]) : -1;
      if (kGrid && live) s_gi[tid] = grid_time(vtau[i], pb.tau_scale);
    }
    __syncthreads();
    for (int e = tid; e < MT * MK; e += 256) {
      const int al = e / MK, il = e - al * MK;
      const int a = a0 + al, d = s_row[il];
      A v = (A)0;
      if (a < ntm && d >= 0) {
        const double* row = row_base + (size_t)d * np1;
        if (kGrid) {
          v = (A)g0_interp_grid(g0f_row(pb, sp, d), pb.n_tau, s_ga[al], s_gi[il]);
        } else {
          const double ta_ = ((double)a + 0.5) * pb.beta / (double)ntm;
          v = (A)g0_interp(row, pb.n_tau, pb.beta, pb.tau_scale, ta_ - vtau[i0 + il]);
        }
      }
      As[al][il] = v;
    }
    for (int e = tid; e < MK * MR; e += 256) {
      const int il = e / MR, rp = e - il * MR;
      const int i = i0 + il;
      Bs[il][rp] = (i < n && rp < nc) ? reinterpret_cast<const A*>(w.bvec)[((size_t)sp * nc + rp) * ld + i] : (A)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < MK; ++k) {
      const A g = As[ta][k];
#pragma unroll
      for (int m = 0; m < MR / 4; ++m) acc[m] += g * Bs[k][tr + 4 * m];
    }
  }
  const int a = a0 + ta;
  if (a < ntm) {
#pragma unroll
    for (int m = 0; m < MR / 4; ++m) {
      const int rp = tr + 4 * m;
      if (rp < nc) {
        const int d = __ldg(pb.site_sub + x * nc + rp);
        atomicAdd(&w.Gtmp[((size_t)sp * nc + d) * ntm + a], (double)acc[m]);
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

// From-scratch N for the vertex list held in the current buffer of every walker
// of cfg (used by the standalone fresh-N operations): build A, invert in place.
void launch_fresh_inverse(const Config& cfg, int max_n, int* d_sgn, cudaStream_t st) {
  const int W = cfg.n_walkers;
  if (max_n <= 0) return;
  k_build_A<<<grid_for(2LL * W * blocks_of((long long)max_n * max_n, 256)), 256, 0, st>>>(cfg, 0);
  launch_gj(cfg, 0, max_n, d_sgn, st);
}

// g0 = -G0 in FP64 and its FP32 copy.
__global__ void k_negate(const double* src, double* dst, float* dstf, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    dst[i] = -src[i];
    dstf[i] = (float)(-src[i]);
  }
}

void launch_negate(const double* src, double* dst, float* dstf, size_t n, cudaStream_t st) {
  k_negate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, dstf, n);
}

int launch_measure(const Config& cfg, int max_cap, int max_nc, cudaStream_t st) {
  const int W = cfg.n_walkers;
  const long long S = 2LL * W;
  k_meas_gr<<<grid_for(S * blocks_of((long long)max_nc * max_cap, 256)), 256, 0, st>>>(cfg);
  const int gb = grid_for(S * blocks_of(max_cap, 8));
  if (cfg.prec == PREC_MIXED) k_meas_b<float, float><<<gb, 256, 0, st>>>(cfg);
  else k_meas_b<double, double><<<gb, 256, 0, st>>>(cfg);
  const int gg = grid_for(S * max_nc * blocks_of(cfg.n_tau_meas, MT));
  if (cfg.prec == PREC_MIXED) {
    k_meas_gemm<float, 16><<<gg, 256, 0, st>>>(cfg);
    if (max_nc > 16) k_meas_gemm<float, 32><<<gg, 256, 0, st>>>(cfg);
    if (max_nc > 32) k_meas_gemm<float, 64><<<gg, 256, 0, st>>>(cfg);
  } else {
    k_meas_gemm<double, 16><<<gg, 256, 0, st>>>(cfg);
    if (max_nc > 16) k_meas_gemm<double, 32><<<gg, 256, 0, st>>>(cfg);
    if (max_nc > 32) k_meas_gemm<double, 64><<<gg, 256, 0, st>>>(cfg);
  }
  k_meas_acc<<<grid_for((long long)W * blocks_of(2LL * max_nc * cfg.n_tau_meas, 256)), 256, 0, st>>>(cfg);
  k_meas_finish<<<(W + 127) / 128, 128, 0, st>>>(cfg);
  (void)max_cap;
  return 5 + (max_nc > 16) + (max_nc > 32);
}

void launch_g0_isolated(int nc, const double* d_eps, const double* d_kr, double mu_eff, double beta, int n_tau,
                        double* d_out, cudaStream_t st) {
  const int m = nc * (n_tau + 1);
  k_g0_isolated<<<(m + 255) / 256, 256, 0, st>>>(nc, d_eps, d_kr, mu_eff, beta, n_tau, d_out);
}

}  // namespace dca
