// k_g4.cu -- two-particle measurement of the particle-particle up-down
// channel (DCA++ paper Sec. 2.5, Eq. bse_cluster and G2^{0,pp}; App. B
// four-point type PARTICLE_PARTICLE_UP_DOWN, "four-point-fermionic-
// frequencies", "momentum-transfer", "frequency-transfer").
//
// Within one configuration the two spins are independent, so
//   G2(K, K', q) = < G_up(K, K') G_dn(q - K, q - K') >,
//   G_sigma(k1, k2) = G0(k1) delta - G0(k1) M_sigma(k1, k2) G0(k2),
//   M_sigma(k1, k2) = 1/(beta Nc) sum_ij E_sigma(i, k1) c_ij conj(E_sigma(j, k2)),
// E(j, k) = e^{i (w tau_j - K.r_j)}, c = (e^V - 1) N.  Measured points s = (K, n),
// n = -n_w4 .. n_w4 - 1, s = K * 2 n_w4 + n + n_w4; the spin-down factor at
// q - s = (Q - K, i w_{m - n - 1}).  Per measurement and walker:
//   k_g4_phase  E_sigma(j, s) for every vertex j and point s (0 for dead j);
//   k_g4_t      T_sigma(i, s) = f_i sum_j N_ij conj(E_sigma(j, s)), f_i = e^{V_i} - 1:
//               a dense product N (n x n) times E* (n x S), 4 n^2 S flop per spin;
//   k_g4_m      M_sigma(s1, s2) = 1/(beta Nc) sum_i E_sigma(i, s1) T_sigma(i, s2) for
//               both spins of one 32 x 32 tile of (s1, s2) (8 S^2 n flop per spin), then
//               A(s1, s2) += sign M_up M_dn and, on the diagonal, D_sigma(s) += sign M_sigma(s, s)
//               (each entry owned by one thread: no atomics).
// Phases: (2n + 1) tau / beta - 2 K.r / 2 pi modulo 2 in 56-bit fixed point
// from the per-vertex time words (k_freq_prep) and the problem's table of
// K.r / 2 pi, then one sincospi.  Arithmetic: FP64 on the FP64 path; FP32
// products with FP64 accumulators on the mixed path.
#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace dca {

template <typename A>
struct Cplx;
template <>
struct Cplx<float> {
  using type = float2;
};
template <>
struct Cplx<double> {
  using type = double2;
};

__device__ __forceinline__ bool wants_g4(const Config& cfg, const WalkerDev& w) {
  return cfg.n_w4 > 0 && w.active && w.measure_pending;
}

// Momentum index and fermionic frequency index of point s for spin sp.
__device__ __forceinline__ void g4_point(const Config& cfg, const ProblemDev& pb, int sp, int s, int& K, int& n) {
  const int nf = 2 * cfg.n_w4;
  const int k = s / nf;
  const int nu = s - k * nf - cfg.n_w4;
  if (sp == 0) {
    K = k;
    n = nu;
  } else {
    K = pb.k_dn[k];
    n = cfg.m4 - nu - 1;
  }
}

// e^{i pi p} for the phase p = q X 2^-56 - 2 KR 2^-56 (mod 2), q = 2n + 1 of either sign.
template <typename A>
__device__ __forceinline__ void g4_phase(unsigned long long X, int n, unsigned long long KR, A& c, A& s) {
  const long long q = 2LL * n + 1;
  const unsigned long long t = ((unsigned long long)q * X - (KR << 1)) & ((1ull << 57) - 1ull);
  if (sizeof(A) == 4) {
    const float p = (float)(unsigned)(t >> 33) * 0x1.0p-23f;
    sincospif(p, (float*)&s, (float*)&c);
  } else {
    const double p = (double)(t >> 4) * 0x1.0p-52;
    sincospi(p, (double*)&s, (double*)&c);
  }
}

template <typename A>
__device__ __forceinline__ size_t g4_plane(const WalkerDev& w, int sp, int S) {
  return (size_t)sp * w.cap * S;
}

// E_sigma(j, s): item = (walker-spin, 32 vertices); threads over (j, s).
template <typename A>
__global__ void __launch_bounds__(256) k_g4_phase(Config cfg) {
  using C2 = typename Cplx<A>::type;
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return wants_g4(cfg, w) ? blocks_of(w.n, 32) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1;
        const ProblemDev& pb = cfg.P[w.problem];
        const int nc = pb.nc, S = nc * 2 * cfg.n_w4;
        const int j0 = item * 32, j1 = min(w.n, j0 + 32);
        C2* E = reinterpret_cast<C2*>(w.g4E) + g4_plane<A>(w, sp, S);
        for (int e = threadIdx.x; e < (j1 - j0) * S; e += blockDim.x) {
          const int j = j0 + e / S, pt = e - (e / S) * S;
          const unsigned long long wj = w.vx[j];
          C2 v;
          v.x = (A)0;
          v.y = (A)0;
          if (wj != 0ull) {
            int K, n;
            g4_point(cfg, pb, sp, pt, K, n);
            const int site = (int)((wj & 0xffull) - 1ull);
            g4_phase<A>(wj >> 8, n, pb.kr56[K * nc + site], v.x, v.y);
          }
          E[(size_t)j * S + pt] = v;
        }
      });
}

// T_sigma(i, s) = f_i sum_j N_ij conj(E(j, s)).  Item = (walker-spin, 32 rows,
// 64 points); 256 threads = 4 row groups of 8 rows x 64 points; the columns j
// are streamed 32 at a time through shared memory.
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_g4_t(Config cfg) {
  using C2 = typename Cplx<A>::type;
  constexpr int RT = 32, PT = 64, JC = 32;
  __shared__ A Ms[RT][JC + 1];
  __shared__ C2 Es[JC][PT];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        if (!wants_g4(cfg, w)) return 0;
        const int S = cfg.P[w.problem].nc * 2 * cfg.n_w4;
        return blocks_of(w.n, RT) * blocks_of(S, PT);
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap, par = w.parity;
        const ProblemDev& pb = cfg.P[w.problem];
        const int S = pb.nc * 2 * cfg.n_w4, ptiles = (S + PT - 1) / PT;
        const int rt = item / ptiles, pt = item - rt * ptiles;
        const int i0 = rt * RT, p0 = pt * PT;
        const int tw = threadIdx.x & (PT - 1), tr = threadIdx.x >> 6;
        const T* N = (const T*)w.N[par][sp];
        const C2* E = reinterpret_cast<const C2*>(w.g4E) + g4_plane<A>(w, sp, S);
        A ar[8], ai[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) ar[k] = ai[k] = (A)0;
        for (int j0 = 0; j0 < n; j0 += JC) {
          __syncthreads();
          for (int e = threadIdx.x; e < RT * JC; e += blockDim.x) {
            const int r = e / JC, c = e - r * JC;
            Ms[r][c] = (i0 + r < n && j0 + c < n) ? (A)N[(size_t)(i0 + r) * ld + j0 + c] : (A)0;
          }
          for (int e = threadIdx.x; e < JC * PT; e += blockDim.x) {
            const int c = e / PT, f = e - c * PT;
            C2 v;
            v.x = (A)0;
            v.y = (A)0;
            if (j0 + c < n && p0 + f < S) v = E[(size_t)(j0 + c) * S + p0 + f];
            Es[c][f] = v;
          }
          __syncthreads();
          const int cend = min(JC, n - j0);
          for (int c = 0; c < cend; ++c) {
            const C2 e = Es[c][tw];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const A m = Ms[tr * 8 + k][c];
              ar[k] += m * e.x;  // N_ij conj(E)
              ai[k] -= m * e.y;
            }
          }
        }
        C2* Tp = reinterpret_cast<C2*>(w.g4T) + g4_plane<A>(w, sp, S);
        if (p0 + tw < S) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int i = i0 + tr * 8 + k;
            if (i < n) {
              const int si = w.vs[par][i];
              const A fi = si != 0 ? (A)(expV(pb, sp, si) - 1.0) : (A)0;
              C2 v;
              v.x = fi * ar[k];
              v.y = fi * ai[k];
              Tp[(size_t)i * S + p0 + tw] = v;
            }
          }
        }
      });
}

// M_sigma(s1, s2) for both spins of one 32 x 32 tile, then the accumulators.
// Item = (walker, tile); 256 threads: s2 = tx (32), s1 = ty + 8 a (a < 4).
template <typename A>
__global__ void __launch_bounds__(256) k_g4_m(Config cfg) {
  using C2 = typename Cplx<A>::type;
  constexpr int TL = 32, IC = 32;
  __shared__ C2 Ei[IC][TL + 1];
  __shared__ C2 Ti[IC][TL + 1];
  for_each_item(
      cfg.n_walkers,
      [&](int wi) -> long long {
        const WalkerDev& w = cfg.W[wi];
        if (!wants_g4(cfg, w)) return 0;
        const long long t = blocks_of(cfg.P[w.problem].nc * 2 * cfg.n_w4, TL);
        return t * t;
      },
      [&](int wi, int item) {
        const WalkerDev& w = cfg.W[wi];
        const ProblemDev& pb = cfg.P[w.problem];
        const int n = w.n, S = pb.nc * 2 * cfg.n_w4, tiles = (S + TL - 1) / TL;
        const int b1 = (item / tiles) * TL, b2 = (item - (item / tiles) * tiles) * TL;
        const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
        A mr[2][4], mi[2][4];
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
          const C2* E = reinterpret_cast<const C2*>(w.g4E) + g4_plane<A>(w, sp, S);
          const C2* Tp = reinterpret_cast<const C2*>(w.g4T) + g4_plane<A>(w, sp, S);
          A accr[4] = {(A)0, (A)0, (A)0, (A)0}, acci[4] = {(A)0, (A)0, (A)0, (A)0};
          for (int i0 = 0; i0 < n; i0 += IC) {
            __syncthreads();
            for (int e = threadIdx.x; e < IC * TL; e += blockDim.x) {
              const int r = e / TL, c = e - r * TL;
              C2 ve, vt;
              ve.x = ve.y = vt.x = vt.y = (A)0;
              if (i0 + r < n) {
                if (b1 + c < S) ve = E[(size_t)(i0 + r) * S + b1 + c];
                if (b2 + c < S) vt = Tp[(size_t)(i0 + r) * S + b2 + c];
              }
              Ei[r][c] = ve;
              Ti[r][c] = vt;
            }
            __syncthreads();
            const int iend = min(IC, n - i0);
            for (int r = 0; r < iend; ++r) {
              const C2 t = Ti[r][tx];
#pragma unroll
              for (int a = 0; a < 4; ++a) {
                const C2 e = Ei[r][ty + 8 * a];
                accr[a] += e.x * t.x - e.y * t.y;
                acci[a] += e.x * t.y + e.y * t.x;
              }
            }
          }
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            mr[sp][a] = accr[a];
            mi[sp][a] = acci[a];
          }
        }
        const double norm = 1.0 / (pb.beta * (double)pb.nc);
        const int s2 = b2 + tx;
        if (s2 < S) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int s1 = b1 + ty + 8 * a;
            if (s1 >= S) continue;
            const double ur = norm * (double)mr[0][a], ui = norm * (double)mi[0][a];
            const double dr = norm * (double)mr[1][a], di = norm * (double)mi[1][a];
            double* Ae = w.g4A + ((size_t)s1 * S + s2) * 2;
            Ae[0] += w.sign * (ur * dr - ui * di);
            Ae[1] += w.sign * (ur * di + ui * dr);
            if (s1 == s2) {
              w.g4D[2 * s1] += w.sign * ur;
              w.g4D[2 * s1 + 1] += w.sign * ui;
              w.g4D[2 * ((size_t)S + s1)] += w.sign * dr;
              w.g4D[2 * ((size_t)S + s1) + 1] += w.sign * di;
            }
          }
        }
      });
}

int launch_meas_g4(const Config& cfg, int max_cap, int max_nc, cudaStream_t st) {
  if (cfg.n_w4 <= 0) return 0;
  const long long S = (long long)max_nc * 2 * cfg.n_w4;
  const long long ip = 2LL * cfg.n_walkers * blocks_of(max_cap, 32);
  const long long it = 2LL * cfg.n_walkers * blocks_of(max_cap, 32) * blocks_of(S, 64);
  const long long im = (long long)cfg.n_walkers * blocks_of(S, 32) * blocks_of(S, 32);
  if (cfg.prec == PREC_MIXED) {
    k_g4_phase<float><<<persist_grid((const void*)k_g4_phase<float>, ip, 256), 256, 0, st>>>(cfg);
    k_g4_t<float, float><<<persist_grid((const void*)k_g4_t<float, float>, it, 256), 256, 0, st>>>(cfg);
    k_g4_m<float><<<persist_grid((const void*)k_g4_m<float>, im, 256), 256, 0, st>>>(cfg);
  } else {
    k_g4_phase<double><<<persist_grid((const void*)k_g4_phase<double>, ip, 256), 256, 0, st>>>(cfg);
    k_g4_t<double, double><<<persist_grid((const void*)k_g4_t<double, double>, it, 256), 256, 0, st>>>(cfg);
    k_g4_m<double><<<persist_grid((const void*)k_g4_m<double>, im, 256), 256, 0, st>>>(cfg);
  }
  return 3;
}

// Read-out: G2 from one set of accumulators (see dca_g4_assemble).
__global__ void k_g4_assemble(int S, const double* A, const double* D, double sign_sum, const double* Gu,
                              const double* Gd, double* out) {
  const long long total = (long long)S * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int s1 = (int)(e / S), s2 = (int)(e - (long long)s1 * S);
    // P(s) = G0u(s) G0d(s)
    const double p1r = Gu[2 * s1] * Gd[2 * s1] - Gu[2 * s1 + 1] * Gd[2 * s1 + 1];
    const double p1i = Gu[2 * s1] * Gd[2 * s1 + 1] + Gu[2 * s1 + 1] * Gd[2 * s1];
    const double p2r = Gu[2 * s2] * Gd[2 * s2] - Gu[2 * s2 + 1] * Gd[2 * s2 + 1];
    const double p2i = Gu[2 * s2] * Gd[2 * s2 + 1] + Gu[2 * s2 + 1] * Gd[2 * s2];
    const double ar = A[2 * e], ai = A[2 * e + 1];
    // A P(s2), then times P(s1)
    double xr = ar * p2r - ai * p2i, xi = ar * p2i + ai * p2r;
    if (s1 == s2) {
      // sign_sum - D_up G0u - D_dn G0d
      const double ur = D[2 * s1], ui = D[2 * s1 + 1], dr = D[2 * ((long long)S + s1)], di = D[2 * ((long long)S + s1) + 1];
      xr += sign_sum - (ur * Gu[2 * s1] - ui * Gu[2 * s1 + 1]) - (dr * Gd[2 * s1] - di * Gd[2 * s1 + 1]);
      xi += -(ur * Gu[2 * s1 + 1] + ui * Gu[2 * s1]) - (dr * Gd[2 * s1 + 1] + di * Gd[2 * s1]);
    }
    out[2 * e] = (p1r * xr - p1i * xi) / sign_sum;
    out[2 * e + 1] = (p1r * xi + p1i * xr) / sign_sum;
  }
}

void launch_g4_assemble(int S, const double* A, const double* D, double sign_sum, const double* Gu, const double* Gd,
                        double* out, cudaStream_t st) {
  const long long total = (long long)S * S;
  const int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
  k_g4_assemble<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(S, A, D, sign_sum, Gu, Gd, out);
}

}  // namespace dca
