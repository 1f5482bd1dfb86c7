// k_nfft.cu -- frequency-domain measurement of M by the delayed NFFT
// (DCA++ paper Sec. 2.3, "Non-equidistant FFT measurements", Eq.
// convolution_theorem and Eq. nfft).
//
// Every measured configuration contributes, per spin and cluster difference
// dr = r_i - r_j, the samples c_ij = sign (e^{V_i} - 1) N_ij / (beta Nc) at
// the times t_ij = tau_i - tau_j, and the measurement wanted is
//     M(dr, i w_n) = sum_{i,j : r_i - r_j = dr} c_ij e^{i w_n t_ij},
//     w_n = (2n + 1) pi / beta,   n = 0 .. n_omega - 1,
// from which G(K, i w_n) = g0 + g0^2 M(K, i w_n), M(K) = sum_dr e^{-iK.dr} M(dr)
// (g0 = -G0; the paper's G = G0 - G0 M G0 / beta with its M = beta times this).
//
// Spreading (k_meas_nfft, once per measurement): each sample is convolved
// with a truncated Gaussian onto an equispaced grid of L = 4 n_omega points
// over [0, beta) (oversampling 2 of the band -n_omega .. n_omega - 1), the
// grid antiperiodic like the fermionic functions (a time t < 0 is t + beta
// with the sign flipped; window points past either end wrap with a sign
// flip).  The grid is accumulated over all measurements (the "delayed" NFFT:
// the transform is linear, so one transform at the end serves every
// measurement).
//
// Transform (k_nfft_finish, at read-out): C(n) = sum_l g_l e^{i w_n l h},
// h = beta / L, divided by the window's Fourier transform.
//
// Window (Greengard and Lee, "Accelerating the nonuniform fast Fourier
// transform", SIAM Rev. 46 (2004)): phi(u) = exp(-a u^2) in grid units with
// a = pi (R - 1/2) / (R M_sp), oversampling R = 2, 2 M_sp grid points per
// sample; truncation and aliasing errors ~ exp(-pi M_sp (R - 1/2) / R):
// M_sp = 12 (FP64 path, ~1e-12) or 8 (mixed path, ~1e-8).  The weights come
// from exp(-a (d - k)^2) = exp(-a d^2) exp(2 a d)^k exp(-a k^2) (two
// exponentials per sample, the last factor tabulated).
#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace dca {

constexpr int NFFT_RB = 128;       // rows of N per item
constexpr int NFFT_MSP_MAX = 12;

__device__ __forceinline__ bool wants_nfft(const Config& cfg, const WalkerDev& w) {
  return cfg.n_omega > 0 && w.active && w.measure_pending;
}

// Spread one sample (value m at grid position l0 + d, d in [0, 1), the
// position split in FP64 so that an FP32 fraction keeps it to 2^-24 of a grid
// step) into the grid row `g` (length L) with atomic adds in the accumulation
// type S.
template <typename A, typename S>
__device__ __forceinline__ void spread_sample(S* g, int L, int msp, A a, const A* e3, int l0, A d, A m) {
  const A e1 = m * (A)exp(-a * d * d);
  const A e2 = (A)exp((A)2 * a * d);
  const A e2i = (A)1 / e2;
  // k = 0 .. msp: weight e1 * e2^k * e3[k];  k = -1 .. -(msp - 1): e1 * e2^k * e3[-k]
  A p = e1;
  for (int k = 0; k <= msp; ++k) {
    int l = l0 - k;  // grid point of offset u = d + k (the sample sits at l0 + d)
    A v = p * e3[k];
    if (l < 0) {
      l += L;
      v = -v;
    }
    atomicAdd(g + l, (S)v);
    p *= e2i;
  }
  p = e1 * e2;
  for (int k = 1; k < msp; ++k) {
    int l = l0 + k;  // offset u = d - k
    A v = p * e3[k];
    if (l >= L) {
      l -= L;
      v = -v;
    }
    atomicAdd(g + l, (S)v);
    p *= e2;
  }
}

// Item = (walker-spin, block of NFFT_RB rows of N).  SMEM: the block stages
// the whole grid of its walker-spin (nc x L accumulators) in shared memory and
// adds it to the walker's FP64 grid at the end of the item; otherwise it adds
// every weight to the global grid directly.
template <typename T, typename A, bool SMEM>
__global__ void __launch_bounds__(256) k_meas_nfft(Config cfg) {
  extern __shared__ __align__(16) unsigned char nfft_raw[];
  __shared__ A s_e3[NFFT_MSP_MAX + 1];
  const int L = cfg.nfft_L, msp = cfg.nfft_msp;
  const A a = (A)(0.75 * 3.14159265358979323846 / (double)msp);  // pi (R - 1/2) / (R M_sp), R = 2
  if (threadIdx.x <= msp) s_e3[threadIdx.x] = (A)exp(-(double)a * threadIdx.x * threadIdx.x);
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return wants_nfft(cfg, w) ? blocks_of(w.n, NFFT_RB) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap, par = w.parity;
        const ProblemDev& pb = cfg.P[w.problem];
        const int nc = pb.nc;
        const T* N = (const T*)w.N[par][sp];
        const int* vs = w.vs[par];
        const int* vsite = w.vsite[par];
        const double* vtau = w.vtau[par];
        double* gglob = w.Mgrid + (size_t)sp * nc * L;
        // accumulation: the staged grid in A (one item's sums), the walker's grid in FP64
        using S = typename std::conditional<SMEM, A, double>::type;
        S* g = SMEM ? reinterpret_cast<S*>(nfft_raw) : reinterpret_cast<S*>(gglob);
        __syncthreads();  // the previous item of this block is done with the staged grid
        if (SMEM)
          for (int e = threadIdx.x; e < nc * L; e += blockDim.x) g[e] = (S)0;
        __syncthreads();
        const double scale = w.sign / (pb.beta * (double)nc);
        const double inv_h = (double)L / pb.beta;
        const int i0 = item * NFFT_RB;
        const int i1 = min(n, i0 + NFFT_RB);
        for (int i = i0; i < i1; ++i) {
          const int si = vs[i];
          if (si == 0) continue;  // dead row: its factor e^{V} - 1 is zero
          const double fi = (expV(pb, sp, si) - 1.0) * scale;
          const double ti = vtau[i];
          const int* sub_row = pb.site_sub + vsite[i] * nc;
          for (int j = threadIdx.x; j < n; j += blockDim.x) {
            if (vs[j] == 0) continue;  // dead column of N: the unit vector, zero after the factor
            double t = ti - vtau[j];
            double m = fi * (double)N[(size_t)i * ld + j];
            if (t < 0.0) {
              t += pb.beta;
              m = -m;
            }
            double x = t * inv_h;
            if (x >= (double)L) x = (double)L - 0.5;  // t within rounding of beta
            const int l0 = (int)x;
            const int d = __ldg(sub_row + vsite[j]);
            spread_sample<A, S>(g + (size_t)d * L, L, msp, a, s_e3, l0, (A)(x - (double)l0), (A)m);
          }
        }
        if (SMEM) {
          __syncthreads();
          for (int e = threadIdx.x; e < nc * L; e += blockDim.x) {
            const double v = (double)g[e];
            if (v != 0.0) atomicAdd(gglob + e, v);
          }
        }
      });
}

// Read-out: M(dr, i w_n) = [sum_l g_l e^{i w_n l h}] / phi_hat(w_n h) for every
// walker, spin, difference and frequency; out [w][2][nc][n_omega][re, im]
// at offset base[w].  One thread per output value; the phases are exact
// multiples of pi / L ((2n + 1) l mod 2L).
__global__ void __launch_bounds__(256) k_nfft_finish(Config cfg, const long long* base, double* out) {
  const int L = cfg.nfft_L, msp = cfg.nfft_msp, nw = cfg.n_omega;
  const double a = 0.75 * 3.14159265358979323846 / (double)msp;
  const double root = sqrt(3.14159265358979323846 / a);
  const int wi = blockIdx.y;
  const WalkerDev& w = cfg.W[wi];
  const int nc = cfg.P[w.problem].nc;
  const int total = 2 * nc * nw;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int k = e % nw, row = e / nw;  // row = sp * nc + dr
    const double* g = w.Mgrid + (size_t)row * L;
    const long long q = 2LL * k + 1;
    double re = 0.0, im = 0.0;
    for (int l = 0; l < L; ++l) {
      const double gl = g[l];
      if (gl == 0.0) continue;
      double sn, cs;
      sincospi((double)((q * l) % (2LL * L)) / (double)L, &sn, &cs);
      re += gl * cs;
      im += gl * sn;
    }
    const double nu = 3.14159265358979323846 * (double)q / (double)L;
    const double ph = root * exp(-nu * nu / (4.0 * a));
    double* o = out + base[wi] + 2 * (size_t)e;
    o[0] = re / ph;
    o[1] = im / ph;
  }
}

// Largest grid staged in shared memory per block (bytes); larger grids are
// accumulated in global memory directly.
constexpr size_t NFFT_SMEM_MAX = 160 * 1024;

size_t nfft_smem_bytes(const Config& cfg, int max_nc) {
  const size_t acc = cfg.prec == PREC_MIXED ? sizeof(float) : sizeof(double);
  return (size_t)max_nc * (size_t)cfg.nfft_L * acc;
}

cudaError_t setup_nfft() {
  cudaError_t e = cudaFuncSetAttribute(k_meas_nfft<double, double, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NFFT_SMEM_MAX);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_meas_nfft<float, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)NFFT_SMEM_MAX);
  return e;
}

int launch_meas_nfft(const Config& cfg, int max_cap, int max_nc, cudaStream_t st) {
  if (cfg.n_omega <= 0) return 0;
  const long long items = 2LL * cfg.n_walkers * blocks_of(max_cap, NFFT_RB);
  const size_t smem = nfft_smem_bytes(cfg, max_nc);
  if (smem <= NFFT_SMEM_MAX) {
    if (cfg.prec == PREC_MIXED) {
      const void* fn = (const void*)k_meas_nfft<float, float, true>;
      k_meas_nfft<float, float, true><<<persist_grid(fn, items, 256, smem), 256, smem, st>>>(cfg);
    } else {
      const void* fn = (const void*)k_meas_nfft<double, double, true>;
      k_meas_nfft<double, double, true><<<persist_grid(fn, items, 256, smem), 256, smem, st>>>(cfg);
    }
  } else {
    if (cfg.prec == PREC_MIXED)
      k_meas_nfft<float, float, false><<<sm_grid(items, 4), 256, 0, st>>>(cfg);
    else
      k_meas_nfft<double, double, false><<<sm_grid(items, 4), 256, 0, st>>>(cfg);
  }
  return 1;
}

void launch_nfft_finish(const Config& cfg, int max_nc, const long long* d_base, double* d_out, cudaStream_t st) {
  const long long per = 2LL * max_nc * cfg.n_omega;
  const int bx = (int)((per + 255) / 256 < 64 ? (per + 255) / 256 : 64);
  k_nfft_finish<<<dim3(bx, cfg.n_walkers), 256, 0, st>>>(cfg, d_base, d_out);
}

}  // namespace dca
