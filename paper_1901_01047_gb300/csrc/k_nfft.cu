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
//
// Times enter as per-vertex fixed-point words (k_freq_prep, once per
// measurement): X = floor(tau / beta 2^56).  A difference X_i - X_j modulo
// 2^56 is frac((tau_i - tau_j) / beta) exactly, its grid position and offset
// come from one 64-bit integer product, and the phase (2n + 1) tau / beta
// modulo 2 from another, so the sample loops of both variants run without
// FP64 arithmetic (FP64 is 1/64 of the FP32 rate on this GPU).
#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace dca {

constexpr int NFFT_RB = 64;        // rows of N per item
constexpr int NFFT_MSP_MAX = 12;
constexpr unsigned long long X56_MASK = (1ull << 56) - 1ull;

// A measured walker needs the time words for the frequency measurement of M
// and for the two-particle measurement.
__device__ __forceinline__ bool wants_freq(const Config& cfg, const WalkerDev& w) {
  return (cfg.n_omega > 0 || cfg.n_w4 > 0) && w.active && w.measure_pending;
}

__device__ __forceinline__ bool wants_nfft(const Config& cfg, const WalkerDev& w) {
  return cfg.n_omega > 0 && !cfg.freq_dft && wants_freq(cfg, w);
}

__device__ __forceinline__ bool wants_dft(const Config& cfg, const WalkerDev& w) {
  return cfg.n_omega > 0 && cfg.freq_dft && wants_freq(cfg, w);
}

// Time word of a vertex: (floor(tau / beta 2^56) << 8) | (site + 1), 0 for a
// dead vertex (tau / beta within rounding of 1 kept below 1).
__device__ __forceinline__ unsigned long long time_word(double tau, double inv_beta, int site, int s) {
  if (s == 0) return 0ull;
  const double v = tau * inv_beta * 0x1.0p56;
  const unsigned long long X = v >= 0x1.0p56 ? X56_MASK : (v <= 0.0 ? 0ull : (unsigned long long)v);
  return (X << 8) | (unsigned long long)(site + 1);
}

// e^{i pi q x} for odd q = 2n + 1 and x = X 2^-56 in [0, 1): q X modulo 2^57
// (the low bits of the wrapped 64-bit product) is q x modulo 2 in units of
// 2^-56, exact; then one sincospi of the reduced phase (24 bits of it in FP32).
template <typename A>
__device__ __forceinline__ void phase_cs(unsigned long long X, uint32_t q, A& c, A& s) {
  const unsigned long long t = ((unsigned long long)q * X) & ((1ull << 57) - 1ull);
  if (sizeof(A) == 4) {
    const float p = (float)(unsigned)(t >> 33) * 0x1.0p-23f;  // in [0, 2)
    sincospif(p, (float*)&s, (float*)&c);
  } else {
    const double p = (double)(t >> 4) * 0x1.0p-52;
    sincospi(p, (double*)&s, (double*)&c);
  }
}

// Fraction of a 64-bit fixed-point value (2^-64 units) in the arithmetic type.
template <typename A>
__device__ __forceinline__ A frac64(unsigned long long lo) {
  if (sizeof(A) == 4) return (A)((float)(unsigned)(lo >> 40) * 0x1.0p-24f);
  return (A)((double)(lo >> 11) * 0x1.0p-53);
}

constexpr int DFT_RT = 32, DFT_WT = 64, DFT_JC = 32;

// Once per measurement and walker (one block each): the time words of the
// vertices, and for the dense variant the live columns sorted by site (perm)
// with the group offsets goff[nc + 1].
__global__ void __launch_bounds__(256) k_freq_prep(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  if (!wants_freq(cfg, w)) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int nc = pb.nc, n = w.n, par = w.parity;
  const double inv_beta = 1.0 / pb.beta;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    w.vx[j] = time_word(w.vtau[par][j], inv_beta, w.vsite[par][j], w.vs[par][j]);
  if (!cfg.freq_dft || cfg.n_omega <= 0) return;
  __shared__ int s_cnt[65], s_pos[65];
  for (int r = threadIdx.x; r <= nc; r += blockDim.x) s_cnt[r] = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (w.vs[par][j] != 0) atomicAdd(&s_cnt[w.vsite[par][j]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int r = 0; r < nc; ++r) {
      w.goff[r] = run;
      s_pos[r] = run;
      run += s_cnt[r];
    }
    w.goff[nc] = run;
  }
  __syncthreads();
  // stable within a site: one thread per site walks the columns in order
  for (int r = threadIdx.x; r < nc; r += blockDim.x) {
    int pos = s_pos[r];
    for (int j = 0; j < n; ++j)
      if (w.vs[par][j] != 0 && w.vsite[par][j] == r) w.perm[pos++] = j;
  }
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

// Item = (walker-spin, block of NFFT_RB rows of N); each warp takes every
// eighth row of the block and its lanes stride over the columns.  SMEM: the
// block stages the whole grid of its walker-spin (nc x L accumulators) in
// shared memory and adds it to the walker's FP64 grid at the end of the item;
// otherwise it adds every weight to the global grid directly.
template <typename T, typename A, bool SMEM>
__global__ void __launch_bounds__(256) k_meas_nfft(Config cfg) {
  extern __shared__ __align__(16) unsigned char nfft_raw[];
  __shared__ A s_e3[NFFT_MSP_MAX + 1];
  const int L = cfg.nfft_L, msp = cfg.nfft_msp;
  const A a = (A)(0.75 * 3.14159265358979323846 / (double)msp);  // pi (R - 1/2) / (R M_sp), R = 2
  if (threadIdx.x <= msp) s_e3[threadIdx.x] = (A)exp(-(double)a * threadIdx.x * threadIdx.x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
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
        const unsigned long long* vx = w.vx;
        double* gglob = w.Mgrid + (size_t)sp * nc * L;
        // accumulation: the staged grid in A (one item's sums), the walker's grid in FP64
        using S = typename std::conditional<SMEM, A, double>::type;
        S* g = SMEM ? reinterpret_cast<S*>(nfft_raw) : reinterpret_cast<S*>(gglob);
        __syncthreads();  // the previous item of this block is done with the staged grid
        if (SMEM)
          for (int e = threadIdx.x; e < nc * L; e += blockDim.x) g[e] = (S)0;
        __syncthreads();
        const double scale = w.sign / (pb.beta * (double)nc);
        const int i0 = item * NFFT_RB;
        const int i1 = min(n, i0 + NFFT_RB);
        for (int i = i0 + warp; i < i1; i += nwarps) {
          const unsigned long long wi = vx[i];
          if (wi == 0ull) continue;  // dead row: its factor e^{V} - 1 is zero
          const int si = w.vs[par][i];
          const A fi = (A)((expV(pb, sp, si) - 1.0) * scale);
          const unsigned long long Xi = wi >> 8;
          const int* sub_row = pb.site_sub + (int)((wi & 0xffull) - 1ull) * nc;
          const T* Nrow = N + (size_t)i * ld;
          for (int j = lane; j < n; j += 32) {
            const unsigned long long wj = __ldg(vx + j);
            if (wj == 0ull) continue;  // dead column of N: the unit vector, zero after the factor
            const unsigned long long Xj = wj >> 8;
            // t = tau_i - tau_j, moved into [0, beta) with the antiperiodic sign
            A m = fi * (A)Nrow[j];
            if (Xi < Xj) m = -m;
            const unsigned long long sh = ((Xi - Xj) & X56_MASK) << 8;  // frac(t / beta) in 2^-64 units
            const int l0 = (int)__umul64hi(sh, (unsigned long long)L);
            const A d = frac64<A>(sh * (unsigned long long)L);
            const int dd = __ldg(sub_row + (int)((wj & 0xffull) - 1ull));
            spread_sample<A, S>(g + (size_t)dd * L, L, msp, a, s_e3, l0, d, m);
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

cudaError_t setup_ndft();

cudaError_t setup_nfft() {
  cudaError_t e = setup_ndft();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_meas_nfft<double, double, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NFFT_SMEM_MAX);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_meas_nfft<float, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)NFFT_SMEM_MAX);
  return e;
}

int launch_meas_nfft(const Config& cfg, int max_cap, int max_nc, cudaStream_t st) {
  if (cfg.n_omega <= 0 && cfg.n_w4 <= 0) return 0;
  k_freq_prep<<<cfg.n_walkers, 256, 0, st>>>(cfg);
  if (cfg.n_omega <= 0) return 1;
  if (cfg.freq_dft) return 1 + launch_meas_ndft(cfg, max_cap, max_nc, st);
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
  return 2;
}

void launch_nfft_finish(const Config& cfg, int max_nc, const long long* d_base, double* d_out, cudaStream_t st) {
  const long long per = 2LL * max_nc * cfg.n_omega;
  const int bx = (int)((per + 255) / 256 < 64 ? (per + 255) / 256 : 64);
  k_nfft_finish<<<dim3(bx, cfg.n_walkers), 256, 0, st>>>(cfg, d_base, d_out);
}

// ---------------------------------------------------------------------------
// The same frequency measurement as a dense contraction (no window, no grid):
//   M(dr, i w_n) = sum_i e^{i w_n tau_i} f_i sum_{j : r_j = rb(i, dr)} N_ij e^{-i w_n tau_j},
// f_i = sign (e^{V_i} - 1) / (beta Nc).  With the columns j sorted by site
// (k_freq_prep, once per measured walker), the inner sums over one site group
// are runs of consecutive sorted columns: per (row i, frequency) a thread
// accumulates one run at a time and adds the finished run, times
// f_i e^{i w tau_i}, to the block's accumulator of difference dr =
// r_i - r_j.  The work is n^2 n_omega multiply-adds per spin, on the FMA pipes.
// Item = (walker-spin, 32 rows, 64 frequencies); block 256 = 4 row groups of 8
// rows x 64 frequencies.  Phases: (2n + 1) tau / beta reduced modulo 2 in
// integer fixed point (the time words), then sincospi.
// ---------------------------------------------------------------------------
// One item: 32 rows i of one walker-spin x 64 frequencies; 256 threads = 4
// groups of 8 rows x 64 frequencies.  The site-sorted columns are streamed in
// chunks of 32 (N gathered through perm, the column phases e^{-i w tau_j}
// computed once per chunk); within a chunk the columns are cut into segments
// at the ends of site groups, and at a group end each thread folds its
// partial sums f_i e^{i w tau_i} sum_j N_ij e^{-i w tau_j} into the item's
// accumulator of dr = r_i - r_j (dynamic shared memory, [max_nc][64][2] in
// the accumulation type), which is added to the walker's sums at the end.
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_meas_ndft(Config cfg) {
  __shared__ A Ms[DFT_RT][DFT_JC + 1];
  __shared__ A Uc[DFT_JC][DFT_WT], Us[DFT_JC][DFT_WT];
  __shared__ int s_goff[65];
  __shared__ int s_seg_end[DFT_JC + 66], s_seg_site[DFT_JC + 66], s_nseg;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  A* Macc = reinterpret_cast<A*>(dyn_smem);  // [dr][frequency][re, im]
  const int nw = cfg.n_omega, wtiles = (nw + DFT_WT - 1) / DFT_WT;
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return wants_dft(cfg, w) ? blocks_of(w.n, DFT_RT) * wtiles : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap, par = w.parity;
        const ProblemDev& pb = cfg.P[w.problem];
        const int nc = pb.nc;
        const int rt = item / wtiles, wt = item - rt * wtiles;
        const int i0 = rt * DFT_RT, w0 = wt * DFT_WT;
        const int tw = threadIdx.x & (DFT_WT - 1), tr = threadIdx.x >> 6;  // frequency, row group
        const int wn = w0 + tw;
        const uint32_t q = 2u * (uint32_t)wn + 1u;
        const T* N = (const T*)w.N[par][sp];
        const int* perm = w.perm;
        const double inv_beta = 1.0 / pb.beta;
        __syncthreads();  // the previous item is done with the shared tiles
        for (int e = threadIdx.x; e < nc * DFT_WT * 2; e += blockDim.x) Macc[e] = (A)0;
        for (int r = threadIdx.x; r <= nc; r += blockDim.x) s_goff[r] = w.goff[r];
        // this thread's rows: f_i e^{i w tau_i} and the site of row i
        A fr[8], fc[8], fs[8];
        int rsite[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = i0 + tr * 8 + k;
          fr[k] = (A)0;
          fc[k] = fs[k] = (A)0;
          rsite[k] = 0;
          if (i < n && w.vs[par][i] != 0 && wn < nw) {
            fr[k] = (A)((expV(pb, sp, w.vs[par][i]) - 1.0) * w.sign * inv_beta / (double)nc);
            phase_cs<A>(w.vx[i] >> 8, q, fc[k], fs[k]);
            rsite[k] = w.vsite[par][i];
          }
        }
        __syncthreads();
        const int ncols = s_goff[nc];
        A ar[8], ai[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) ar[k] = ai[k] = (A)0;
        for (int j0 = 0; j0 < ncols; j0 += DFT_JC) {
          const int cend = min(DFT_JC, ncols - j0);
          __syncthreads();
          for (int e = threadIdx.x; e < DFT_RT * DFT_JC; e += blockDim.x) {
            const int r = e / DFT_JC, c = e - r * DFT_JC;
            const int i = i0 + r;
            Ms[r][c] = (i < n && c < cend) ? (A)N[(size_t)i * ld + perm[j0 + c]] : (A)0;
          }
          for (int e = threadIdx.x; e < DFT_JC * DFT_WT; e += blockDim.x) {
            const int c = e / DFT_WT, f = e - c * DFT_WT;
            A cs = (A)0, sn = (A)0;
            if (c < cend && w0 + f < nw)
              phase_cs<A>(w.vx[perm[j0 + c]] >> 8, 2u * (uint32_t)(w0 + f) + 1u, cs, sn);
            Uc[c][f] = cs;
            Us[c][f] = sn;
          }
          if (threadIdx.x == 0) {
            // segments of this chunk: cut at every group end inside it
            int ns = 0;
            for (int g = 0; g < nc; ++g) {
              const int e = s_goff[g + 1] - j0;
              if (e > 0 && e <= cend && s_goff[g + 1] > s_goff[g]) {
                s_seg_end[ns] = e;
                s_seg_site[ns] = g;
                ++ns;
              }
            }
            if (ns == 0 || s_seg_end[ns - 1] < cend) {
              s_seg_end[ns] = cend;
              s_seg_site[ns] = -1;  // the group goes on into the next chunk
              ++ns;
            }
            s_nseg = ns;
          }
          __syncthreads();
          int c = 0;
          for (int sg = 0; sg < s_nseg; ++sg) {
            const int ce = s_seg_end[sg];
            for (; c < ce; ++c) {
              const A uc = Uc[c][tw], us = Us[c][tw];
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                const A m = Ms[tr * 8 + k][c];
                ar[k] += m * uc;  // N_ij e^{-i w tau_j}
                ai[k] -= m * us;
              }
            }
            const int rb = s_seg_site[sg];
            if (rb >= 0) {
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                if (fr[k] != (A)0) {
                  // f_i e^{i w tau_i} (ar + i ai)
                  const A re = fr[k] * (fc[k] * ar[k] - fs[k] * ai[k]);
                  const A im = fr[k] * (fc[k] * ai[k] + fs[k] * ar[k]);
                  const int d = __ldg(pb.site_sub + rsite[k] * nc + rb);
                  atomicAdd(&Macc[(d * DFT_WT + tw) * 2], re);
                  atomicAdd(&Macc[(d * DFT_WT + tw) * 2 + 1], im);
                }
                ar[k] = ai[k] = (A)0;
              }
            }
          }
        }
        __syncthreads();
        double* out = w.Mfreq + (size_t)sp * nc * nw * 2;
        for (int e = threadIdx.x; e < nc * DFT_WT; e += blockDim.x) {
          const int d = e / DFT_WT, f = e - d * DFT_WT;
          if (w0 + f < nw) {
            const A re = Macc[e * 2], im = Macc[e * 2 + 1];
            if (re != (A)0) atomicAdd(out + ((size_t)d * nw + w0 + f) * 2, (double)re);
            if (im != (A)0) atomicAdd(out + ((size_t)d * nw + w0 + f) * 2 + 1, (double)im);
          }
        }
      });
}

template <typename T, typename A>
static void launch_ndft_kernel(const Config& cfg, long long items, int max_nc, cudaStream_t st) {
  const size_t smem = (size_t)max_nc * DFT_WT * 2 * sizeof(A);
  k_meas_ndft<T, A><<<persist_grid((const void*)k_meas_ndft<T, A>, items, 256, smem), 256, smem, st>>>(cfg);
}

cudaError_t setup_ndft() {
  cudaError_t e = cudaFuncSetAttribute(k_meas_ndft<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(64 * DFT_WT * 2 * sizeof(double)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_meas_ndft<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(64 * DFT_WT * 2 * sizeof(float)));
  return e;
}

int launch_meas_ndft(const Config& cfg, int max_cap, int max_nc, cudaStream_t st) {
  if (cfg.n_omega <= 0 || !cfg.freq_dft) return 0;
  const long long items = 2LL * cfg.n_walkers * blocks_of(max_cap, DFT_RT) * ((cfg.n_omega + DFT_WT - 1) / DFT_WT);
  if (cfg.prec == PREC_MIXED) launch_ndft_kernel<float, float>(cfg, items, max_nc, st);
  else launch_ndft_kernel<double, double>(cfg, items, max_nc, st);
  return 1;
}

// Read-out of the dense variant: the accumulators are the result.
__global__ void k_ndft_copy(Config cfg, const long long* base, double* out) {
  const int wi = blockIdx.y;
  const WalkerDev& w = cfg.W[wi];
  const long long total = 2LL * cfg.P[w.problem].nc * cfg.n_omega * 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    out[base[wi] + e] = w.Mfreq[e];
}

void launch_ndft_copy(const Config& cfg, int max_nc, const long long* d_base, double* d_out, cudaStream_t st) {
  const long long per = 4LL * max_nc * cfg.n_omega;
  const int bx = (int)((per + 255) / 256 < 64 ? (per + 255) / 256 : 64);
  k_ndft_copy<<<dim3(bx, cfg.n_walkers), 256, 0, st>>>(cfg, d_base, d_out);
}

}  // namespace dca
