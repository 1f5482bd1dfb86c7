// device_util.cuh -- small device helpers of the walker kernels.
#pragma once
#include <cstdint>

#include "state.h"

namespace dca {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// 4x32 S-box, round multipliers 0xD2511F53 and 0xCD9E8D57, key bumped by the
// Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.
struct Philox4 {
  uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Philox4 out;
  out.v[0] = c0;
  out.v[1] = c1;
  out.v[2] = c2;
  out.v[3] = c3;
  return out;
}

enum : uint32_t { TAG_PROPOSAL = 0u, TAG_ACCEPT = 1u, TAG_INIT = 2u };

__device__ __forceinline__ Philox4 draw(const WalkerDev& w, uint64_t j, uint32_t tag) {
  return philox4x32_10((uint32_t)j, (uint32_t)(j >> 32), tag, 0u, w.key0, w.key1);
}

// 53-bit uniform in [0, 1) from two words (high word first).
__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
  const uint64_t x = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)(x >> 11) * 0x1.0p-53;
}

// floor(word * m / 2^32), exact integer arithmetic.
__device__ __forceinline__ uint32_t scaled_index(uint32_t word, uint32_t m) { return __umulhi(word, m); }

// g0 at a time difference in (-beta, beta) from one table row: linear
// interpolation on the uniform grid, g0(t - beta) = -g0(t), dt == 0 read as 0+.
__device__ __forceinline__ double g0_interp(const double* __restrict__ row, int n_tau, double beta,
                                            double tau_scale, double dt) {
  double sgn = 1.0;
  if (dt < 0.0) {
    dt += beta;
    sgn = -1.0;
  }
  const double x = dt * tau_scale;
  int l = (int)x;
  l = l < 0 ? 0 : (l >= n_tau ? n_tau - 1 : l);
  const double f = x - (double)l;
  const double a = __ldg(row + l), b = __ldg(row + l + 1);
  return sgn * (a + f * (b - a));
}

// g0_sigma(r_a - r_b, tau_a - tau_b)
__device__ __forceinline__ double g0_pair(const ProblemDev& p, int sp, int ra, double ta, int rb, double tb) {
  const int d = __ldg(p.site_sub + ra * p.nc + rb);
  const double* row = p.g0 + ((size_t)sp * p.nc + d) * (size_t)(p.n_tau + 1);
  return g0_interp(row, p.n_tau, p.beta, p.tau_scale, ta - tb);
}

// Equal-time, same-vertex value g0(0+) on the diagonal.
__device__ __forceinline__ double g0_diag(const ProblemDev& p, int sp, int r) {
  const int d = __ldg(p.site_sub + r * p.nc + r);
  return __ldg(p.g0 + ((size_t)sp * p.nc + d) * (size_t)(p.n_tau + 1));
}

// Mixed-precision interpolation.  An imaginary time is carried on the g0 grid
// as x = tau n_tau / beta split into an integer part and an FP32 fraction
// (formed once per vertex in FP64).  The grid index of a difference x_a - x_b
// is then exact and only the interpolation weight (error ~2^-24 of a grid
// step) and the arithmetic are FP32: no FP64 operation per table lookup.
struct GridTime {
  int i;
  float f;
};

__device__ __forceinline__ GridTime grid_time(double tau, double tau_scale) {
  const double x = tau * tau_scale;
  const double fl = floor(x);
  return GridTime{(int)fl, (float)(x - fl)};
}

// g0(t_a - t_b) from one row of the FP32 copy of the table, with the
// conventions of g0_interp.
__device__ __forceinline__ float g0_interp_grid(const float* __restrict__ row, int n_tau, GridTime a, GridTime b) {
  int l = a.i - b.i;
  float f = a.f - b.f;
  if (f < 0.0f) {
    f += 1.0f;
    --l;
  }
  float sgn = 1.0f;
  if (l < 0) {
    l += n_tau;
    sgn = -1.0f;
  }
  if (l >= n_tau) {
    f += (float)(l - (n_tau - 1));
    l = n_tau - 1;
  }
  const float lo = __ldg(row + l), hi = __ldg(row + l + 1);
  return sgn * (lo + f * (hi - lo));
}

// Row of the FP32 g0 table for displacement class d of spin sp.
__device__ __forceinline__ const float* g0f_row(const ProblemDev& p, int sp, int d) {
  return p.g0f + ((size_t)sp * p.nc + d) * (size_t)(p.n_tau + 1);
}

// e^{V} of a vertex with stored auxiliary spin s: s = 0 marks a dead
// (non-interacting) vertex, V = 0.
__device__ __forceinline__ double expV(const ProblemDev& p, int sp, int s) {
  return s == 0 ? 1.0 : p.expV[sp][s > 0 ? 1 : 0];
}

// Double-float arithmetic on the FP32 pipes (an unevaluated pair hi + lo,
// ~2^-44 relative): GB300 issues 64 FP32 operations per FP64 FMA.  The _rn
// forms are never contracted into FMAs, which the error-free transformations
// rely on (Dekker / Knuth: exact product by FMA, two-sum).
__device__ __forceinline__ float2 df_split(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// (shi, slo) += (ahi + alo)(bhi + blo), dropping alo * blo.
__device__ __forceinline__ void df_fma(float& shi, float& slo, float ahi, float alo, float bhi, float blo) {
  const float p = __fmul_rn(ahi, bhi);
  float e = fmaf(ahi, bhi, -p);
  e = fmaf(ahi, blo, e);
  e = fmaf(alo, bhi, e);
  const float s1 = __fadd_rn(shi, p);
  const float bb = __fsub_rn(s1, shi);
  const float err = __fadd_rn(__fsub_rn(shi, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
  shi = s1;
  slo = __fadd_rn(slo, __fadd_rn(err, e));
}

// Normalised pair (|lo| <= ulp(hi) / 2) of hi + lo.
__device__ __forceinline__ float2 df_norm(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}

// Load of a stored value directly in the arithmetic type A (no FP64 round
// trip for FP32 storage: on GB300 every FP64 conversion costs an FP64 issue).
template <typename A, typename T>
__device__ __forceinline__ A ldA(const T* p, size_t i) {
  return (A)p[i];
}

// Storage of N: FP64 or FP32 (mixed precision); arithmetic around it is FP64.
__device__ __forceinline__ double ldN(const double* p, size_t i) { return p[i]; }
__device__ __forceinline__ double ldN(const float* p, size_t i) { return (double)p[i]; }
__device__ __forceinline__ void stN(double* p, size_t i, double v) { p[i] = v; }
__device__ __forceinline__ void stN(float* p, size_t i, double v) { p[i] = (float)v; }

// Persistent, load-balanced iteration over the work items of `nsets` sets
// (walker-spin pairs, or walkers): set s has count(s) items, and item t of
// set s is global item prefix(s) + t, taken by block (global item) mod
// gridDim.x.  The block evaluates the counts of up to FE_CHUNK sets in
// parallel and scans them in shared memory (a serial walk over the walker
// records costs one dependent global load per set and dominated idle
// launches); items find their set by binary search.  All loop variables are
// uniform over the block, so `body` may use __syncthreads().  blockDim.x must
// be a multiple of 32; a set holds fewer than 2^31 items and a chunk's total
// fits in an int.
constexpr int FE_CHUNK = 1024;

template <typename CountF, typename BodyF>
__device__ __forceinline__ void for_each_item(int nsets, CountF count, BodyF body) {
  __shared__ int fe_pre[FE_CHUNK + 1];  // exclusive prefix of the chunk's counts
  __shared__ int fe_warp[32];
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const long long G = gridDim.x;
  long long base = 0;  // items of the earlier chunks (uniform over the block)
  for (int s0 = 0; s0 < nsets; s0 += FE_CHUNK) {
    const int m = min(FE_CHUNK, nsets - s0);
    __syncthreads();  // earlier readers of fe_pre are done
    // 1. each thread counts a contiguous segment of the chunk's sets
    const int per = (m + nthr - 1) / nthr;
    const int k0 = min(m, tid * per), k1 = min(m, k0 + per);
    int own = 0;
    for (int k = k0; k < k1; ++k) {
      const int c = (int)count(s0 + k);
      fe_pre[k] = c;
      own += c;
    }
    // 2. block-wide scan of the segment totals (warp shuffles, then over warps)
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) fe_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int v = lane < nw ? fe_warp[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (lane < nw) fe_warp[lane] = v;
    }
    __syncthreads();
    // 3. counts -> exclusive prefix, each thread on its own segment
    int run = incl - own + (warp > 0 ? fe_warp[warp - 1] : 0);
    for (int k = k0; k < k1; ++k) {
      const int c = fe_pre[k];
      fe_pre[k] = run;
      run += c;
    }
    const int total = fe_warp[nw - 1];
    if (tid == 0) fe_pre[m] = total;
    __syncthreads();
    // 4. this block's items: global g in [base, base + total) with g = blockIdx (mod G)
    for (long long g = base + ((((long long)blockIdx.x - base) % G) + G) % G; g < base + total; g += G) {
      const int local = (int)(g - base);
      int lo = 0, hi = m;  // fe_pre[lo] <= local < fe_pre[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (fe_pre[mid] <= local) lo = mid;
        else hi = mid;
      }
      body(s0 + lo, local - fe_pre[lo]);
    }
    base += total;
  }
}

__host__ __device__ __forceinline__ long long blocks_of(long long items, int per) { return (items + per - 1) / per; }

}  // namespace dca
