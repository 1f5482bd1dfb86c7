// k_refine.cu -- periodic recompute of the FP32 N matrices (mixed
// precision) as a Newton-Schulz step against the from-scratch inverse
// N^-1 = A = e^V - g0 (e^V - 1) of the current configuration (Eq. Zk), which
// k_build_A forms in FP64 and stores as FP32 pairs (hi, lo):
//     R  = I - A N0      FP64-grade (double-float products and sums)
//     N1 = N0 + N0 R     FP32 (R is of the size of the drift)
// One step squares the relative error of N0: an FP32 N0 that drifted by 1e-5
// comes back to the FP32 rounding level.  Both products are tiled GEMMs on a
// persistent grid over (walker-spin, 64 x 64 output tile), so one walker's
// recompute spreads over every SM.  The residual is the whole cost; it runs
// on the FP32 pipes in double-float arithmetic because GB300's FP64 units
// issue ~2 FMA per clock per SM against 128 FP32 operations.
//
// Buffers (the recompute follows a compaction, all n rows live):
//   A   Ascr[sp] (FP32 pairs)    -> R  into N[parity ^ 1][sp] (FP32)
//   N0  N[parity][sp]            -> N1 into Ascr[sp] viewed as FP32
// k_refine_adopt then measures the drift max|N1 - N0| / max|N1| and copies
// N1 into N[parity ^ 1][sp] for the parity switch.
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace dca {

constexpr int RT = 64;   // output tile
constexpr int RK = 16;   // K step of the FP64 product

__device__ __forceinline__ bool refine_wants(const WalkerDev& w) {
  return w.active && w.recompute_pending && w.status == ST_OK;
}

__device__ __forceinline__ long long refine_tiles(const WalkerDev& w) {
  const long long t = (w.n + RT - 1) / RT;
  return refine_wants(w) ? t * t : 0;
}

// R = I - A N0 with FP64-grade accuracy in double-float arithmetic on the
// FP32 pipes (GB300 issues 64 FP32 operations per FP64 FMA).  A arrives as
// FP32 pairs (hi, lo) from k_build_A, N0 is FP32 (exact).  Per term:
// the product hi*b is split exactly by an FMA (p + e), lo*b joins the error
// term, and p is added to the running sum by an error-free two-sum whose
// rounding error also goes to the low word: the accumulated value carries
// ~2^-44 relative error of sum |A||N0|, against the ~1e-5 drift the step
// removes.  Thread (tx, ty) of 16 x 16 owns rows ty + 16 a and columns
// tx + 16 b (a, b < 4) of the tile.
__global__ void __launch_bounds__(256) k_refine_resid(Config cfg) {
  __shared__ float Ah[RK][RT + 1];  // [k][i]
  __shared__ float Al[RK][RT + 1];
  __shared__ float Bs[RK][RT];      // [k][j]
  for_each_item(
      2 * cfg.n_walkers, [&](int s) -> long long { return refine_tiles(cfg.W[s >> 1]); },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap;
        const int tiles = (n + RT - 1) / RT;
        const int i0 = (item / tiles) * RT, j0 = (item - (item / tiles) * tiles) * RT;
        const float2* A = reinterpret_cast<const float2*>(w.Ascr[sp]);
        const float* N0 = (const float*)w.N[w.parity][sp];
        float* R = (float*)w.N[w.parity ^ 1][sp];
        const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
        float hi[4][4], lo[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.0f;
        for (int k0 = 0; k0 < n; k0 += RK) {
          __syncthreads();
          for (int e = threadIdx.x; e < RT * RK; e += 256) {
            const int i = e / RK, k = e - i * RK;  // k fastest: rows of A
            const float2 v = (i0 + i < n && k0 + k < n) ? A[(size_t)(i0 + i) * ld + k0 + k] : make_float2(0.f, 0.f);
            Ah[k][i] = v.x;
            Al[k][i] = v.y;
            const int kk = e / RT, j = e - kk * RT;  // j fastest: rows of N0
            Bs[kk][j] = (k0 + kk < n && j0 + j < n) ? N0[(size_t)(k0 + kk) * ld + j0 + j] : 0.0f;
          }
          __syncthreads();
#pragma unroll 4
          for (int k = 0; k < RK; ++k) {
            float ah[4], al[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              ah[a] = Ah[k][ty + 16 * a];
              al[a] = Al[k][ty + 16 * a];
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                // the _rn forms are never contracted into FMAs, which the
                // error-free transformations below rely on
                const float p = __fmul_rn(ah[a], bv[b]);
                float e = fmaf(ah[a], bv[b], -p);  // exact: ah * b = p + e
                e = fmaf(al[a], bv[b], e);
                const float s1 = __fadd_rn(hi[a][b], p);  // two-sum of hi and p
                const float bb = __fsub_rn(s1, hi[a][b]);
                const float err = __fadd_rn(__fsub_rn(hi[a][b], __fsub_rn(s1, bb)), __fsub_rn(p, bb));
                hi[a][b] = s1;
                lo[a][b] += err + e;
              }
          }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int i = i0 + ty + 16 * a;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int j = j0 + tx + 16 * b;
            if (i < n && j < n) {
              // (delta - hi) - lo, the difference of nearly equal numbers taken exactly first
              const float d = __fsub_rn(i == j ? 1.0f : 0.0f, hi[a][b]);
              R[(size_t)i * ld + j] = __fsub_rn(d, lo[a][b]);
            }
          }
        }
      });
}

// N1 = N0 + N0 R, FP32, into Ascr[sp] viewed as FP32 (ld = cap).  Item =
// 128 x 128 output tile; thread (tx, ty) of 16 x 16 owns rows ty 4 + a +
// 64 p and columns tx 4 + b + 64 q (a, b < 4; p, q < 2): 64 accumulators and
// four 16-byte shared-memory reads per 64 FMAs.  The next K step's tiles are
// loaded into registers while the current one is multiplied.
constexpr int CT = 128;  // output tile
constexpr int CK = 16;   // K step

__global__ void __launch_bounds__(256) k_refine_correct(Config cfg) {
  __shared__ __align__(16) float As[CK][CT + 4];  // [k][i] of N0
  __shared__ __align__(16) float Bs[CK][CT + 4];  // [k][j] of R
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        const long long t = (w.n + CT - 1) / CT;
        return refine_wants(w) ? t * t : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap;
        const int tiles = (n + CT - 1) / CT;
        const int i0 = (item / tiles) * CT, j0 = (item - (item / tiles) * tiles) * CT;
        const float* N0 = (const float*)w.N[w.parity][sp];
        const float* R = (const float*)w.N[w.parity ^ 1][sp];
        float* N1 = (float*)w.Ascr[sp];
        const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
        float ra[8], rb[8];  // the next K step: A rows (k fastest), R rows (j fastest)
        auto fetch = [&](int k0) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int e = tid + 256 * q;
            const int ia = e >> 4, ka = e & 15;   // A: 128 rows x 16 k
            ra[q] = (i0 + ia < n && k0 + ka < n) ? N0[(size_t)(i0 + ia) * ld + k0 + ka] : 0.0f;
            const int kb = e >> 7, jb = e & 127;  // R: 16 k x 128 columns
            rb[q] = (k0 + kb < n && j0 + jb < n) ? R[(size_t)(k0 + kb) * ld + j0 + jb] : 0.0f;
          }
        };
        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
        fetch(0);
        for (int k0 = 0; k0 < n; k0 += CK) {
          __syncthreads();  // the previous K step (or item) is done with the tiles
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int e = tid + 256 * q;
            As[e & 15][e >> 4] = ra[q];
            Bs[e >> 7][e & 127] = rb[q];
          }
          __syncthreads();
          if (k0 + CK < n) fetch(k0 + CK);
#pragma unroll
          for (int k = 0; k < CK; ++k) {
            float av[8], bv[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][64 + tx * 4]);
            av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
            av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
            bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
            bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
              for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
          }
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int i = i0 + ty * 4 + (a & 3) + 64 * (a >> 2);
          if (i >= n) continue;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int j = j0 + tx * 4 + 64 * q;  // 16-byte aligned: ld and j0 are multiples of 4
            const size_t o = (size_t)i * ld + j;
            if (j + 3 < n) {
              float4 v = *reinterpret_cast<const float4*>(N0 + o);
              v.x += acc[a][4 * q];
              v.y += acc[a][4 * q + 1];
              v.z += acc[a][4 * q + 2];
              v.w += acc[a][4 * q + 3];
              *reinterpret_cast<float4*>(N1 + o) = v;
            } else {
#pragma unroll
              for (int b = 0; b < 4; ++b)
                if (j + b < n) N1[o + b] = N0[o + b] + acc[a][4 * q + b];
            }
          }
        }
      });
}

// Drift max|N1 - N0| and max|N1| (atomicMax on the bits of non-negative
// doubles, folded into the walker by k_recompute_adopt) and the copy of N1
// into N[parity ^ 1].  Persistent grid, 2048 entries per item.
__global__ void __launch_bounds__(256) k_refine_adopt(Config cfg) {
  __shared__ double s_d[8], s_n[8];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return refine_wants(w) ? blocks_of((long long)w.n * w.n, 2048) : 0;
      },
      [&](int s, int item) {
        WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap;
        const float* N0 = (const float*)w.N[w.parity][sp];
        const float* N1 = (const float*)w.Ascr[sp];
        float* dst = (float*)w.N[w.parity ^ 1][sp];
        double dmax = 0.0, nmax = 0.0;
        const long long e0 = (long long)item * 2048, e1 = min(e0 + 2048, (long long)n * n);
        for (long long idx = e0 + threadIdx.x; idx < e1; idx += 256) {
          const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
          const size_t o = (size_t)i * ld + j;
          const float b = N1[o];
          dmax = fmax(dmax, fabs((double)b - (double)N0[o]));
          nmax = fmax(nmax, fabs((double)b));
          dst[o] = b;
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

static int refine_grid(long long items) { return sm_grid(items, 4); }

void launch_refine_gemms(const Config& cfg, int max_cap, cudaStream_t st) {
  // every block resident at once (the residual holds 3 blocks per SM): a grid
  // past the resident blocks would run its last blocks' items as a second wave
  const long long t = (max_cap + RT - 1) / RT;
  const long long items = 2LL * cfg.n_walkers * t * t;
  k_refine_resid<<<persist_grid((const void*)k_refine_resid, items, 256), 256, 0, st>>>(cfg);
  launch_refine_correct(cfg, max_cap, st);
}

void launch_refine_correct(const Config& cfg, int max_cap, cudaStream_t st) {
  const long long t = (max_cap + CT - 1) / CT;
  const long long items = 2LL * cfg.n_walkers * t * t;
  k_refine_correct<<<persist_grid((const void*)k_refine_correct, items, 256), 256, 0, st>>>(cfg);
}

void launch_refine_adopt(const Config& cfg, int max_cap, cudaStream_t st) {
  k_refine_adopt<<<refine_grid(2LL * cfg.n_walkers * blocks_of((long long)max_cap * max_cap, 2048)), 256, 0, st>>>(
      cfg);
}

}  // namespace dca
