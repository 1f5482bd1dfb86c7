// k_extend.cu -- candidate extension of the mixed-precision path as two
// streaming passes over the FP32 N (no atomics, float4 loads, FP32
// arithmetic), Sec. 2.3 "Submatrix updates":
//   k_ext_g   G_ext[i, n + c] = sum_j N[i, j] V[c, j],   V[c, j] = g0(r_j - r_c, tau_j - tau_c)
//   k_ext_x   X[c, j]         = sum_i U[c, i] N[i, j],   U[c, i] = g0(r_c - r_i, tau_c - tau_i) (e^{V_i} - 1)
// V and U are the FP32 tables written by k_cand_zero (zero on dead vertices,
// whose rows and columns therefore drop out).  The FP64 path keeps the tiled
// one-pass kernel k_cand_ext.
#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace dca {

constexpr int XG_ROWS = 16;  // rows of N per item of k_ext_g (2 per warp)
constexpr int XG_CC = 32;    // candidates per pass of k_ext_g
constexpr int XG_J = 128;    // columns per chunk (4 per lane)
constexpr int XX_J = 128;    // columns per item of k_ext_x (4 per lane)
constexpr int XX_CC = 16;    // candidates per pass of k_ext_x
constexpr int XX_IR = 64;    // rows of U staged at a time

__device__ __forceinline__ bool ext_active(const WalkerDev& w) { return w.active && w.n_cand > 0; }

// Four consecutive floats of a row from column j; zero past column n.
__device__ __forceinline__ float4 ld4_row(const float* row, int j, int n) {
  if (j + 3 < n) return *reinterpret_cast<const float4*>(row + j);
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (j < n) r.x = row[j];
  if (j + 1 < n) r.y = row[j + 1];
  if (j + 2 < n) r.z = row[j + 2];
  return r;
}

// On entry every lane holds 32 partial values; on exit lane l holds the sum
// over the warp of value l (recursive halving: 31 shuffles).
__device__ __forceinline__ float warp_reduce_transpose32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = upper ? v[k] : v[k + o];
      const float keep = upper ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// Item = (walker-spin, 16-row block of N).  Warp w owns rows 2w, 2w + 1; lane
// l owns columns 4l .. 4l + 3 of every 128-column chunk; V is staged in
// shared memory one chunk (32 candidates x 128 columns) at a time.
__global__ void __launch_bounds__(256) k_ext_g(Config cfg) {
  __shared__ __align__(16) float Vs[XG_CC][XG_J];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return ext_active(w) ? (long long)((w.n + XG_ROWS - 1) / XG_ROWS) * ((w.n_cand + XG_CC - 1) / XG_CC) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, nc_ = w.n_cand, ld = w.cap;
        const int rblocks = (n + XG_ROWS - 1) / XG_ROWS;
        const int cb = (item / rblocks) * XG_CC, rb = item - (item / rblocks) * rblocks;
        const float* N = (const float*)w.N[w.parity][sp];
        const float* V = reinterpret_cast<const float*>(w.Vb[sp]);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int r0 = rb * XG_ROWS + 2 * warp;
        float acc0[XG_CC], acc1[XG_CC];
#pragma unroll
        for (int c = 0; c < XG_CC; ++c) acc0[c] = acc1[c] = 0.f;
        for (int j0 = 0; j0 < n; j0 += XG_J) {
          __syncthreads();
          for (int e = threadIdx.x; e < XG_CC * (XG_J / 4); e += 256) {
            const int c = e / (XG_J / 4), q = e - c * (XG_J / 4);
            const float4 v = (cb + c < nc_) ? ld4_row(V + (size_t)(cb + c) * ld, j0 + 4 * q, n)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(&Vs[c][4 * q]) = v;
          }
          __syncthreads();
          const int j = j0 + 4 * lane;
          const float4 a = r0 < n ? ld4_row(N + (size_t)r0 * ld, j, n) : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 b = r0 + 1 < n ? ld4_row(N + (size_t)(r0 + 1) * ld, j, n) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int c = 0; c < XG_CC; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(&Vs[c][4 * lane]);
            acc0[c] += a.x * v.x + a.y * v.y + a.z * v.z + a.w * v.w;
            acc1[c] += b.x * v.x + b.y * v.y + b.z * v.z + b.w * v.w;
          }
        }
        const float g0v = warp_reduce_transpose32(acc0, lane);
        const float g1v = warp_reduce_transpose32(acc1, lane);
        const int c = cb + lane;
        if (c < nc_) {
          if (r0 < n) w.Gc[sp][(size_t)c * ld + r0] = (double)g0v;
          if (r0 + 1 < n) w.Gc[sp][(size_t)c * ld + r0 + 1] = (double)g1v;
        }
      });
}

// Item = (walker-spin, 128-column block of N, 16-candidate chunk).  Lane l
// owns columns 4l .. 4l + 3; warp w takes rows w, w + 8, ...; U is staged as
// U^T (64 rows x 16 candidates) and the eight warps' partial sums are added
// in shared memory.
__global__ void __launch_bounds__(256) k_ext_x(Config cfg) {
  __shared__ __align__(16) float Us[XX_IR][XX_CC];
  __shared__ float red[XX_CC][XX_J];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return ext_active(w) ? (long long)((w.n + XX_J - 1) / XX_J) * ((w.n_cand + XX_CC - 1) / XX_CC) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, nc_ = w.n_cand, ld = w.cap;
        const int jblocks = (n + XX_J - 1) / XX_J;
        const int cb = (item / jblocks) * XX_CC, j0 = (item - (item / jblocks) * jblocks) * XX_J;
        const float* N = (const float*)w.N[w.parity][sp];
        const float* U = reinterpret_cast<const float*>(w.Ub[sp]);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int j = j0 + 4 * lane;
        __syncthreads();  // the previous item of this block is done with red
        for (int e = threadIdx.x; e < XX_CC * XX_J; e += 256) red[e / XX_J][e % XX_J] = 0.f;
        float acc[XX_CC][4];
#pragma unroll
        for (int c = 0; c < XX_CC; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.f;
        for (int i0 = 0; i0 < n; i0 += XX_IR) {
          __syncthreads();
          for (int e = threadIdx.x; e < XX_IR * XX_CC; e += 256) {
            const int ii = e % XX_IR, c = e / XX_IR;  // ii fastest: coalesced rows of U
            Us[ii][c] = (cb + c < nc_ && i0 + ii < n) ? U[(size_t)(cb + c) * ld + i0 + ii] : 0.f;
          }
          __syncthreads();
          const int iend = min(XX_IR, n - i0);
          for (int ii = warp; ii < iend; ii += 8) {
            const float4 a = ld4_row(N + (size_t)(i0 + ii) * ld, j, n);
#pragma unroll
            for (int c4 = 0; c4 < XX_CC / 4; ++c4) {
              const float4 u = *reinterpret_cast<const float4*>(&Us[ii][4 * c4]);
              const float uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                acc[4 * c4 + q][0] += uu[q] * a.x;
                acc[4 * c4 + q][1] += uu[q] * a.y;
                acc[4 * c4 + q][2] += uu[q] * a.z;
                acc[4 * c4 + q][3] += uu[q] * a.w;
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < XX_CC; ++c)
#pragma unroll
          for (int q = 0; q < 4; ++q) atomicAdd(&red[c][4 * lane + q], acc[c][q]);
        __syncthreads();
        for (int e = threadIdx.x; e < XX_CC * XX_J; e += 256) {
          const int c = e / XX_J, jj = e - c * XX_J;
          if (cb + c < nc_ && j0 + jj < n) w.Xr[sp][(size_t)(cb + c) * ld + j0 + jj] = (double)red[c][jj];
        }
      });
}

void launch_ext_mixed(const Config& cfg, int max_cap, cudaStream_t st) {
  const long long S = 2LL * cfg.n_walkers;
  const long long kcc = (cfg.ks + XG_CC - 1) / XG_CC, kxc = (cfg.ks + XX_CC - 1) / XX_CC;
  long long ig = S * ((max_cap + XG_ROWS - 1) / XG_ROWS) * kcc, ix = S * ((max_cap + XX_J - 1) / XX_J) * kxc;
  constexpr long long kPersist = 4 * 152;
  ig = ig < 1 ? 1 : (ig < kPersist ? ig : kPersist);
  ix = ix < 1 ? 1 : (ix < kPersist ? ix : kPersist);
  k_ext_g<<<(int)ig, 256, 0, st>>>(cfg);
  k_ext_x<<<(int)ix, 256, 0, st>>>(cfg);
}

}  // namespace dca
