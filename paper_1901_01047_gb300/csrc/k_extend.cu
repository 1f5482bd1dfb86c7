// k_extend.cu -- candidate extension of the mixed-precision path as two
// register-tiled FP32 products over N (no atomics; each output written once),
// Sec. 2.3 "Submatrix updates":
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

constexpr int XB = 128;  // rows of N (k_ext_g) or columns of N (k_ext_x) per item
constexpr int XC = 32;   // candidates per item
constexpr int XK = 32;   // K step (columns of N for G, rows of N for X)

__device__ __forceinline__ bool ext_active(const WalkerDev& w) { return w.active && w.n_cand > 0; }

__device__ __forceinline__ long long ext_items(const WalkerDev& w) {
  return ext_active(w) ? (long long)((w.n + XB - 1) / XB) * ((w.n_cand + XC - 1) / XC) : 0;
}

// G_ext[i, n + c] = sum_j N[i, j] V[c, j] for a 128-row block and 32
// candidates.  Per K step of 32 columns: Nt[k][i] (N transposed) and
// Vs[k][c] (V transposed); thread (tc, tr) of (8, 32) owns rows 4 tr .. 4 tr + 3
// and candidates 4 tc .. 4 tc + 3: two 16-byte shared loads per 16 FMAs.
__global__ void __launch_bounds__(256) k_ext_g(Config cfg) {
  __shared__ __align__(16) float Nt[XK][XB + 4];  // padded: 4-way conflicts on the transposing fill
  __shared__ __align__(16) float Vs[XK][XC + 4];
  for_each_item(
      2 * cfg.n_walkers, [&](int s) -> long long { return ext_items(cfg.W[s >> 1]); },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, nc_ = w.n_cand, ld = w.cap;
        const int rblocks = (n + XB - 1) / XB;
        const int cb = (item / rblocks) * XC, i0 = (item - (item / rblocks) * rblocks) * XB;
        const float* N = (const float*)w.N[w.parity][sp];
        const float* V = reinterpret_cast<const float*>(w.Vb[sp]);
        const int tid = threadIdx.x, tc = tid >> 5, tr = tid & 31;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
        for (int k0 = 0; k0 < n; k0 += XK) {
          __syncthreads();
          for (int e = tid; e < XB * XK; e += 256) {
            const int r = e / XK, k = e - r * XK;  // k fastest: rows of N
            Nt[k][r] = (i0 + r < n && k0 + k < n) ? N[(size_t)(i0 + r) * ld + k0 + k] : 0.f;
          }
          for (int e = tid; e < XC * XK; e += 256) {
            const int c = e / XK, k = e - c * XK;  // k fastest: rows of V
            Vs[k][c] = (cb + c < nc_ && k0 + k < n) ? V[(size_t)(cb + c) * ld + k0 + k] : 0.f;
          }
          __syncthreads();
#pragma unroll 8
          for (int k = 0; k < XK; ++k) {
            const float4 v = *reinterpret_cast<const float4*>(&Vs[k][4 * tc]);
            const float4 a4 = *reinterpret_cast<const float4*>(&Nt[k][4 * tr]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              acc[r][0] += av[r] * v.x;
              acc[r][1] += av[r] * v.y;
              acc[r][2] += av[r] * v.z;
              acc[r][3] += av[r] * v.w;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = i0 + 4 * tr + r;
          if (i < n)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int c = cb + 4 * tc + q;
              if (c < nc_) w.Gc[sp][(size_t)c * ld + i] = (double)acc[r][q];
            }
        }
      });
}

// X[c, j] = sum_i U[c, i] N[i, j] for a 128-column block and 32 candidates.
// Per K step of 32 rows: Ns[k][j] (row segments of N, coalesced) and Us[k][c]
// (U transposed); thread (tc, tj) of (8, 32) owns columns 4 tj .. 4 tj + 3
// and candidates 4 tc .. 4 tc + 3: two 16-byte shared loads per 16 FMAs.
__global__ void __launch_bounds__(256) k_ext_x(Config cfg) {
  __shared__ __align__(16) float Ns[XK][XB];
  __shared__ __align__(16) float Us[XK][XC + 4];
  for_each_item(
      2 * cfg.n_walkers, [&](int s) -> long long { return ext_items(cfg.W[s >> 1]); },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, nc_ = w.n_cand, ld = w.cap;
        const int jblocks = (n + XB - 1) / XB;
        const int cb = (item / jblocks) * XC, j0 = (item - (item / jblocks) * jblocks) * XB;
        const float* N = (const float*)w.N[w.parity][sp];
        const float* U = reinterpret_cast<const float*>(w.Ub[sp]);
        const int tid = threadIdx.x, tc = tid >> 5, tj = tid & 31;
        float acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        for (int k0 = 0; k0 < n; k0 += XK) {
          __syncthreads();
          for (int e = tid; e < XK * (XB / 4); e += 256) {
            const int k = e / (XB / 4), q4 = e - k * (XB / 4);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k0 + k < n) {
              const float* row = N + (size_t)(k0 + k) * ld;
              const int j = j0 + 4 * q4;
              if (j + 3 < n) {
                v = *reinterpret_cast<const float4*>(row + j);
              } else {
                if (j < n) v.x = row[j];
                if (j + 1 < n) v.y = row[j + 1];
                if (j + 2 < n) v.z = row[j + 2];
              }
            }
            *reinterpret_cast<float4*>(&Ns[k][4 * q4]) = v;
          }
          for (int e = tid; e < XC * XK; e += 256) {
            const int c = e / XK, k = e - c * XK;  // k fastest: rows of U
            Us[k][c] = (cb + c < nc_ && k0 + k < n) ? U[(size_t)(cb + c) * ld + k0 + k] : 0.f;
          }
          __syncthreads();
#pragma unroll 8
          for (int k = 0; k < XK; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(&Ns[k][4 * tj]);
            const float4 u4 = *reinterpret_cast<const float4*>(&Us[k][4 * tc]);
            const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[q][0] += uv[q] * a.x;
              acc[q][1] += uv[q] * a.y;
              acc[q][2] += uv[q] * a.z;
              acc[q][3] += uv[q] * a.w;
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = cb + 4 * tc + q;
          if (c < nc_)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const int j = j0 + 4 * tj + m;
              if (j < n) reinterpret_cast<float*>(w.Xr[sp])[(size_t)c * ld + j] = acc[q][m];
            }
        }
      });
}

int launch_ext_mixed(const Config& cfg, int max_cap, cudaStream_t st) {
  const long long S = 2LL * cfg.n_walkers;
  const long long items = sm_grid(S * ((max_cap + XB - 1) / XB) * ((cfg.ks + XC - 1) / XC), 8);
  if (cfg.ext_tc) {
    launch_ext_g_tc(cfg, st);
    launch_ext_x_tc(cfg, st);
  } else {
    k_ext_g<<<(int)items, 256, 0, st>>>(cfg);
    k_ext_x<<<(int)items, 256, 0, st>>>(cfg);
  }
  return 2;
}

}  // namespace dca
