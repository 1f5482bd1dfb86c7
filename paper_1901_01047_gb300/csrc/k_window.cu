// k_window.cu -- one submatrix update ("window") of every walker, FP64.
//
// Sequence per window (DCA++ paper Sec. 2.3, "Submatrix updates"):
//   k_begin       proposals of the window from Philox (counter tag 0 / 1);
//                 insertion candidates appended as non-interacting rows
//   k_cand_g      G_ext[i, n+c] = sum_j N[i,j] g0(r_j - r_c, tau_j - tau_c)
//   k_cand_x      X[c, j]     = sum_i g0(r_c - r_i, tau_c - tau_i) (e^{V_i} - 1) N[i,j]
//   k_cand_cc     G_ext[n+c', n+c] = X[c',:] . g0[:, c] + g0(c', c)
//   k_metropolis  serial single-spin decisions from B_P^-1 (bordered growth)
//   k_upd_*       N <- N + (G[:,P] - E_P) diag(a_P) B^-1 N[P,:] on the
//                 surviving rows / columns, written compacted to the other
//                 buffer (compaction of non-interacting spins fused in)
//   k_window_end  compact the vertex list, swap buffers
#include <cstdint>
#include <cstdio>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace dca {

// ---------------------------------------------------------------------------
// k_begin: one block per walker.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_begin(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  __shared__ int s_active, s_len, s_n, s_cap, s_par;
  __shared__ int s_type[KS_MAX];
  if (threadIdx.x == 0) {
    w.n_acc = 0;
    w.n_removed = 0;
    w.n_eval = 0;
    w.aborted = 0;
    w.n_cand = 0;
    w.measure_pending = 0;
    w.recompute_pending = 0;
    int act = (w.status == ST_OK && w.sweeps_done < w.sweeps_target) ? 1 : 0;
    if (act) {
      if (w.sweep_pos == 0) {
        if (w.sweeps_done < cfg.warmup) {
          w.sweep_len_cur = w.n > 1 ? w.n : 1;
          w.warm_k_sum += w.n;
        } else {
          if (w.sweep_len == 0) {
            const int64_t L = cfg.warmup > 0 ? (2 * w.warm_k_sum + cfg.warmup) / (2 * (int64_t)cfg.warmup)
                                             : (int64_t)w.n;
            w.sweep_len = L > 1 ? L : 1;
          }
          w.sweep_len_cur = w.sweep_len;
        }
      }
      const int64_t rem = w.sweep_len_cur - w.sweep_pos;
      w.win_len = (int)(rem < cfg.ks ? rem : cfg.ks);
    } else {
      w.win_len = 0;
    }
    w.active = act;
    s_active = act;
    s_len = w.win_len;
    s_n = w.n;
    s_cap = w.cap;
    s_par = w.parity;
  }
  __syncthreads();
  if (!s_active) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int j = threadIdx.x;
  Proposal pr;
  if (j < s_len) {
    const uint64_t qj = w.q + (uint64_t)j;
    const Philox4 r = draw(w, qj, TAG_PROPOSAL);
    const Philox4 a = draw(w, qj, TAG_ACCEPT);
    pr.u = uniform53(a.v[0], a.v[1]);
    pr.type = (int)(r.v[0] & 1u);
    pr.s = (r.v[0] & 2u) ? 1 : -1;
    pr.site = (int)scaled_index(r.v[1], (uint32_t)pb.nc);
    pr.tau = pb.beta * uniform53(r.v[2], r.v[3]);
    pr.word = r.v[1];
    pr.slot = -1;
    pr.pad = 0;
    s_type[j] = pr.type;
  }
  __syncthreads();
  if (j < s_len) {
    int slot = 0;
    for (int i = 0; i < j; ++i) slot += (s_type[i] == 0);
    if (pr.type == 0) pr.slot = slot;
    w.prop[j] = pr;
    if (pr.type == 0) {
      const int row = s_n + slot;
      if (row < s_cap) {
        w.vsite[s_par][row] = pr.site;
        w.vtau[s_par][row] = pr.tau;
        w.vs[s_par][row] = pr.s;
      }
    }
  }
  if (threadIdx.x == 0) {
    int c = 0;
    for (int i = 0; i < s_len; ++i) c += (s_type[i] == 0);
    w.n_cand = c;
    if (s_n + c > s_cap) {
      w.status = ST_ERR_CAPACITY;
      w.active = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Candidate extension GEMMs (FP64, 32x32 tiles, 256 threads).
// grid = (row tiles, candidate tiles, walkers * 2 spins)
// ---------------------------------------------------------------------------
constexpr int TT = 32;

__global__ void __launch_bounds__(256) k_cand_g(Config cfg) {
  const int wi = blockIdx.z >> 1, sp = blockIdx.z & 1;
  const WalkerDev& w = cfg.W[wi];
  if (!w.active) return;
  const int n = w.n, nc_ = w.n_cand;
  const int i0 = blockIdx.x * TT, c0 = blockIdx.y * TT;
  if (i0 >= n || c0 >= nc_) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int ld = w.cap, par = w.parity;
  const double* __restrict__ N = w.N[par][sp];
  const int* vsite = w.vsite[par];
  const double* vtau = w.vtau[par];
  __shared__ double As[TT][TT + 1];
  __shared__ double Bs[TT][TT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < n; k0 += TT) {
    for (int r = ty; r < TT; r += 8) {
      const int i = i0 + r, k = k0 + tx;
      As[r][tx] = (i < n && k < n) ? N[(size_t)i * ld + k] : 0.0;
      // B[k, c] = g0(r_k - r_c, tau_k - tau_c)
      const int kk = k0 + r, c = c0 + tx;
      double b = 0.0;
      if (kk < n && c < nc_) {
        const int rc = vsite[n + c];
        b = g0_pair(pb, sp, vsite[kk], vtau[kk], rc, vtau[n + c]);
      }
      Bs[r][tx] = b;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TT; ++k) {
      const double b = Bs[k][tx];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] += As[ty + 8 * m][k] * b;
    }
    __syncthreads();
  }
  const int c = c0 + tx;
  if (c < nc_) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = i0 + ty + 8 * m;
      if (i < n) w.Gc[sp][(size_t)c * ld + i] = acc[m];
    }
  }
}

__global__ void __launch_bounds__(256) k_cand_x(Config cfg) {
  const int wi = blockIdx.z >> 1, sp = blockIdx.z & 1;
  const WalkerDev& w = cfg.W[wi];
  if (!w.active) return;
  const int n = w.n, nc_ = w.n_cand;
  const int j0 = blockIdx.x * TT, c0 = blockIdx.y * TT;
  if (j0 >= n || c0 >= nc_) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int ld = w.cap, par = w.parity;
  const double* __restrict__ N = w.N[par][sp];
  const int* vsite = w.vsite[par];
  const double* vtau = w.vtau[par];
  const int* vs = w.vs[par];
  __shared__ double Us[TT][TT + 1];   // [c][k]
  __shared__ double Bs[TT][TT + 1];   // [k][j]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < n; k0 += TT) {
    for (int r = ty; r < TT; r += 8) {
      // U[c, k] = g0(r_c - r_k, tau_c - tau_k) (e^{V_k} - 1)
      const int c = c0 + r, k = k0 + tx;
      double u = 0.0;
      if (c < nc_ && k < n)
        u = g0_pair(pb, sp, vsite[n + c], vtau[n + c], vsite[k], vtau[k]) * (expV(pb, sp, vs[k]) - 1.0);
      Us[r][tx] = u;
      const int kk = k0 + r, jj = j0 + tx;
      Bs[r][tx] = (kk < n && jj < n) ? N[(size_t)kk * ld + jj] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TT; ++k) {
      const double b = Bs[k][tx];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] += Us[ty + 8 * m][k] * b;
    }
    __syncthreads();
  }
  const int jj = j0 + tx;
  if (jj < n) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int c = c0 + ty + 8 * m;
      if (c < nc_) w.Xr[sp][(size_t)c * ld + jj] = acc[m];
    }
  }
}

// G_ext[n+c', n+c] = X[c',:] . g0[:, c] + g0(r_c' - r_c, tau_c' - tau_c).
// grid = (KS_MAX candidates c, walkers * 2); block = 128 (4 warps over c').
__global__ void __launch_bounds__(128) k_cand_cc(Config cfg) {
  const int wi = blockIdx.y >> 1, sp = blockIdx.y & 1;
  const WalkerDev& w = cfg.W[wi];
  if (!w.active) return;
  const int c = blockIdx.x;
  const int n = w.n, nc_ = w.n_cand;
  if (c >= nc_) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int ld = w.cap, par = w.parity;
  const int* vsite = w.vsite[par];
  const double* vtau = w.vtau[par];
  const int rc = vsite[n + c];
  const double tc = vtau[n + c];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double v[1024];
  double acc[KS_MAX / 4];
#pragma unroll
  for (int m = 0; m < KS_MAX / 4; ++m) acc[m] = 0.0;
  for (int j0 = 0; j0 < n; j0 += 1024) {
    __syncthreads();
    for (int t = threadIdx.x; t < 1024; t += 128) {
      const int j = j0 + t;
      v[t] = j < n ? g0_pair(pb, sp, vsite[j], vtau[j], rc, tc) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < KS_MAX / 4; ++m) {
      const int cp = warp + 4 * m;
      if (cp < nc_) {
        const double* X = w.Xr[sp] + (size_t)cp * ld;
        double s = 0.0;
        for (int t = lane; t < 1024 && j0 + t < n; t += 32) s += X[j0 + t] * v[t];
        acc[m] += s;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < KS_MAX / 4; ++m) {
    const int cp = warp + 4 * m;
    double s = acc[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && cp < nc_) {
      const double g = (cp == c) ? g0_diag(pb, sp, rc) : g0_pair(pb, sp, vsite[n + cp], vtau[n + cp], rc, tc);
      w.Gc[sp][(size_t)c * ld + n + cp] = s + g;
    }
  }
}

// ---------------------------------------------------------------------------
// Metropolis over the window (one block per walker, both spins).
// ---------------------------------------------------------------------------
struct ExtView {
  const double* N;   // current N (ld)
  const double* X;   // candidate rows [c][ld]
  const double* Gc;  // candidate columns [c][ld]
  const int* vs;
  int n, ld;
};

// G_ext[x, y]; y interacting existing vertex uses G = (N e^{V} - I) / (e^{V} - 1)
// column-wise, which follows from N = [I + G (e^V - I)] e^{-V}.
__device__ __forceinline__ double g_ext(const ExtView& v, const ProblemDev& pb, int sp, int x, int y) {
  if (y >= v.n) return v.Gc[(size_t)(y - v.n) * v.ld + x];
  const double nxy = (x < v.n) ? v.N[(size_t)x * v.ld + y] : v.X[(size_t)(x - v.n) * v.ld + y];
  const double ev = expV(pb, sp, v.vs[y]);
  return (nxy * ev - (x == y ? 1.0 : 0.0)) / (ev - 1.0);
}

__global__ void __launch_bounds__(256) k_metropolis(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = w.active;
  __syncthreads();
  if (!s_active) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int tid = threadIdx.x;
  const int n = w.n, ld = w.cap, par = w.parity, len = w.win_len;
  ExtView ev[2];
  for (int sp = 0; sp < 2; ++sp) {
    ev[sp].N = w.N[par][sp];
    ev[sp].X = w.Xr[sp];
    ev[sp].Gc = w.Gc[sp];
    ev[sp].vs = w.vs[par];
    ev[sp].n = n;
    ev[sp].ld = ld;
  }
  double* Binv[2] = {w.Binv[0], w.Binv[1]};

  __shared__ double s_brow[2][KS_MAX], s_bcol[2][KS_MAX], s_t[2][KS_MAX], s_s[2][KS_MAX];
  __shared__ double s_aP[2][KS_MAX];
  __shared__ int s_P[KS_MAX];
  __shared__ int s_removed[KS_MAX];
  __shared__ double s_anew[2], s_Btt[2], s_d[2];
  __shared__ int s_target, s_kind, s_stop, s_accept, s_l, s_nrem, s_nins, s_kcur, s_eval;
  __shared__ double s_sign;

  if (tid == 0) {
    s_l = 0;
    s_nrem = 0;
    s_nins = 0;
    s_stop = 0;
    s_sign = w.sign;
    s_eval = 0;
  }
  __syncthreads();

  for (int j = 0; j < len; ++j) {
    // 1. target of proposal j
    if (tid == 0) {
      const Proposal pr = w.prop[j];
      const int kcur = n - s_nrem + s_nins;
      int kind = 0, target = -1;
      if (pr.type == 0) {
        kind = 0;
        target = n + pr.slot;
        const int s = pr.s;
        for (int sp = 0; sp < 2; ++sp) s_anew[sp] = expV(pb, sp, s) - 1.0;
      } else if (kcur == 0) {
        kind = 2;
      } else {
        const int idx = (int)scaled_index(pr.word, (uint32_t)kcur);
        const int nexist = n - s_nrem;
        if (idx >= nexist) {
          s_stop = 1;  // picks a spin inserted in this window: end the window here
        } else {
          int x = idx;
          for (int r = 0; r < s_nrem; ++r) {
            if (s_removed[r] <= x) ++x;
            else break;
          }
          kind = 1;
          target = x;
          const int s = ev[0].vs[x];
          for (int sp = 0; sp < 2; ++sp) s_anew[sp] = expV(pb, sp, -s) - 1.0;
        }
      }
      s_kind = kind;
      s_target = target;
      s_kcur = kcur;
    }
    __syncthreads();
    if (s_stop) break;
    const int l = s_l;
    if (s_kind == 2) {
      if (tid == 0) {
        const uint64_t q = w.q + (uint64_t)j;
        if ((int64_t)q < w.log_cap) w.log[q] = 0;
        w.n_prop++;
        s_eval = j + 1;
      }
      __syncthreads();
      continue;
    }
    const int t = s_target;
    // 2. border of B: row / column against P, and the new diagonal entry
    for (int idx = tid; idx < 4 * l + 2; idx += blockDim.x) {
      if (idx < 4 * l) {
        const int sp = idx / (2 * l);
        const int rem = idx - sp * 2 * l;
        const int p = rem >> 1;
        const int P = s_P[p];
        if (rem & 1) {
          // column: B[P_p, t] = -G[P_p, t] a_t
          const double a = s_anew[sp];
          s_bcol[sp][p] = (a == 0.0) ? 0.0 : -g_ext(ev[sp], pb, sp, P, t) * a;
        } else {
          // row: B[t, P_p] = -G[t, P_p] a_{P_p}
          const double a = s_aP[sp][p];
          s_brow[sp][p] = (a == 0.0) ? 0.0 : -g_ext(ev[sp], pb, sp, t, P) * a;
        }
      } else {
        const int sp = idx - 4 * l;
        const double a = s_anew[sp];
        s_Btt[sp] = (a == 0.0) ? 1.0 : 1.0 + (1.0 - g_ext(ev[sp], pb, sp, t, t)) * a;
      }
    }
    __syncthreads();
    // 3. t = Binv b_col
    if (tid < 2 * KS_MAX) {
      const int sp = tid / KS_MAX, i = tid - sp * KS_MAX;
      if (i < l) {
        const double* B = Binv[sp] + (size_t)i * KS_MAX;
        double acc = 0.0;
        for (int p = 0; p < l; ++p) acc += B[p] * s_bcol[sp][p];
        s_t[sp][i] = acc;
      }
    }
    __syncthreads();
    // 4. Schur complement d = B_tt - b_row . t  (warp 0: up, warp 1: down)
    if (tid < 64) {
      const int sp = tid >> 5, lane = tid & 31;
      double acc = 0.0;
      for (int i = lane; i < l; i += 32) acc += s_brow[sp][i] * s_t[sp][i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) s_d[sp] = s_Btt[sp] - acc;
    }
    __syncthreads();
    // 5. decision
    if (tid == 0) {
      const Proposal pr = w.prop[j];
      const uint64_t q = w.q + (uint64_t)j;
      const int kcur = s_kcur;
      const double R = (s_kind == 0 ? pb.K / (double)(kcur + 1) : (double)kcur / pb.K) * s_d[0] * s_d[1];
      int acc = 0, tie = 0;
      if (!isfinite(R)) {
        w.status = ST_ERR_NUMERIC;
        s_stop = 1;
      } else {
        const double absR = fabs(R);
        acc = pr.u < absR;
        tie = fabs(absR - pr.u) < cfg.tie_eps;
        if ((int64_t)q < w.forced_n) acc = w.forced[q] & 1;
        if (acc && R < 0.0) s_sign = -s_sign;
        if ((int64_t)q < w.log_cap) w.log[q] = (uint8_t)(acc | (tie << 1));
        w.n_prop++;
        w.n_ties += tie;
        w.n_accept += acc;
        s_eval = j + 1;
      }
      s_accept = acc;
    }
    __syncthreads();
    if (s_stop) break;
    if (!s_accept) continue;
    // 6. s = b_row Binv
    if (tid < 2 * KS_MAX) {
      const int sp = tid / KS_MAX, jj = tid - sp * KS_MAX;
      if (jj < l) {
        double acc = 0.0;
        for (int i = 0; i < l; ++i) acc += s_brow[sp][i] * Binv[sp][(size_t)i * KS_MAX + jj];
        s_s[sp][jj] = acc;
      }
    }
    __syncthreads();
    // 7. bordered inverse:
    //    [[Binv + t s / d, -t / d], [-s / d, 1 / d]]
    for (int sp = 0; sp < 2; ++sp) {
      const double rd = 1.0 / s_d[sp];
      for (int idx = tid; idx < (l + 1) * (l + 1); idx += blockDim.x) {
        const int i = idx / (l + 1), jj = idx - i * (l + 1);
        double* B = Binv[sp] + (size_t)i * KS_MAX + jj;
        if (i < l && jj < l) *B += s_t[sp][i] * s_s[sp][jj] * rd;
        else if (i < l) *B = -s_t[sp][i] * rd;
        else if (jj < l) *B = -s_s[sp][jj] * rd;
        else *B = rd;
      }
    }
    __syncthreads();
    if (tid == 0) {
      s_P[l] = t;
      s_aP[0][l] = s_anew[0];
      s_aP[1][l] = s_anew[1];
      if (s_kind == 1) {
        // keep the removed list ascending
        int r = s_nrem;
        while (r > 0 && s_removed[r - 1] > t) {
          s_removed[r] = s_removed[r - 1];
          --r;
        }
        s_removed[r] = t;
        s_nrem++;
      } else {
        s_nins++;
      }
      s_l = l + 1;
    }
    __syncthreads();
  }
  __syncthreads();

  // Epilogue: window bookkeeping, accepted set, survivor map.
  const int l = s_l, nrem = s_nrem, nins = s_nins;
  const int n_s = n - nrem + nins;
  for (int p = tid; p < l; p += blockDim.x) {
    w.P[p] = s_P[p];
    w.aP[0][p] = s_aP[0][p];
    w.aP[1][p] = s_aP[1][p];
  }
  for (int r = tid; r < nrem; r += blockDim.x) w.removed[r] = s_removed[r];
  for (int i = tid; i < n; i += blockDim.x) {
    int below = 0, gone = 0;
    for (int r = 0; r < nrem; ++r) {
      below += (s_removed[r] < i);
      gone |= (s_removed[r] == i);
    }
    if (!gone) w.surv[i - below] = i;
  }
  if (tid == 0) {
    int m = n - nrem;
    for (int p = 0; p < l; ++p)
      if (s_P[p] >= n) w.surv[m++] = s_P[p];
    const int eval = s_eval;
    w.n_acc = l;
    w.n_removed = nrem;
    w.n_surv = n_s;
    w.n_eval = eval;
    w.aborted = (eval < len) && w.status == ST_OK;
    w.sign = s_sign;
    if (w.status == ST_OK) {
      w.q += (uint64_t)eval;
      w.sweep_pos += eval;
      w.n_windows++;
      if (w.aborted) w.n_aborts++;
      if (w.sweep_pos >= w.sweep_len_cur) {
        w.measure_pending = (w.sweeps_done >= cfg.warmup) ? 1 : 0;
        w.sweeps_done++;
        w.sweep_pos = 0;
      }
      w.windows_since_recompute++;
      if (cfg.recompute_every > 0 && w.windows_since_recompute >= cfg.recompute_every) {
        w.recompute_pending = 1;
        w.windows_since_recompute = 0;
      }
      const double ns = (double)n_s, ll = (double)l;
      // N update per spin: 2 n_s^2 l + 2 n_s l^2 flop; reads and writes n_s^2
      // entries plus the n_s x l factors (8-byte words).
      if (l > 0) {
        w.flops += 2.0 * (2.0 * ns * ns * ll + 2.0 * ns * ll * ll);
        w.upd_bytes += 2.0 * 8.0 * (2.0 * ns * ns + 2.0 * ns * ll);
      }
      // candidate extension per spin: G columns (n x n x c) and X rows
      // (c x n x n), each reading N once.
      const double nn = (double)n, cc = (double)w.n_cand;
      if (w.n_cand > 0) {
        w.ext_flops += 2.0 * (4.0 * nn * nn * cc);
        w.ext_bytes += 2.0 * 8.0 * (2.0 * nn * nn);
      }
    } else {
      w.active = 0;
      w.n_acc = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// N update on the surviving rows / columns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double n_ext(const ExtView& v, int x, int y) {
  if (x < v.n) return (y < v.n) ? v.N[(size_t)x * v.ld + y] : 0.0;
  if (y < v.n) return v.X[(size_t)(x - v.n) * v.ld + y];
  return x == y ? 1.0 : 0.0;
}

__device__ __forceinline__ ExtView make_view(const WalkerDev& w, int sp) {
  ExtView v;
  v.N = w.N[w.parity][sp];
  v.X = w.Xr[sp];
  v.Gc = w.Gc[sp];
  v.vs = w.vs[w.parity];
  v.n = w.n;
  v.ld = w.cap;
  return v;
}

// Lrow[i', p] = (G_ext[surv(i'), P_p] - delta) a_p ; grid = (row blocks, walkers*2), block 256
__global__ void __launch_bounds__(256) k_upd_lrow(Config cfg) {
  const int wi = blockIdx.y >> 1, sp = blockIdx.y & 1;
  const WalkerDev& w = cfg.W[wi];
  if (!w.active || w.n_acc == 0) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int l = w.n_acc, ns = w.n_surv;
  const ExtView v = make_view(w, sp);
  const int total = ns * l;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int i = idx / l, p = idx - i * l;
    const int x = w.surv[i], P = w.P[p];
    const double a = w.aP[sp][p];
    double val = 0.0;
    if (a != 0.0) val = (g_ext(v, pb, sp, x, P) - (x == P ? 1.0 : 0.0)) * a;
    w.Lrow[sp][(size_t)i * KS_MAX + p] = val;
  }
}

// Lp = Lrow Binv ; Rr[p, j'] = N_ext[P_p, surv(j')]
__global__ void __launch_bounds__(256) k_upd_lp_rr(Config cfg) {
  const int wi = blockIdx.y >> 1, sp = blockIdx.y & 1;
  const WalkerDev& w = cfg.W[wi];
  if (!w.active || w.n_acc == 0) return;
  const int l = w.n_acc, ns = w.n_surv;
  const ExtView v = make_view(w, sp);
  const double* Bi = w.Binv[sp];
  const int total = ns * l;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int i = idx / l, p = idx - i * l;
    const double* Lr = w.Lrow[sp] + (size_t)i * KS_MAX;
    double acc = 0.0;
    for (int q = 0; q < l; ++q) acc += Lr[q] * Bi[(size_t)q * KS_MAX + p];
    w.Lp[sp][(size_t)i * KS_MAX + p] = acc;
  }
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int p = idx / ns, j = idx - p * ns;
    w.Rr[sp][(size_t)p * w.cap + j] = n_ext(v, w.P[p], w.surv[j]);
  }
}

// Nnew[i', j'] = N_ext[surv i', surv j'] + sum_p Lp[i', p] Rr[p, j'].
// grid = (col tiles, row tiles, walkers*2), block 256, 32x32 tile.
__global__ void __launch_bounds__(256) k_upd_apply(Config cfg) {
  const int wi = blockIdx.z >> 1, sp = blockIdx.z & 1;
  const WalkerDev& w = cfg.W[wi];
  if (!w.active || w.n_acc == 0) return;
  const int ns = w.n_surv, l = w.n_acc;
  const int j0 = blockIdx.x * TT, i0 = blockIdx.y * TT;
  if (i0 >= ns || j0 >= ns) return;
  const ExtView v = make_view(w, sp);
  double* Nn = w.N[w.parity ^ 1][sp];
  const int ld = w.cap;
  __shared__ double Ls[TT][TT + 1];  // [i][p]
  __shared__ double Rs[TT][TT + 1];  // [p][j]
  __shared__ int si[TT], sj[TT];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x < TT) {
    const int i = i0 + threadIdx.x;
    si[threadIdx.x] = i < ns ? w.surv[i] : 0;
  } else if (threadIdx.x < 2 * TT) {
    const int j = j0 + threadIdx.x - TT;
    sj[threadIdx.x - TT] = j < ns ? w.surv[j] : 0;
  }
  double acc[4] = {0, 0, 0, 0};
  for (int p0 = 0; p0 < l; p0 += TT) {
    __syncthreads();
    for (int r = ty; r < TT; r += 8) {
      const int i = i0 + r, p = p0 + tx;
      Ls[r][tx] = (i < ns && p < l) ? w.Lp[sp][(size_t)i * KS_MAX + p] : 0.0;
      const int pp = p0 + r, jj = j0 + tx;
      Rs[r][tx] = (pp < l && jj < ns) ? w.Rr[sp][(size_t)pp * ld + jj] : 0.0;
    }
    __syncthreads();
    const int pend = (l - p0) < TT ? (l - p0) : TT;
    for (int p = 0; p < pend; ++p) {
      const double r = Rs[p][tx];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] += Ls[ty + 8 * m][p] * r;
    }
  }
  __syncthreads();
  const int jj = j0 + tx;
  if (jj < ns) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = i0 + ty + 8 * m;
      if (i < ns) Nn[(size_t)i * ld + jj] = n_ext(v, si[ty + 8 * m], sj[tx]) + acc[m];
    }
  }
}

// Compact the vertex list into the other buffer and swap.  grid = walkers.
__global__ void __launch_bounds__(256) k_window_end(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  if (!w.active || w.n_acc == 0) return;
  const int par = w.parity, ns = w.n_surv;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const int x = w.surv[i];
    w.vsite[par ^ 1][i] = w.vsite[par][x];
    w.vtau[par ^ 1][i] = w.vtau[par][x];
    w.vs[par ^ 1][i] = w.vs[par][x];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    w.n = ns;
    w.parity = par ^ 1;
  }
}

__global__ void k_count_active(Config cfg) {
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < cfg.n_walkers; i += blockDim.x) {
    const WalkerDev& w = cfg.W[i];
    if (w.status == ST_OK && w.sweeps_done < w.sweeps_target) atomicAdd(&s_cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *cfg.active_count = s_cnt;
}

__global__ void k_add_target(Config cfg, int64_t n_sweeps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cfg.n_walkers) cfg.W[i].sweeps_target = cfg.W[i].sweeps_done + n_sweeps;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
int launch_window_group(int group, const Config& cfg, int max_cap, cudaStream_t st) {
  const int W = cfg.n_walkers;
  const int rt = (max_cap + TT - 1) / TT;
  const int ct = (cfg.ks + TT - 1) / TT;
  switch (group) {
    case GROUP_PROPOSE:
      k_begin<<<W, 128, 0, st>>>(cfg);
      return 1;
    case GROUP_EXTEND:
      k_cand_g<<<dim3(rt, ct, 2 * W), 256, 0, st>>>(cfg);
      k_cand_x<<<dim3(rt, ct, 2 * W), 256, 0, st>>>(cfg);
      k_cand_cc<<<dim3(cfg.ks, 2 * W), 128, 0, st>>>(cfg);
      return 3;
    case GROUP_METROPOLIS:
      k_metropolis<<<W, 256, 0, st>>>(cfg);
      return 1;
    case GROUP_UPDATE: {
      const int rows = (max_cap * cfg.ks + 255) / 256;
      const int gb = rows < 512 ? rows : 512;
      k_upd_lrow<<<dim3(gb, 2 * W), 256, 0, st>>>(cfg);
      k_upd_lp_rr<<<dim3(gb, 2 * W), 256, 0, st>>>(cfg);
      k_upd_apply<<<dim3(rt, rt, 2 * W), 256, 0, st>>>(cfg);
      k_window_end<<<W, 256, 0, st>>>(cfg);
      return 4;
    }
    default:
      return 0;
  }
}

void launch_count_active(const Config& cfg, cudaStream_t st) { k_count_active<<<1, 256, 0, st>>>(cfg); }

void launch_add_target(const Config& cfg, int64_t n_sweeps, cudaStream_t st) {
  k_add_target<<<(cfg.n_walkers + 127) / 128, 128, 0, st>>>(cfg, n_sweeps);
}

}  // namespace dca

namespace dca {

// Loop control of the device-side window loop (body of a conditional WHILE
// graph node): continue while any walker still has sweeps to do, and stop
// with a timeout flag after max_iters windows (every window advances each
// active walker by at least one proposal, so the host's bound is never
// reached unless something is wrong).
__global__ void k_loop_control(Config cfg, cudaGraphConditionalHandle handle, LoopState* ls) {
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < cfg.n_walkers; i += blockDim.x) {
    const WalkerDev& w = cfg.W[i];
    if (w.status == ST_OK && w.sweeps_done < w.sweeps_target) atomicAdd(&s_cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ls->iters++;
    unsigned int cont = s_cnt > 0 ? 1u : 0u;
    if (cont && ls->iters >= ls->max_iters) {
      ls->timed_out = 1;
      cont = 0u;
    }
    cudaGraphSetConditional(handle, cont);
  }
}

__global__ void k_loop_reset(LoopState* ls, int64_t max_iters) {
  ls->iters = 0;
  ls->max_iters = max_iters;
  ls->timed_out = 0;
}

void launch_loop_control(const Config& cfg, cudaGraphConditionalHandle handle, LoopState* ls, cudaStream_t st) {
  k_loop_control<<<1, 256, 0, st>>>(cfg, handle, ls);
}

void launch_loop_reset(LoopState* ls, int64_t max_iters, cudaStream_t st) { k_loop_reset<<<1, 1, 0, st>>>(ls, max_iters); }

}  // namespace dca
