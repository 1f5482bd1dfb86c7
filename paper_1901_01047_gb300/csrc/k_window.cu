// k_window.cu -- one submatrix update ("window") of every walker.
//
// Sequence per window (DCA++ paper Sec. 2.3, "Submatrix updates"):
//   k_begin       proposals of the window from Philox (counter tag 0 / 1);
//                 insertion candidates appended as non-interacting rows n + c
//   k_cand_ext    one pass over N for both candidate products:
//                 G_ext[i, n+c] = sum_j N[i,j] g0(r_j - r_c, tau_j - tau_c)
//                 X[c, j]     = sum_i g0(r_c - r_i, tau_c - tau_i) (e^{V_i} - 1) N[i,j]
//   k_cand_cc     G_ext[n+c', n+c] = X[c',:] . g0[:, c] + g0(c', c)
//   k_metropolis  serial single-spin decisions from B_P^-1 (bordered growth)
//   k_upd_*       N <- N + (G[:,P] - E_P) diag(a_P) B^-1 N[P,:]: in place on
//                 rows / columns 0..n-1, plus the rows and columns of the
//                 accepted insertions appended at n, n+1, ...
//   k_window_end  removed vertices marked dead, insertions appended to the
//                 vertex list, live-row index and compaction schedule updated
//   k_compact_*   (when due) live rows / columns gathered into the other buffer
// N is stored as T and the dense products (candidate extension, the G block
// of the candidates, L B^-1, the update term) run in arithmetic type A: both
// double on the FP64 path, both float on the mixed path, where the g0
// lookups of the candidate factors also interpolate in FP32 on the split grid
// time.  Ratios, B^-1 and the recompute are always FP64.
#include <cstdint>
#include <cstdio>

#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"
#include "tc_ptx.cuh"

namespace dca {

// ---------------------------------------------------------------------------
// k_begin: one block per walker.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_begin(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  __shared__ int s_active, s_len, s_n, s_cap, s_par;
  __shared__ int s_type[KS_MAX];
  // Lockstep sweeps: a walker works only while the sweeps it has done in the
  // current call equal the smallest such count among the walkers that still
  // have sweeps to do, so every walker starts the m-th sweep of the call in
  // the same window (each chain is unchanged; only the interleaving of the
  // walkers is fixed).  Counting from the call's start keeps walkers whose
  // totals differ (after pooled calls) running together.
  __shared__ unsigned long long s_min;
  if (threadIdx.x == 0) s_min = ~0ull;
  __syncthreads();
  if (!cfg.pooled)
    for (int i = threadIdx.x; i < cfg.n_walkers; i += blockDim.x) {
      const WalkerDev& o = cfg.W[i];
      if (o.status == ST_OK && o.sweeps_done < o.sweeps_target)
        atomicMin(&s_min, (unsigned long long)(o.sweeps_done - o.sweeps_base));
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    w.n_acc = 0;
    w.n_removed = 0;
    w.n_ins = 0;
    w.n_eval = 0;
    w.aborted = 0;
    w.n_cand = 0;
    w.measure_pending = 0;
    w.recompute_pending = 0;
    int act = cfg.pooled ? ((w.status == ST_OK && cfg.pool->go) ? 1 : 0)
                         : ((w.status == ST_OK && w.sweeps_done < w.sweeps_target &&
                             (unsigned long long)(w.sweeps_done - w.sweeps_base) == s_min) ? 1 : 0);
    if (act) {
      w.first_window = w.sweep_pos == 0 ? 1 : 0;
      if (w.sweep_pos == 0) {
        const int k = w.n_live;
        if (w.sweeps_done < cfg.warmup) {
          w.sweep_len_cur = k > 1 ? k : 1;
          w.warm_k_sum += k;
        } else {
          if (w.sweep_len == 0) {
            const int64_t L = cfg.warmup > 0 ? (2 * w.warm_k_sum + cfg.warmup) / (2 * (int64_t)cfg.warmup)
                                             : (int64_t)k;
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
    const bool flip = cfg.flip_thr > 0u && (r.v[0] >> 2) < cfg.flip_thr;
    pr.type = flip ? 2 : (int)(r.v[0] & 1u);
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
      set_status(w, ST_ERR_CAPACITY);
      w.active = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Candidate extension, both products in one pass over N (SIMT).  A 64 x 64
// tile N[I, J] contributes
//   G_ext[I, n+c] += N[I, J] V[J, c],  V[j, c] = g0(r_j - r_c, tau_j - tau_c)
//   X[c, J]       += U[c, I] N[I, J],  U[c, i] = g0(r_c - r_i, tau_c - tau_i) (e^{V_i} - 1)
// and the partial sums are reduced into the FP64 buffers Gc / Xr with
// atomics (zeroed by k_cand_zero).  Dead rows have e^V - 1 = 0 and dead
// columns of N are unit columns, so both are skipped.
// grid = (tiles^2, walkers * 2), block 256, dynamic shared memory.
// ---------------------------------------------------------------------------
constexpr int TT = 32;   // tile of the update kernel
constexpr int METRO_SMEM_KS = 96;  // largest k_s whose B^-1 (both spins) lives in shared memory
constexpr int ET = 64;   // tile of the extension kernel
constexpr int EC = 32;   // candidates per pass

// Persistent grid; one item = 256 vertices i of one walker-spin, all
// candidates c: clears the reduction targets (the FP64 path's Gc / Xr, and
// the candidate-block rows of Gc) and tabulates the candidate factors V and U
// once per window (the tile kernels then read them instead of interpolating;
// the tensor-core path takes U only in its split form).  The mixed path interpolates on the split grid
// time (FP32 arithmetic), the FP64 path in FP64.
__global__ void __launch_bounds__(256) k_cand_zero(Config cfg) {
  __shared__ GridTime s_gc[KS_MAX];
  __shared__ double s_tc[KS_MAX];
  __shared__ int s_rc[KS_MAX];
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        // columns up to n + n_cand (candidate-block targets) and up to the
        // 32-column padding of the tensor-core extension's last K chunk
        return (w.active && w.n_cand > 0) ? blocks_of(max(w.n + w.n_cand, (w.n + 31) & ~31), 256) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, n = w.n, ld = w.cap, nc_ = w.n_cand, par = w.parity;
        const ProblemDev& pb = cfg.P[w.problem];
        const bool mixed = cfg.prec == PREC_MIXED;
        __syncthreads();  // the previous item of this block is done with the candidate table
        for (int c = threadIdx.x; c < nc_; c += 256) {
          s_rc[c] = w.vsite[par][n + c];
          s_tc[c] = w.vtau[par][n + c];
          if (mixed) s_gc[c] = grid_time(s_tc[c], pb.tau_scale);
        }
        __syncthreads();
        const int i = item * 256 + threadIdx.x;
        // split V for the tensor-core extension: [hi | lo] planes x KS_MAX rows x ld columns
        float* Vop = cfg.ext_tc ? reinterpret_cast<float*>(w.Aop[sp]) : nullptr;
        float* Uop = cfg.ext_tc ? reinterpret_cast<float*>(w.Bop[sp]) : nullptr;
        if (i >= n) {
          if (i < n + nc_)  // targets of the candidate block (k_cand_cc adds into them)
            for (int c = 0; c < nc_; ++c) w.Gc[sp][(size_t)c * ld + i] = 0.0;
          if (Vop && i < ((n + 31) & ~31))  // K padding of the last chunk: finite zeros
            for (int c = 0; c < nc_; ++c) {
              Vop[(size_t)c * ld + i] = 0.f;
              Vop[(size_t)(KS_MAX + c) * ld + i] = 0.f;
              Uop[(size_t)c * ld + i] = 0.f;
              Uop[(size_t)(KS_MAX + c) * ld + i] = 0.f;
            }
          return;
        }
        const int si = w.vs[par][i], ri = w.vsite[par][i];
        const double ti = w.vtau[par][i];
        const double em1 = si != 0 ? expV(pb, sp, si) - 1.0 : 0.0;
        const GridTime gi = grid_time(ti, pb.tau_scale);
        const float em1f = (float)em1;
        // unrolled: the table loads of several candidates are in flight together
#pragma unroll 4
        for (int c = 0; c < nc_; ++c) {
          const size_t o = (size_t)c * ld + i;
          if (!mixed) {  // targets of the FP64 path's atomics (the mixed-path kernels store rows < n whole)
            w.Gc[sp][o] = 0.0;
            w.Xr[sp][o] = 0.0;
          }
          const int rc = s_rc[c];
          if (mixed) {
            float v = 0.0f, u = 0.0f;
            if (si != 0) {
              v = g0_interp_grid(g0f_row(pb, sp, __ldg(pb.site_sub + ri * pb.nc + rc)), pb.n_tau, gi, s_gc[c]);
              u = g0_interp_grid(g0f_row(pb, sp, __ldg(pb.site_sub + rc * pb.nc + ri)), pb.n_tau, s_gc[c], gi) * em1f;
            }
            reinterpret_cast<float*>(w.Vb[sp])[o] = v;
            if (!Vop) reinterpret_cast<float*>(w.Ub[sp])[o] = u;  // read only by the CUDA-core X pass
            if (Vop) {
              float hv, lv, hu, lu;
              tc::tf32_split(v, hv, lv);
              tc::tf32_split(u, hu, lu);
              Vop[(size_t)c * ld + i] = hv;
              Vop[(size_t)(KS_MAX + c) * ld + i] = lv;
              Uop[(size_t)c * ld + i] = hu;
              Uop[(size_t)(KS_MAX + c) * ld + i] = lu;
            }
          } else {
            double v = 0.0, u = 0.0;
            if (si != 0) {
              v = g0_pair(pb, sp, ri, ti, rc, s_tc[c]);
              u = g0_pair(pb, sp, rc, s_tc[c], ri, ti) * em1;
            }
            w.Vb[sp][o] = v;
            w.Ub[sp][o] = u;
          }
        }
      });
}

template <typename T, typename A>
__device__ __forceinline__ void cand_ext_tile(const Config& cfg, int wi, int sp, int tile);

// Persistent grid over (walker-spin, 64 x 64 tile of N).
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_cand_ext(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        const long long t = (w.n + ET - 1) / ET;
        return (w.active && w.n_cand > 0) ? t * t : 0;
      },
      [&](int s, int item) { cand_ext_tile<T, A>(cfg, s >> 1, s & 1, item); });
}

template <typename T, typename A>
__device__ __forceinline__ void cand_ext_tile(const Config& cfg, int wi, int sp, int tile) {
  const WalkerDev& w = cfg.W[wi];
  const int n = w.n, nc_ = w.n_cand;
  const int tiles = (n + ET - 1) / ET;
  const int ti = tile / tiles, tj = tile - ti * tiles;
  const int i0 = ti * ET, j0 = tj * ET;
  const int ld = w.cap, par = w.parity;
  const T* __restrict__ N = (const T*)w.N[par][sp];
  // Shared tiles: N[i][j] and its transpose (so that both products read two
  // adjacent outputs' operands with one vector load), V[j][c], U^T[i][c].
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A(*Ns)[ET] = reinterpret_cast<A(*)[ET]>(smem_raw);          // [i][j]
  A(*Vs)[EC] = reinterpret_cast<A(*)[EC]>(Ns + ET);           // [j][c]
  A(*Ut)[EC] = Vs + ET;                                       // [i][c]
  A(*Nt)[ET + 1] = reinterpret_cast<A(*)[ET + 1]>(Ut + ET);   // [j][i], padded: conflict-free transpose
  const int tid = threadIdx.x;
  __syncthreads();  // the previous tile of this block is done with the shared tiles
  for (int e = tid; e < ET * ET; e += 256) {
    const int r = e / ET, cc = e - r * ET;
    const int i = i0 + r, j = j0 + cc;
    const A v = (i < n && j < n) ? ldA<A>(N, (size_t)i * ld + j) : (A)0;
    Ns[r][cc] = v;
    Nt[cc][r] = v;
  }
  // thread: outputs 2 rows (or columns) x 4 candidates
  const int tp = tid & 31, tc = tid >> 5;  // pair index, candidate quad (uniform per warp)
  for (int cb = 0; cb < nc_; cb += EC) {
    __syncthreads();
    for (int e = tid; e < ET * EC; e += 256) {
      const int r = e & (ET - 1), c = e >> 6;  // r fastest: coalesced rows of V and U
      const int j = j0 + r, i = i0 + r, cg = cb + c;
      const bool okc = cg < nc_;
      Vs[r][c] = (okc && j < n) ? reinterpret_cast<const A*>(w.Vb[sp])[(size_t)cg * ld + j] : (A)0;
      Ut[r][c] = (okc && i < n) ? reinterpret_cast<const A*>(w.Ub[sp])[(size_t)cg * ld + i] : (A)0;
    }
    __syncthreads();
    A g[2][4], x[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) g[a][b] = x[a][b] = (A)0;
    // G partial: rows 2 tp, 2 tp + 1 of the tile, candidates 4 tc .. 4 tc + 3 (sum over j);
    // X partial: columns 2 tp, 2 tp + 1, same candidates (sum over i).
#pragma unroll 4
    for (int k = 0; k < ET; ++k) {
      const A n0 = Nt[k][2 * tp], n1 = Nt[k][2 * tp + 1];      // N[2tp][k], N[2tp+1][k]
      const A m0 = Ns[k][2 * tp], m1 = Ns[k][2 * tp + 1];      // N[k][2tp], N[k][2tp+1]
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const A v = Vs[k][4 * tc + b], u = Ut[k][4 * tc + b];
        g[0][b] += n0 * v;
        g[1][b] += n1 * v;
        x[0][b] += u * m0;
        x[1][b] += u * m1;
      }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int cg = cb + 4 * tc + b;
      if (cg < nc_) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const int r = 2 * tp + a;
          if (i0 + r < n) atomicAdd(&w.Gc[sp][(size_t)cg * ld + i0 + r], (double)g[a][b]);
          if (j0 + r < n) atomicAdd(reinterpret_cast<T*>(w.Xr[sp]) + (size_t)cg * ld + j0 + r, (T)x[a][b]);
        }
      }
    }
  }
}

template <typename A>
constexpr int ext_smem_bytes() {
  return (int)sizeof(A) * (ET * ET + ET * (ET + 1) + 2 * ET * EC);
}

// G_ext[n+c', n+c] = X[c',:] . V[c,:] + g0(r_c' - r_c, tau_c' - tau_c)
// (V[c, j] = g0(r_j - r_c, tau_j - tau_c), zero on dead j).  Item = TS x TS
// tile of candidate pairs (TS = 32 for up to 32 candidates, else 64) and one
// segment of CC_SEG columns of one walker-spin; the X and V rows pass through
// shared memory CC_KC columns at a time, the next chunk's loads in flight in
// registers while the current one is multiplied.  Thread (tx, ty) of 16 x 16
// owns c' = ty + 16 a, c = tx + 16 b (a, b < TS / 16).  The segment sums are
// added into the targets (zeroed by k_cand_zero) with FP64 atomics and
// segment 0 adds the g0 term.  The products run in the storage type A of N
// and X.
constexpr int CC_SEG = 128;
constexpr int CC_KC = 32;

__device__ __forceinline__ int cc_tile(int nc_) { return nc_ <= 32 ? 32 : 64; }

template <typename A, int TS>
__device__ __forceinline__ void cand_cc_item(const Config& cfg, const WalkerDev& w, int sp, int tile, int seg,
                                             A (*Xs)[65], A (*Vs)[65]) {
  constexpr int MT = TS / 16, PR = TS * CC_KC / 256;  // outputs per thread per axis, loads per thread per operand
  const int n = w.n, nc_ = w.n_cand, ld = w.cap, par = w.parity;
  const int tiles = (nc_ + TS - 1) / TS;
  const int cpb = (tile / tiles) * TS, cb = (tile - (tile / tiles) * tiles) * TS;
  const int jlo = seg * CC_SEG, jhi = min(n, jlo + CC_SEG);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const A* X = reinterpret_cast<const A*>(w.Xr[sp]);
  const A* V = reinterpret_cast<const A*>(w.Vb[sp]);
  A xr[PR], vr[PR];
  auto fetch = [&](int j0) {
#pragma unroll
    for (int q = 0; q < PR; ++q) {
      const int e = tid + 256 * q, col = e & (CC_KC - 1), r = e / CC_KC, j = j0 + col;
      xr[q] = (cpb + r < nc_ && j < jhi) ? X[(size_t)(cpb + r) * ld + j] : (A)0;
      vr[q] = (cb + r < nc_ && j < jhi) ? V[(size_t)(cb + r) * ld + j] : (A)0;
    }
  };
  A acc[MT][MT];
#pragma unroll
  for (int a = 0; a < MT; ++a)
#pragma unroll
    for (int b = 0; b < MT; ++b) acc[a][b] = (A)0;
  if (jlo < jhi) fetch(jlo);
  for (int j0 = jlo; j0 < jhi; j0 += CC_KC) {
    __syncthreads();  // the previous chunk (or item) is done with the shared rows
#pragma unroll
    for (int q = 0; q < PR; ++q) {
      const int e = tid + 256 * q, col = e & (CC_KC - 1), r = e / CC_KC;
      Xs[col][r] = xr[q];
      Vs[col][r] = vr[q];
    }
    __syncthreads();
    if (j0 + CC_KC < jhi) fetch(j0 + CC_KC);
#pragma unroll 8
    for (int k = 0; k < CC_KC; ++k) {
      A xa[MT], vb[MT];
#pragma unroll
      for (int a = 0; a < MT; ++a) xa[a] = Xs[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < MT; ++b) vb[b] = Vs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int b = 0; b < MT; ++b) acc[a][b] += xa[a] * vb[b];
    }
  }
  const ProblemDev& pb = cfg.P[w.problem];
#pragma unroll
  for (int b = 0; b < MT; ++b) {
    const int c = cb + tx + 16 * b;
    if (c >= nc_) continue;
    const int rc = w.vsite[par][n + c];
    const double tc = w.vtau[par][n + c];
#pragma unroll
    for (int a = 0; a < MT; ++a) {
      const int cp = cpb + ty + 16 * a;
      if (cp < nc_) {
        double v = (double)acc[a][b];
        if (seg == 0)
          v += (cp == c) ? g0_diag(pb, sp, rc) : g0_pair(pb, sp, w.vsite[par][n + cp], w.vtau[par][n + cp], rc, tc);
        atomicAdd(&w.Gc[sp][(size_t)c * ld + n + cp], v);
      }
    }
  }
}

template <typename A>
__global__ void __launch_bounds__(256, sizeof(A) == 4 ? 3 : 2) k_cand_cc(Config cfg) {
  __shared__ A Xs[CC_KC][65];  // [column][c'], padded: conflict-free transposed stores
  __shared__ A Vs[CC_KC][65];  // [column][c]
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        const int ts = cc_tile(w.n_cand);
        const long long t = (w.n_cand + ts - 1) / ts;
        return (w.active && w.n_cand > 0) ? t * t * ((w.n + CC_SEG - 1) / CC_SEG + (w.n == 0)) : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int segs = (w.n + CC_SEG - 1) / CC_SEG + (w.n == 0);
        const int seg = item % segs, tile = item / segs;
        if (cc_tile(w.n_cand) == 32) cand_cc_item<A, 32>(cfg, w, s & 1, tile, seg, Xs, Vs);
        else cand_cc_item<A, 64>(cfg, w, s & 1, tile, seg, Xs, Vs);
      });
}

// ---------------------------------------------------------------------------
// Metropolis over the window (one block per walker, both spins).
// ---------------------------------------------------------------------------
template <typename T>
struct ExtView {
  const T* N;        // current N (ld)
  const T* X;        // candidate rows [c][ld] (stored like N)
  const double* Gc;  // candidate columns [c][ld]
  const int* vs;
  int n, ld;
};

template <typename T>
__device__ __forceinline__ ExtView<T> make_view(const WalkerDev& w, int sp) {
  ExtView<T> v;
  v.N = (const T*)w.N[w.parity][sp];
  v.X = reinterpret_cast<const T*>(w.Xr[sp]);
  v.Gc = w.Gc[sp];
  v.vs = w.vs[w.parity];
  v.n = w.n;
  v.ld = w.cap;
  return v;
}

// G_ext[x, y]; for an interacting existing column y, G = (N e^{V} - I) / (e^{V} - 1)
// column-wise, which follows from N = [I + G (e^V - I)] e^{-V}.
template <typename T>
__device__ __forceinline__ double g_ext(const ExtView<T>& v, const ProblemDev& pb, int sp, int x, int y) {
  if (y >= v.n) return v.Gc[(size_t)(y - v.n) * v.ld + x];
  const double nxy = ldN(x < v.n ? v.N : v.X, (size_t)(x < v.n ? x : x - v.n) * v.ld + y);
  const int sy = v.vs[y];
  const double ev = expV(pb, sp, sy);
  // (N e^V - 1) / (e^V - 1) with the reciprocal tabulated per spin (no FP64 division)
  return (nxy * ev - (x == y ? 1.0 : 0.0)) * pb.rexpVm1[sp][sy > 0 ? 1 : 0];
}

// G_ext[x, y] with the spin factors of column y given: e^{V_y} and
// 1 / (e^{V_y} - 1) (unused for a candidate column y >= n).
template <typename T>
__device__ __forceinline__ double g_ext_at(const ExtView<T>& v, int x, int y, double ev, double rv) {
  if (y >= v.n) return v.Gc[(size_t)(y - v.n) * v.ld + x];
  const double nxy = ldN(x < v.n ? v.N : v.X, (size_t)(x < v.n ? x : x - v.n) * v.ld + y);
  return (nxy * ev - (x == y ? 1.0 : 0.0)) * rv;
}

// Address of the stored entry g_ext_at reads for (x, y).
template <typename T>
__device__ __forceinline__ const void* g_ext_ptr(const ExtView<T>& v, int x, int y) {
  if (y >= v.n) return v.Gc + (size_t)(y - v.n) * v.ld + x;
  return (x < v.n) ? (const void*)(v.N + (size_t)x * v.ld + y) : (const void*)(v.X + (size_t)(x - v.n) * v.ld + y);
}

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Arithmetic M of the bordered growth of B^-1 and of the Schur complements
// (the determinant ratios): FP64 (double), or double-float pairs (hi, lo) of
// FP32 (float2), about 44 significant bits at the FP32 issue rate.  The
// update kernels of the mixed path read B^-1 as such pairs, so the FP64
// variant on the mixed path converts B^-1 into them at the end of the window.

__device__ __forceinline__ void m_set(double& r, double x) { r = x; }
__device__ __forceinline__ void m_set(float2& r, double x) { r = df_split(x); }
__device__ __forceinline__ double m_val(double a) { return a; }
__device__ __forceinline__ double m_val(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ void m_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void m_zero(float2& a) { a = make_float2(0.f, 0.f); }
// acc += a b
__device__ __forceinline__ void m_fma(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void m_fma(float2& acc, float2 a, float2 b) { df_fma(acc.x, acc.y, a.x, a.y, b.x, b.y); }
// acc += b
__device__ __forceinline__ void m_acc(double& acc, double b) { acc += b; }
__device__ __forceinline__ void m_acc(float2& acc, float2 b) { df_fma(acc.x, acc.y, b.x, b.y, 1.f, 0.f); }
// normalised value of an accumulator
__device__ __forceinline__ double m_fin(double a) { return a; }
__device__ __forceinline__ float2 m_fin(float2 a) { return df_norm(a.x, a.y); }
__device__ __forceinline__ double m_neg(double a) { return -a; }
__device__ __forceinline__ float2 m_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double m_mul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 m_mul(float2 a, float2 b) {
  float hi = 0.f, lo = 0.f;
  df_fma(hi, lo, a.x, a.y, b.x, b.y);
  return df_norm(hi, lo);
}
__device__ __forceinline__ double m_shfl_xor(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ float2 m_shfl_xor(float2 a, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
}

// Lanes per row for the l-term row sums of the Metropolis kernel (256
// threads, both spins): the largest power of two G <= 32 with 2 l G <= 256.
__device__ __forceinline__ int row_lanes(int l) {
  int G = 1;
  while (G < 32 && 4 * l * G <= 256) G <<= 1;
  return G;
}

constexpr int METRO_LIVE = 2048;  // live vertices whose rows and spins are staged in shared memory

// One block per walker, both spins.  Per proposal: (1) its target and a_t,
// (2) the border of B against the accepted set P, (3) t = B^-1 b_col, (4) the
// Schur complements d_sigma = B_tt - b_row t, (5) the decision on
// R = (K / (k + 1) or k / K) d_up d_down, and on acceptance (6) s = b_row B^-1 / d
// and (7) the bordered inverse [[B^-1 + t s, -t / d], [-s, 1 / d]].  Thread 0
// plans proposal j + 1 (step 1) together with decision j, so a rejection
// costs three block barriers and an acceptance four.
template <typename T, typename M>
__global__ void __launch_bounds__(256) k_metropolis(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = w.active;
  __syncthreads();
  if (!s_active) return;
  const ProblemDev& pb = cfg.P[w.problem];
  const int tid = threadIdx.x;
  const int n = w.n, n_live = w.n_live, len = w.win_len;
  const ExtView<T> ev[2] = {make_view<T>(w, 0), make_view<T>(w, 1)};
  // B^-1 of both spins: in shared memory when k_s <= METRO_SMEM_KS, with row
  // stride k_s | 1 (odd: the row-wise products of step 3 are free of bank
  // conflicts), copied to the global buffers at the end; else in the global
  // buffers (row stride KS_MAX).
  extern __shared__ double s_binv[];
  const bool in_smem = cfg.ks <= METRO_SMEM_KS;
  const int bst = in_smem ? (cfg.ks | 1) : KS_MAX;
  M* const Binv[2] = {in_smem ? reinterpret_cast<M*>(s_binv) : reinterpret_cast<M*>(w.Binv[0]),
                      in_smem ? reinterpret_cast<M*>(s_binv) + (size_t)cfg.ks * bst : reinterpret_cast<M*>(w.Binv[1])};

  __shared__ Proposal s_prop[KS_MAX];
  __shared__ int s_live[METRO_LIVE];  // 2 row + (s > 0) of the live vertex of each rank
  __shared__ M s_brow[2][KS_MAX], s_bcol[2][KS_MAX], s_t[2][KS_MAX], s_s[2][KS_MAX];
  __shared__ M s_rd[2];
  __shared__ double s_aP[2][KS_MAX];
  __shared__ int s_P[KS_MAX];
  __shared__ int s_Pup[KS_MAX];       // spin of a live P_p > 0
  __shared__ int s_removed[KS_MAX];   // live ranks removed in this window, ascending
  __shared__ int s_flipped[KS_MAX];   // live ranks whose auxiliary spin was flipped in this window
  __shared__ int s_flip_p[KS_MAX];    // their positions in P
  __shared__ int s_ins_p[KS_MAX];     // positions in P of the vertices inserted in this window, in order
  __shared__ int s_gone[KS_MAX];      // P entry of a vertex inserted and removed again in this window
  __shared__ int s_dupq, s_dupi, s_upq;  // duplicate update: P position, list index; P position being applied
  __shared__ double s_ev[2][2], s_rv[2][2];  // e^{V} and 1 / (e^{V} - 1): [spin][s > 0]
  __shared__ double s_anew_tab[3][2][2];      // a_t of an insertion / removal / flip: [kind][spin][s > 0]
  __shared__ double s_anew[2], s_Btt[2];
  __shared__ int s_target, s_tup, s_kind, s_stop, s_accept, s_l, s_nrem, s_nins, s_kcur, s_eval, s_rank, s_nflip;
  __shared__ double s_sign;

  const bool live_smem = n_live <= METRO_LIVE;
  for (int j = tid; j < len; j += blockDim.x) s_prop[j] = w.prop[j];
  if (live_smem)
    for (int r = tid; r < n_live; r += blockDim.x) {
      const int x = w.live_idx[r];
      s_live[r] = 2 * x + (ev[0].vs[x] > 0 ? 1 : 0);
    }
  if (tid < 4) {
    const int sp = tid >> 1, up = tid & 1;
    s_ev[sp][up] = pb.expV[sp][up];
    const double e = pb.expV[sp][up ? 0 : 1];  // e^{V(-s)}: removal e^{-V} - 1, flip e^{-2V} - 1
    s_anew_tab[0][sp][up] = pb.expV[sp][up] - 1.0;
    s_anew_tab[1][sp][up] = e - 1.0;
    s_anew_tab[2][sp][up] = e * e - 1.0;
    s_rv[sp][up] = pb.rexpVm1[sp][up];
  }
  if (tid == 0) {
    s_l = 0;
    s_nrem = 0;
    s_nins = 0;
    s_nflip = 0;
    s_stop = 0;
    s_sign = w.sign;
    s_eval = 0;
  }
  // thread 0's view of the chain state
  const uint64_t q0 = w.q;
  const int64_t forced_n = w.forced_n, log_cap = w.log_cap;
  const double K = pb.K;
  int64_t c_prop = 0, c_acc = 0, c_ties = 0, c_negl = 0;
  __syncthreads();

  // Step 1 (thread 0): target of proposal j, its spin and the new a_t.
  // Kinds: 0 insert, 1 remove, 3 flip, 2 rejected without a ratio (removal or
  // flip from the empty configuration, or a proposal the neglect rule drops).
  // A removal or flip that picks a spin already changed in this window (an
  // insertion or a flip of this window) ends the window (the abort variant;
  // the proposal is re-evaluated first in the next window), is rejected (the
  // neglect rule), or is evaluated in place (kinds 4 to 7, the update rule:
  // a rank-1 change of one column of B).
  auto plan = [&](int j) {
    const Proposal& pr = s_prop[j];
    const int kcur = n_live - s_nrem + s_nins;
    int kind = 0, target = -1, rank = -1, up = 0;
    if (pr.type == 0) {
      target = n + pr.slot;
      up = pr.s > 0 ? 1 : 0;  // the candidate's spin (its factors e^V are not needed: G_ext is tabulated)
      for (int sp = 0; sp < 2; ++sp) s_anew[sp] = s_anew_tab[0][sp][up];
    } else if (kcur == 0) {
      kind = 2;
    } else {
      const int idx = (int)scaled_index(pr.word, (uint32_t)kcur);
      const int nold = n_live - s_nrem;
      bool dup = idx >= nold;  // a spin inserted in this window
      int dupq = dup ? s_ins_p[idx - nold] : -1, dupi = idx - nold;
      if (!dup) {
        // idx-th live vertex not yet removed in this window: rank = idx + r*,
        // r* the first r with s_removed[r] - r > idx (s_removed ascending and
        // distinct, so s_removed[r] - r is non-decreasing): binary search
        int lo = 0, hi = s_nrem;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_removed[mid] - mid <= idx) lo = mid + 1;
          else hi = mid;
        }
        rank = idx + lo;
        for (int r = 0; r < s_nflip; ++r)
          if (s_flipped[r] == rank) {
            dup = true;
            dupq = s_flip_p[r];
            dupi = r;
          }
      }
      if (dup) {
        if (cfg.dup_rule == 1) {
          kind = 2;  // neglect rule: rejected
        } else if (cfg.dup_rule == 2) {
          // the spin at P position dupq changes again: kinds 4 / 5 remove / flip a
          // vertex inserted in this window, 6 / 7 remove / flip one flipped in it;
          // a' is the total change against the start of the window
          const bool ins = idx >= nold;
          kind = (ins ? 4 : 6) + (pr.type == 2 ? 1 : 0);
          target = s_P[dupq];
          up = s_Pup[dupq];
          for (int sp = 0; sp < 2; ++sp)
            s_anew[sp] = kind == 4 || kind == 7 ? 0.0 : (kind == 5 ? s_anew_tab[0][sp][up ^ 1] : s_anew_tab[1][sp][up]);
          s_dupq = dupq;
          s_dupi = dupi;
        } else {
          s_stop = 1;  // abort rule: end the window here
        }
      } else {
        kind = pr.type == 2 ? 3 : 1;
        if (live_smem) {
          const int v = s_live[rank];
          target = v >> 1;
          up = v & 1;
        } else {
          target = w.live_idx[rank];
          up = ev[0].vs[target] > 0 ? 1 : 0;
        }
        for (int sp = 0; sp < 2; ++sp) s_anew[sp] = s_anew_tab[kind == 3 ? 2 : 1][sp][up];
      }
    }
    s_kind = kind;
    s_target = target;
    s_rank = rank;
    s_kcur = kcur;
    s_tup = up;
  };
  if (tid == 0 && len > 0) plan(0);
  __syncthreads();

  for (int j = 0; j < len; ++j) {
    if (s_stop) break;
    const int l = s_l;
    if (s_kind == 2) {
      // a removal or flip from the empty configuration (ratio zero), or a
      // proposal dropped by the neglect rule: rejected
      __syncthreads();  // every thread has read s_kind and s_l
      if (tid == 0) {
        const uint64_t q = q0 + (uint64_t)j;
        if ((int64_t)q < log_cap) w.log[q] = 0;
        ++c_prop;
        c_negl += s_kcur > 0;
        s_eval = j + 1;
        if (j + 1 < len) plan(j + 1);
      }
      __syncthreads();
      continue;
    }
    if (s_kind >= 4) {
      // A spin changed earlier in this window changes again: column q of B
      // changes by u = (e_q - G_Pq)(a' - a) = c (B e_q - e_q), c = (a' - a) / a, so
      // det B'/det B = 1 + c (1 - (B^-1)_qq) and, by Sherman-Morrison,
      // B'^-1 = B^-1 - (c / rho) (e_q - B^-1 e_q) e_q^T B^-1.  Exact: the chain
      // of single-spin updates without ending the window.
      __syncthreads();  // every thread has read s_kind
      if (tid == 0) {
        const int qp = s_dupq, kind = s_kind;
        const Proposal& pr = s_prop[j];
        const uint64_t q = q0 + (uint64_t)j;
        double rho[2], coef[2];
        for (int sp = 0; sp < 2; ++sp) {
          // a = 0 only where every factor is (U = 0, e^V = 1): then a' = a, no change
          const double a = s_aP[sp][qp], c = s_anew[sp] == a ? 0.0 : (s_anew[sp] - a) / a;
          rho[sp] = 1.0 + c * (1.0 - m_val(Binv[sp][(size_t)qp * bst + qp]));
          coef[sp] = c / rho[sp];
        }
        const double R = (kind == 4 || kind == 6 ? (double)s_kcur / K : 1.0) * rho[0] * rho[1];
        int acc = 0, tie = 0;
        if (!isfinite(R)) {
          set_status(w, ST_ERR_NUMERIC);
          s_stop = 1;
        } else {
          const double absR = fabs(R);
          acc = pr.u < absR;
          tie = fabs(absR - pr.u) < cfg.tie_eps;
          if ((int64_t)q < forced_n) acc = w.forced[q] & 1;
          if (acc && R < 0.0) s_sign = -s_sign;
          if ((int64_t)q < log_cap) w.log[q] = (uint8_t)(acc | (tie << 1));
          ++c_prop;
          c_ties += tie;
          c_acc += acc;
          s_eval = j + 1;
          if (acc) {
            s_upq = qp;
            m_set(s_rd[0], coef[0]);
            m_set(s_rd[1], coef[1]);
            s_aP[0][qp] = s_anew[0];
            s_aP[1][qp] = s_anew[1];
            const int di = s_dupi;
            if (kind == 4) {  // the inserted vertex goes: later insertions move up one place
              for (int r = di; r + 1 < s_nins; ++r) s_ins_p[r] = s_ins_p[r + 1];
              s_nins--;
              s_gone[qp] = 1;
            } else if (kind == 5) {  // the inserted vertex keeps its place with the other spin
              s_Pup[qp] ^= 1;
            } else {  // kinds 6, 7: no longer a flipped vertex
              for (int r = di; r + 1 < s_nflip; ++r) {
                s_flipped[r] = s_flipped[r + 1];
                s_flip_p[r] = s_flip_p[r + 1];
              }
              s_nflip--;
              if (kind == 6) {  // removed: its rank joins the removed ranks (ascending)
                int r = s_nrem;
                while (r > 0 && s_removed[r - 1] > s_rank) {
                  s_removed[r] = s_removed[r - 1];
                  --r;
                }
                s_removed[r] = s_rank;
                s_nrem++;
              }
            }
          }
          if (j + 1 < len) plan(j + 1);
        }
        s_accept = acc;
      }
      __syncthreads();
      if (!s_accept) continue;
      {
        const int qp = s_upq;
        for (int idx = tid; idx < 2 * l; idx += blockDim.x) {
          const int sp = idx >= l ? 1 : 0, i = idx - sp * l;
          const M* B = Binv[sp];
          m_set(s_t[sp][i], -m_val(s_rd[sp]) * ((i == qp ? 1.0 : 0.0) - m_val(B[(size_t)i * bst + qp])));
          s_s[sp][i] = B[(size_t)qp * bst + i];
        }
        __syncthreads();
        for (int idx = tid; idx < 2 * l * l; idx += blockDim.x) {
          const int sp = idx >= l * l ? 1 : 0, r = idx - sp * l * l;
          const int i = r / l, jj = r - i * l;
          M* B = Binv[sp] + (size_t)i * bst + jj;
          M b = *B;
          m_fma(b, s_t[sp][i], s_s[sp][jj]);
          *B = m_fin(b);
        }
        // no barrier: as after step 7
      }
      continue;
    }
    const int t = s_target, tup = s_tup;
    // 2. border of B: row / column against P, and the new diagonal entry
    for (int idx = tid; idx < 4 * l + 2; idx += blockDim.x) {
      if (idx < 4 * l) {
        const int sp = idx / (2 * l);
        const int rem = idx - sp * 2 * l;
        const int p = rem >> 1;
        const int P = s_P[p];
        if (rem & 1) {
          const double a = s_anew[sp];  // column: B[P_p, t] = -G[P_p, t] a_t
          m_set(s_bcol[sp][p], a == 0.0 ? 0.0 : -g_ext_at(ev[sp], P, t, s_ev[sp][tup], s_rv[sp][tup]) * a);
        } else {
          const double a = s_aP[sp][p];  // row: B[t, P_p] = -G[t, P_p] a_{P_p}
          const int up = s_Pup[p];
          m_set(s_brow[sp][p], a == 0.0 ? 0.0 : -g_ext_at(ev[sp], t, P, s_ev[sp][up], s_rv[sp][up]) * a);
        }
      } else {
        const int sp = idx - 4 * l;
        const double a = s_anew[sp];
        s_Btt[sp] = (a == 0.0) ? 1.0 : 1.0 + (1.0 - g_ext_at(ev[sp], t, t, s_ev[sp][tup], s_rv[sp][tup])) * a;
      }
    }
    __syncthreads();
    // 3. t = B^-1 b_col.  Each of the 2 l rows (both spins) is summed by a
    // group of G lanes (the largest power of two with 2 l G <= 256, at most a
    // warp), so the dependent chain of a row is l / G terms long.
    const int G = row_lanes(l);
    {
      const int r = tid / G, g = tid - r * G;
      const bool ok = r < 2 * l;
      const int sp = ok ? r / l : 0, i = ok ? r - sp * l : 0;
      M acc;
      m_zero(acc);
      if (ok) {
        const M* B = Binv[sp] + (size_t)i * bst;
        for (int p = g; p < l; p += G) m_fma(acc, B[p], s_bcol[sp][p]);
      }
      for (int o = G >> 1; o > 0; o >>= 1) m_acc(acc, m_shfl_xor(acc, o));
      if (ok && g == 0) s_t[sp][i] = m_fin(acc);
    }
    __syncthreads();
    // 4. Schur complements d = B_tt - b_row . t, and 5. the decision (warp 0);
    //    thread 0 then records an acceptance and plans proposal j + 1
    if (tid < 32) {
      M a0, a1;
      m_zero(a0);
      m_zero(a1);
      for (int i = tid; i < l; i += 32) {
        m_fma(a0, s_brow[0][i], s_t[0][i]);
        m_fma(a1, s_brow[1][i], s_t[1][i]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        m_acc(a0, m_shfl_xor(a0, o));
        m_acc(a1, m_shfl_xor(a1, o));
      }
      // the Schur complements of lane 0; then the three quotients the decision
      // needs (the ratio's prefactor, 1/d0 and 1/d1) in one pass of the warp
      const double d0 = __shfl_sync(0xffffffffu, s_Btt[0] - m_val(a0), 0);
      const double d1 = __shfl_sync(0xffffffffu, s_Btt[1] - m_val(a1), 0);
      const int kcur = s_kcur;
      double num = 1.0, den = 1.0;
      if (tid == 0) {
        if (s_kind == 0) {
          num = K;
          den = (double)(kcur + 1);
        } else if (s_kind == 1) {
          num = (double)kcur;
          den = K;
        }
      } else if (tid == 1) {
        den = d0;
      } else if (tid == 2) {
        den = d1;
      }
      const double quo = num / den;
      const double rd0 = __shfl_sync(0xffffffffu, quo, 1), rd1 = __shfl_sync(0xffffffffu, quo, 2);
      if (tid == 0) {
        const Proposal& pr = s_prop[j];
        const uint64_t q = q0 + (uint64_t)j;
        const double R = quo * d0 * d1;
        int acc = 0, tie = 0;
        if (!isfinite(R)) {
          set_status(w, ST_ERR_NUMERIC);
          s_stop = 1;
        } else {
          const double absR = fabs(R);
          acc = pr.u < absR;
          tie = fabs(absR - pr.u) < cfg.tie_eps;
          if ((int64_t)q < forced_n) acc = w.forced[q] & 1;
          if (acc && R < 0.0) s_sign = -s_sign;
          if ((int64_t)q < log_cap) w.log[q] = (uint8_t)(acc | (tie << 1));
          ++c_prop;
          c_ties += tie;
          c_acc += acc;
          s_eval = j + 1;
          if (acc) {
            m_set(s_rd[0], rd0);
            m_set(s_rd[1], rd1);
            s_P[l] = t;
            s_Pup[l] = tup;
            s_gone[l] = 0;
            s_aP[0][l] = s_anew[0];
            s_aP[1][l] = s_anew[1];
            if (s_kind == 1) {
              int r = s_nrem;  // keep the removed ranks ascending
              while (r > 0 && s_removed[r - 1] > s_rank) {
                s_removed[r] = s_removed[r - 1];
                --r;
              }
              s_removed[r] = s_rank;
              s_nrem++;
            } else if (s_kind == 3) {
              s_flip_p[s_nflip] = l;
              s_flipped[s_nflip++] = s_rank;
            } else {
              s_ins_p[s_nins++] = l;
            }
            s_l = l + 1;
          }
          if (j + 1 < len) plan(j + 1);
        }
        s_accept = acc;
      }
    }
    __syncthreads();
    // The next proposal is planned: start the loads of its border entries
    // (steps 6 and 7 of an accepted proposal run meanwhile).
    if (j + 1 < len && !s_stop && s_kind != 2 && s_kind < 4) {
      const int l1 = s_l, t1 = s_target;
      for (int idx = tid; idx < 4 * l1 + 2; idx += blockDim.x) {
        int sp, x = t1, y = t1;
        if (idx < 4 * l1) {
          sp = idx / (2 * l1);
          const int rem = idx - sp * 2 * l1;
          const int P = s_P[rem >> 1];
          if (rem & 1) x = P;
          else y = P;
        } else {
          sp = idx - 4 * l1;
        }
        prefetch_l1(g_ext_ptr(ev[sp], x, y));
      }
    }
    if (!s_accept) continue;
    // 6. s = b_row B^-1 / d (column sums, G lanes per column as in step 3)
    {
      const int r = tid / G, g = tid - r * G;
      const bool ok = r < 2 * l;
      const int sp = ok ? r / l : 0, jj = ok ? r - sp * l : 0;
      M acc;
      m_zero(acc);
      if (ok)
        for (int i = g; i < l; i += G) m_fma(acc, s_brow[sp][i], Binv[sp][(size_t)i * bst + jj]);
      for (int o = G >> 1; o > 0; o >>= 1) m_acc(acc, m_shfl_xor(acc, o));
      if (ok && g == 0) s_s[sp][jj] = m_mul(m_fin(acc), s_rd[sp]);
    }
    __syncthreads();
    // 7. bordered inverse: [[B^-1 + t s, -t / d], [-s, 1 / d]] (s already / d)
    {
      const int e = (l + 1) * (l + 1);
      for (int idx = tid; idx < 2 * e; idx += blockDim.x) {
        const int sp = idx >= e ? 1 : 0, r = idx - sp * e;
        const int i = r / (l + 1), jj = r - i * (l + 1);
        M* B = Binv[sp] + (size_t)i * bst + jj;
        if (i < l && jj < l) {
          M b = *B;
          m_fma(b, s_t[sp][i], s_s[sp][jj]);
          *B = m_fin(b);
        } else if (i < l) {
          *B = m_neg(m_mul(s_t[sp][i], s_rd[sp]));
        } else if (jj < l) {
          *B = m_neg(s_s[sp][jj]);
        } else {
          *B = s_rd[sp];
        }
      }
    }
    // no barrier: the next reads of B^-1 and of s_t / s_s / s_rd follow the
    // barrier after step 2, and steps 1-2 write nothing step 7 reads
  }
  __syncthreads();

  // Epilogue: window bookkeeping and the accepted set.
  const int l = s_l, nrem = s_nrem, nins = s_nins, nflip = s_nflip;
  // B^-1 for the update kernels: FP64 on the FP64 path, FP32 pairs on the
  // mixed path (converted in place, element by element, when the growth ran
  // in FP64 in the global buffer)
  constexpr bool to_pairs = sizeof(T) == 4 && sizeof(M) == 8 && !std::is_same<M, float2>::value;
  if (in_smem || to_pairs)
    for (int sp = 0; sp < 2; ++sp)
      for (int idx = tid; idx < l * l; idx += blockDim.x) {
        const int i = idx / l, jj = idx - i * l;
        const M b = Binv[sp][(size_t)i * bst + jj];
        if (to_pairs) reinterpret_cast<float2*>(w.Binv[sp])[(size_t)i * KS_MAX + jj] = df_split(m_val(b));
        else reinterpret_cast<M*>(w.Binv[sp])[(size_t)i * KS_MAX + jj] = b;
      }
  for (int p = tid; p < l; p += blockDim.x) {
    w.P[p] = s_P[p];
    w.aP[0][p] = s_aP[0][p];
    w.aP[1][p] = s_aP[1][p];
  }
  for (int r = tid; r < nrem; r += blockDim.x) w.removed[r] = s_removed[r];
  for (int r = tid; r < nflip; r += blockDim.x) w.flipped[r] = s_flipped[r];
  if (tid == 0) {
    w.n_flipped = nflip;
    w.n_neglected += c_negl;
    w.n_prop += c_prop;
    w.n_ties += c_ties;
    w.n_accept += c_acc;
    int m = 0;
    for (int p = 0; p < l; ++p)
      if (s_P[p] >= n && !s_gone[p]) {  // an inserted candidate (not removed again)
        w.acc_slot[m] = s_P[p] - n;
        w.acc_p[m] = p;
        w.vs[w.parity][s_P[p]] = s_Pup[p] ? 1 : -1;  // its spin (a flip in the window may have changed it)
        ++m;
      }
    const int eval = s_eval;
    w.n_acc = l;
    w.n_removed = nrem;
    w.n_ins = nins;
    w.n_eval = eval;
    w.aborted = (eval < len) && w.status == ST_OK;
    w.sign = s_sign;
    if (w.status == ST_OK) {
      w.q += (uint64_t)eval;
      w.sweep_pos += eval;
      w.n_windows++;
      if (w.aborted) w.n_aborts++;
      const int64_t sweep_no = w.sweeps_done;  // the sweep this window belongs to
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
      // Batched schedule: every walker recomputes after the first window of
      // every recompute_sweeps-th sweep (the same window for all walkers).
      // (With N recomputed at every measurement the measured sweeps need no other.)
      if (cfg.recompute_sweeps > 0 && w.first_window && sweep_no > 0 && sweep_no % cfg.recompute_sweeps == 0 &&
          !(cfg.recompute_at_measure && sweep_no > cfg.warmup)) {
        w.recompute_pending = 1;
        w.windows_since_recompute = 0;
      }
      // Fresh N for every measurement: the recompute runs in the window that
      // ends the sweep, before the measurement.
      if (cfg.recompute_at_measure && w.measure_pending) {
        w.recompute_pending = 1;
        w.windows_since_recompute = 0;
      }
      // Algorithmic work per spin on the k live vertices after the window:
      // update 2 k^2 l + 2 k l^2 flop, reading and writing k^2 entries of N
      // plus the k x l factors; extension 4 k0^2 c flop and one read of N (both
      // candidate products need only that one read).
      const double b = cfg.prec == PREC_MIXED ? 4.0 : 8.0;
      const double kk = (double)(n_live - nrem + nins), ll = (double)l;
      if (l > 0) {
        w.flops += 2.0 * (2.0 * kk * kk * ll + 2.0 * kk * ll * ll);
        w.upd_bytes += 2.0 * (b * 2.0 * kk * kk + 8.0 * 2.0 * kk * ll);
      }
      const double k0 = (double)n_live, cc = (double)w.n_cand;
      if (w.n_cand > 0) {
        w.ext_flops += 2.0 * (4.0 * k0 * k0 * cc);
        w.ext_bytes += 2.0 * b * (k0 * k0);
      }
    } else {
      w.active = 0;
      w.n_acc = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// N update.  Rows of L = (G[:,P] - E_P) diag(a_P) and of L Binv are kept at
// the extended row index: existing rows 0..n-1, candidate c at n + c.  R is
// N_ext[P, 0:n).  Dead rows get L = 0 (they never matter).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool upd_active(const WalkerDev& w) { return w.active && w.n_acc > 0; }

// L' = L B^-1 is stored as FP64 (FP64 path) or as FP32 pairs (mixed path).
template <typename A>
__device__ __forceinline__ A lp_value(const double* Lp, size_t i) {
  if (sizeof(A) == 4) return (A)reinterpret_cast<const float2*>(Lp)[i].x;
  return (A)Lp[i];
}
template <typename A>
__device__ __forceinline__ double lp_pair_value(const double* Lp, size_t i) {
  if (sizeof(A) == 4) {
    const float2 v = reinterpret_cast<const float2*>(Lp)[i];
    return (double)v.x + (double)v.y;
  }
  return Lp[i];
}

// Extended row of the t-th row of the update (existing rows first).
__device__ __forceinline__ int upd_row(const WalkerDev& w, int t) { return t < w.n ? t : w.n + w.acc_slot[t - w.n]; }

// Lrow[x, p] = (G_ext[x, P_p] - delta) a_p ; grid = (row blocks, walkers*2), block 256
template <typename T>
__global__ void __launch_bounds__(256) k_upd_lrow(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        return upd_active(w) ? blocks_of((long long)(w.n + w.n_ins) * w.n_acc, 256) : 0;
      },
      [&](int s, int item) {
  const WalkerDev& w = cfg.W[s >> 1];
  const int sp = s & 1;
  const ProblemDev& pb = cfg.P[w.problem];
  const int l = w.n_acc, rows = w.n + w.n_ins;
  const ExtView<T> v = make_view<T>(w, sp);
  const int total = rows * l;
  const int idx = item * 256 + threadIdx.x;
  if (idx < total) {
    const int t = idx / l, p = idx - t * l;
    const int x = upd_row(w, t), P = w.P[p];
    const double a = w.aP[sp][p];
    double val = 0.0;
    if (a != 0.0 && !(x < w.n && v.vs[x] == 0)) val = (g_ext(v, pb, sp, x, P) - (x == P ? 1.0 : 0.0)) * a;
    if (sizeof(T) == 4) reinterpret_cast<float2*>(w.Lrow[sp])[(size_t)x * KS_MAX + p] = df_split(val);
    else w.Lrow[sp][(size_t)x * KS_MAX + p] = val;
  }
      });
}

// Lp = Lrow Binv on the same rows ; Rr[p, j] = N_ext[P_p, j] for j < n,
// stored in the arithmetic type A of the update product
// Per thread: one output (FP64 path) or four consecutive outputs of a row
// (mixed path: four independent double-float chains sharing the loads of L).
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_upd_lp_rr(Config cfg) {
  constexpr int PT = sizeof(T) == 4 ? 4 : 1;
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        if (!upd_active(w)) return 0;
        const int lq = (w.n_acc + PT - 1) / PT;
        return blocks_of((long long)(w.n + w.n_ins) * lq, 256) + blocks_of((long long)w.n_acc * w.n, 256);
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1;
        const int l = w.n_acc, n = w.n, rows = n + w.n_ins;
        const int lq = (l + PT - 1) / PT;
        const int lp_blocks = (int)blocks_of((long long)rows * lq, 256);
        if (item < lp_blocks) {
          const int idx = item * 256 + threadIdx.x;
          if (idx < rows * lq) {
            const int t = idx / lq, p = (idx - t * lq) * PT;
            const int x = upd_row(w, t);
            // FP64-grade on both paths (B^-1 carries the conditioning of the
            // window): FP64, or double-float on FP32 pairs on the mixed path
            if (sizeof(T) == 4) {
              const float2* Lr = reinterpret_cast<const float2*>(w.Lrow[sp]) + (size_t)x * KS_MAX;
              const float2* Bi = reinterpret_cast<const float2*>(w.Binv[sp]);
              float hi[PT], lo[PT];
#pragma unroll
              for (int u = 0; u < PT; ++u) hi[u] = lo[u] = 0.f;
              for (int q = 0; q < l; ++q) {
                const float2 a = Lr[q];
                const float2* brow = Bi + (size_t)q * KS_MAX + p;
#pragma unroll
                for (int u = 0; u < PT; ++u) {
                  const float2 b = brow[u];  // columns >= l of B^-1 are never read back
                  df_fma(hi[u], lo[u], a.x, a.y, b.x, b.y);
                }
              }
              float2* out = reinterpret_cast<float2*>(w.Lp[sp]) + (size_t)x * KS_MAX + p;
#pragma unroll
              for (int u = 0; u < PT; ++u)
                if (p + u < l) out[u] = df_norm(hi[u], lo[u]);
            } else {
              const double* Lr = w.Lrow[sp] + (size_t)x * KS_MAX;
              const double* Bi = w.Binv[sp];
              double acc = 0.0;
              for (int q = 0; q < l; ++q) acc += Lr[q] * Bi[(size_t)q * KS_MAX + p];
              w.Lp[sp][(size_t)x * KS_MAX + p] = acc;
            }
          }
        } else {
          const int idx = (item - lp_blocks) * 256 + threadIdx.x;
          if (idx < l * n) {
            const ExtView<T> v = make_view<T>(w, sp);
            const int p = idx / n, j = idx - p * n;
            const int P = w.P[p];
            ((A*)w.Rr[sp])[(size_t)p * w.cap + j] =
                P < n ? ldA<A>(v.N, (size_t)P * v.ld + j) : ldA<A>(v.X, (size_t)(P - n) * v.ld + j);
          }
        }
      });
}

// In place: N[i, j] += sum_p Lp[i, p] Rr[p, j] for i, j < n.
// grid = (col tiles, row tiles, walkers*2), block 256, 32x32 tile.
template <typename T, typename A>
__device__ __forceinline__ void upd_apply_tile(const Config& cfg, int wi, int sp, int tile);

template <typename T, typename A>
__global__ void __launch_bounds__(256) k_upd_apply(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        const long long t = (w.n + TT - 1) / TT;
        return upd_active(w) ? t * t : 0;
      },
      [&](int s, int item) { upd_apply_tile<T, A>(cfg, s >> 1, s & 1, item); });
}

template <typename T, typename A>
__device__ __forceinline__ void upd_apply_tile(const Config& cfg, int wi, int sp, int tile) {
  const WalkerDev& w = cfg.W[wi];
  const int n = w.n, l = w.n_acc;
  const int tiles = (n + TT - 1) / TT;
  const int ti = tile / tiles, tj = tile - ti * tiles;
  const int j0 = tj * TT, i0 = ti * TT;
  T* N = (T*)w.N[w.parity][sp];
  const A* Rr = (const A*)w.Rr[sp];
  const int ld = w.cap;
  __shared__ A Ls[TT][TT + 1];  // [i][p]
  __shared__ A Rs[TT][TT + 1];  // [p][j]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  A acc[4] = {0, 0, 0, 0};
  for (int p0 = 0; p0 < l; p0 += TT) {
    __syncthreads();
    for (int r = ty; r < TT; r += 8) {
      const int i = i0 + r, p = p0 + tx;
      Ls[r][tx] = (i < n && p < l) ? lp_value<A>(w.Lp[sp], (size_t)i * KS_MAX + p) : (A)0;
      const int pp = p0 + r, jj = j0 + tx;
      Rs[r][tx] = (pp < l && jj < n) ? Rr[(size_t)pp * ld + jj] : (A)0;
    }
    __syncthreads();
    const int pend = (l - p0) < TT ? (l - p0) : TT;
    for (int p = 0; p < pend; ++p) {
      const A r = Rs[p][tx];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] += Ls[ty + 8 * m][p] * r;
    }
  }
  const int jj = j0 + tx;
  if (jj < n) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = i0 + ty + 8 * m;
      if (i < n) {
        const size_t o = (size_t)i * ld + jj;
        stN(N, o, ldN(N, o) + (double)acc[m]);
      }
    }
  }
}

// Rows and columns of the accepted insertions, appended at n + m:
//   N[n+m, j]    = X[c_m, j] + Lp[n+c_m, :] . Rr[:, j]          (j < n)
//   N[i, n+m']   = Lp[i, p(c_m')]                                (i < n)
//   N[n+m, n+m'] = delta + Lp[n+c_m, p(c_m')]
// (R[p, n+c] is 1 only where P_p is candidate c itself.)
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_upd_border(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        if (!upd_active(w) || w.n_ins == 0) return 0;
        return blocks_of(2LL * w.n_ins * w.n + (long long)w.n_ins * w.n_ins, 256);
      },
      [&](int s, int item) {
  const WalkerDev& w = cfg.W[s >> 1];
  const int sp = s & 1;
  const int n = w.n, l = w.n_acc, ni = w.n_ins, ld = w.cap;
  T* N = (T*)w.N[w.parity][sp];
  const A* Rr = (const A*)w.Rr[sp];
  const int rows_total = ni * n, cols_total = n * ni, corner = ni * ni;
  const int total = rows_total + cols_total + corner;
  const int idx = item * 256 + threadIdx.x;
  if (idx < total) {
    if (idx < rows_total) {
      const int m = idx / n, j = idx - m * n;
      const int c = w.acc_slot[m];
      // FP64-grade on both paths: the new row X + L'R is formed with
      // cancellation (double-float on the mixed path)
      if (sizeof(A) == 4) {
        // two independent double-float chains (even and odd p), joined by an
        // error-free sum: the latency of one dependent chain of l terms halves
        const float2* L = reinterpret_cast<const float2*>(w.Lp[sp]) + (size_t)(n + c) * KS_MAX;
        float hi = reinterpret_cast<const float*>(w.Xr[sp])[(size_t)c * ld + j], lo = 0.f, hi2 = 0.f, lo2 = 0.f;
        int p = 0;
        for (; p + 1 < l; p += 2) {
          const float2 a = L[p], b = L[p + 1];
          df_fma(hi, lo, a.x, a.y, (float)Rr[(size_t)p * ld + j], 0.f);
          df_fma(hi2, lo2, b.x, b.y, (float)Rr[(size_t)(p + 1) * ld + j], 0.f);
        }
        if (p < l) {
          const float2 a = L[p];
          df_fma(hi, lo, a.x, a.y, (float)Rr[(size_t)p * ld + j], 0.f);
        }
        const float s1 = __fadd_rn(hi, hi2), bb = __fsub_rn(s1, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s1, bb)), __fsub_rn(hi2, bb));
        stN(N, (size_t)(n + m) * ld + j, (double)__fadd_rn(s1, __fadd_rn(__fadd_rn(lo, lo2), err)));
      } else {
        const double* L = w.Lp[sp] + (size_t)(n + c) * KS_MAX;
        double acc = w.Xr[sp][(size_t)c * ld + j];
        for (int p = 0; p < l; ++p) acc += L[p] * (double)Rr[(size_t)p * ld + j];
        stN(N, (size_t)(n + m) * ld + j, acc);
      }
    } else if (idx < rows_total + cols_total) {
      const int t = idx - rows_total;
      const int i = t / ni, m = t - i * ni;
      stN(N, (size_t)i * ld + n + m, (double)lp_value<A>(w.Lp[sp], (size_t)i * KS_MAX + w.acc_p[m]));
    } else {
      const int t = idx - rows_total - cols_total;
      const int m = t / ni, m2 = t - m * ni;
      const double v = (m == m2 ? 1.0 : 0.0) + lp_pair_value<A>(w.Lp[sp], (size_t)(n + w.acc_slot[m]) * KS_MAX + w.acc_p[m2]);
      stN(N, (size_t)(n + m) * ld + n + m2, v);
    }
  }
      });
}

// Vertex list after the window: removed vertices dead, insertions appended,
// live-row index rebuilt, compaction scheduled.  grid = walkers.
__global__ void __launch_bounds__(256) k_window_end(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  if (!w.active) return;
  const int par = w.parity, n = w.n, nrem = w.n_removed, ni = w.n_ins, nl = w.n_live;
  if (w.n_acc > 0) {
    for (int r = threadIdx.x; r < nrem; r += blockDim.x) w.vs[par][w.live_idx[w.removed[r]]] = 0;
    for (int r = threadIdx.x; r < w.n_flipped; r += blockDim.x) {
      const int x = w.live_idx[w.flipped[r]];
      w.vs[par][x] = -w.vs[par][x];
    }
    // new live list: surviving ranks in order, then the appended rows
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
      int below = 0, gone = 0;
      for (int r = 0; r < nrem; ++r) {
        below += (w.removed[r] < i);
        gone |= (w.removed[r] == i);
      }
      if (!gone) w.surv_tmp[i - below] = w.live_idx[i];
    }
    __syncthreads();
    const int keep = nl - nrem;
    for (int i = threadIdx.x; i < keep; i += blockDim.x) w.live_idx[i] = w.surv_tmp[i];
    for (int m = threadIdx.x; m < ni; m += blockDim.x) w.live_idx[keep + m] = n + m;
    if (threadIdx.x == 0) {
      // slot c_m >= m and ascending in m: moving in increasing m never
      // overwrites a candidate that is still to be moved
      for (int m = 0; m < ni; ++m) {
        const int src = n + w.acc_slot[m], dst = n + m;
        w.vsite[par][dst] = w.vsite[par][src];
        w.vtau[par][dst] = w.vtau[par][src];
        w.vs[par][dst] = w.vs[par][src];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.n = n + ni;
    w.n_live = nl - nrem + ni;
    w.n_dead += nrem;
    const int thr = w.n / 8 > 16 ? w.n / 8 : 16;
    w.compact_pending = w.n_dead > 0 && (w.n_dead >= thr || w.n + cfg.ks > w.cap || w.recompute_pending);
  }
}

// Compaction: live rows / columns into the other buffer.
// grid = (col tiles, row tiles, walkers*2), block 256.
// Persistent grid over (walker-spin, 32 x 32 tile of the compacted matrix).
template <typename T>
__global__ void __launch_bounds__(256) k_compact_N(Config cfg) {
  for_each_item(
      2 * cfg.n_walkers,
      [&](int s) -> long long {
        const WalkerDev& w = cfg.W[s >> 1];
        const long long t = (w.n_live + TT - 1) / TT;
        return (w.active && w.compact_pending) ? t * t : 0;
      },
      [&](int s, int item) {
        const WalkerDev& w = cfg.W[s >> 1];
        const int sp = s & 1, k = w.n_live, ld = w.cap;
        const int tiles = (k + TT - 1) / TT;
        const int ti = item / tiles, tj = item - ti * tiles;
        const int j = tj * TT + (threadIdx.x & 31);
        const T* N = (const T*)w.N[w.parity][sp];
        T* Nn = (T*)w.N[w.parity ^ 1][sp];
        if (j < k) {
          const int cj = w.live_idx[j];
          for (int i = ti * TT + (threadIdx.x >> 5); i < k && i < (ti + 1) * TT; i += 8)
            Nn[(size_t)i * ld + j] = N[(size_t)w.live_idx[i] * ld + cj];
        }
      });
}

__global__ void __launch_bounds__(256) k_compact_end(Config cfg) {
  WalkerDev& w = cfg.W[blockIdx.x];
  if (!w.active || !w.compact_pending) return;
  const int par = w.parity, k = w.n_live;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const int x = w.live_idx[i];
    w.vsite[par ^ 1][i] = w.vsite[par][x];
    w.vtau[par ^ 1][i] = w.vtau[par][x];
    w.vs[par ^ 1][i] = w.vs[par][x];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) w.live_idx[i] = i;
  if (threadIdx.x == 0) {
    w.parity = par ^ 1;
    w.n = k;
    w.n_dead = 0;
    w.compact_pending = 0;
  }
}

// Pooled schedule (one block over all walkers): the summed sweep count and
// whether the target is still ahead; returns the go flag to every thread.
__device__ int pool_refresh(const Config& cfg) {
  __shared__ unsigned long long s_sum;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    s_sum = 0ull;
    s_ok = 0;
  }
  __syncthreads();
  unsigned long long sum = 0ull;
  int ok = 0;
  for (int i = threadIdx.x; i < cfg.n_walkers; i += blockDim.x) {
    const WalkerDev& w = cfg.W[i];
    sum += (unsigned long long)w.sweeps_done;
    ok |= w.status == ST_OK ? 1 : 0;
  }
  atomicAdd(&s_sum, sum);
  if (ok) atomicOr(&s_ok, 1);
  __syncthreads();
  const int go = (s_ok && (int64_t)s_sum < cfg.pool->target) ? 1 : 0;
  if (threadIdx.x == 0) {
    cfg.pool->sum = (int64_t)s_sum;
    cfg.pool->go = go;
  }
  return go;
}

__global__ void k_pool_target(Config cfg, int64_t n_sweeps) {
  if (threadIdx.x == 0) cfg.pool->target = INT64_MAX;
  __syncthreads();
  pool_refresh(cfg);  // the current sum
  __syncthreads();
  if (threadIdx.x == 0) {
    cfg.pool->target = cfg.pool->sum + n_sweeps * (int64_t)cfg.n_walkers;
    cfg.pool->go = (cfg.pool->go && n_sweeps > 0) ? 1 : 0;
  }
}

__global__ void k_count_active(Config cfg) {
  if (cfg.pooled) {
    const int go = pool_refresh(cfg);
    if (threadIdx.x == 0) *cfg.active_count = go;
    return;
  }
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
  if (i < cfg.n_walkers) {
    cfg.W[i].sweeps_base = cfg.W[i].sweeps_done;
    cfg.W[i].sweeps_target = cfg.W[i].sweeps_done + n_sweeps;
  }
}

// Loop control of the device-side window loop (body of a conditional WHILE
// graph node): continue while any walker still has sweeps to do (lockstep)
// or the pooled sweep target is still ahead (pooled), and stop
// with a timeout flag after max_iters windows (every window advances each
// active walker by at least one proposal, so the host's bound is never
// reached unless something is wrong).
__global__ void k_loop_control(Config cfg, cudaGraphConditionalHandle handle, LoopState* ls) {
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  if (cfg.pooled) {
    const int go = pool_refresh(cfg);
    if (threadIdx.x == 0) s_cnt = go;
  } else {
    for (int i = threadIdx.x; i < cfg.n_walkers; i += blockDim.x) {
      const WalkerDev& w = cfg.W[i];
      if (w.status == ST_OK && w.sweeps_done < w.sweeps_target) atomicAdd(&s_cnt, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ls->iters++;
    ls->total_iters++;
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
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
int device_sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && cache[dev] > 0) return cache[dev];
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  if (dev < 64) cache[dev] = sms;
  return sms;
}

int sm_grid(long long items, int per_sm) {
  const long long total = (long long)per_sm * device_sm_count();
  return (int)(items < 1 ? 1 : (items < total ? items : total));
}

int persist_grid(const void* fn, long long items, int block, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;  // resident blocks on the device
  int total = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(fn);
    if (it != cache.end()) {
      total = it->second;
    } else {
      int dev = 0, sms = 0, per_sm = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem) != cudaSuccess)
        per_sm = 0;
      total = (per_sm > 0 && sms > 0) ? per_sm * sms : 4 * device_sm_count();
      cache.emplace(fn, total);
    }
  }
  return (int)(items < 1 ? 1 : (items < total ? items : total));
}

// Grid of a persistent kernel: four blocks per SM, at most the largest
// possible number of work items.
static int grid_for(long long items) { return sm_grid(items, 4); }

template <typename T, typename A>
static int launch_group_t(int group, const Config& cfg, int max_cap, cudaStream_t st) {
  const int W = cfg.n_walkers;
  const long long S = 2LL * W;  // walker-spin pairs
  const long long t64 = (max_cap + ET - 1) / ET, t32 = (max_cap + TT - 1) / TT;
  const long long kc = blocks_of((long long)cfg.ks * max_cap, 256);
  switch (group) {
    case GROUP_PROPOSE:
      k_begin<<<W, 128, 0, st>>>(cfg);
      return 1;
    case GROUP_EXTEND:
      k_cand_zero<<<persist_grid((const void*)k_cand_zero, S * kc, 256), 256, 0, st>>>(cfg);
      if (cfg.prec == PREC_MIXED) {
        int k = launch_ext_mixed(cfg, max_cap, st);
        k_cand_cc<A><<<persist_grid((const void*)k_cand_cc<A>, S * 16, 256), 256, 0, st>>>(cfg);
        return 2 + k;
      }
      k_cand_ext<T, A><<<grid_for(S * t64 * t64), 256, ext_smem_bytes<A>(), st>>>(cfg);
      k_cand_cc<A><<<grid_for(S * 16), 256, 0, st>>>(cfg);
      return 3;
    case GROUP_METROPOLIS: {
      const int sm = cfg.ks <= METRO_SMEM_KS ? (int)sizeof(double) * 2 * cfg.ks * (cfg.ks | 1) : 0;
      if (sizeof(T) == 8 || cfg.gamma_fp64) k_metropolis<T, double><<<W, 256, sm, st>>>(cfg);
      else k_metropolis<T, float2><<<W, 256, sm, st>>>(cfg);
      return 1;
    }
    case GROUP_UPDATE_PRE:
      if (cfg.prec == PREC_MIXED && cfg.upd_kernel == UPD_TCGEN05) {
        launch_upd_factors(cfg, max_cap, st);
        return 1;
      }
      k_upd_lrow<T><<<persist_grid((const void*)k_upd_lrow<T>, S * kc, 256), 256, 0, st>>>(cfg);
      k_upd_lp_rr<T, A><<<persist_grid((const void*)k_upd_lp_rr<T, A>, 2 * S * kc, 256), 256, 0, st>>>(cfg);
      return 2;
    case GROUP_UPDATE:
      if (cfg.prec == PREC_MIXED && cfg.upd_kernel == UPD_TCGEN05)
        launch_upd_tc(cfg, st);
      else
        k_upd_apply<T, A><<<grid_for(S * t32 * t32), 256, 0, st>>>(cfg);
      return 1;
    case GROUP_UPDATE_POST:
      k_upd_border<T, A><<<persist_grid((const void*)k_upd_border<T, A>, 2 * S * kc, 256), 256, 0, st>>>(cfg);
      k_window_end<<<W, 256, 0, st>>>(cfg);
      k_compact_N<T><<<persist_grid((const void*)k_compact_N<T>, S * t32 * t32, 256), 256, 0, st>>>(cfg);
      k_compact_end<<<W, 256, 0, st>>>(cfg);
      return 4;
    default:
      return 0;
  }
  (void)max_cap;
}

cudaError_t setup_window_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_cand_ext<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ext_smem_bytes<double>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cand_ext<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ext_smem_bytes<float>());
  const int msm = (int)sizeof(double) * 2 * METRO_SMEM_KS * (METRO_SMEM_KS | 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_metropolis<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, msm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_metropolis<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, msm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_metropolis<float, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, msm);
  return e;
}

int launch_window_group(int group, const Config& cfg, int max_cap, cudaStream_t st) {
  return cfg.prec == PREC_MIXED ? launch_group_t<float, float>(group, cfg, max_cap, st)
                                : launch_group_t<double, double>(group, cfg, max_cap, st);
}

void launch_count_active(const Config& cfg, cudaStream_t st) { k_count_active<<<1, 256, 0, st>>>(cfg); }

void launch_add_target(const Config& cfg, int64_t n_sweeps, cudaStream_t st) {
  if (cfg.pooled) k_pool_target<<<1, 256, 0, st>>>(cfg, n_sweeps);
  else k_add_target<<<(cfg.n_walkers + 127) / 128, 128, 0, st>>>(cfg, n_sweeps);
}

void launch_loop_control(const Config& cfg, cudaGraphConditionalHandle handle, LoopState* ls, cudaStream_t st) {
  k_loop_control<<<1, 256, 0, st>>>(cfg, handle, ls);
}

void launch_loop_reset(LoopState* ls, int64_t max_iters, cudaStream_t st) { k_loop_reset<<<1, 1, 0, st>>>(ls, max_iters); }

}  // namespace dca
