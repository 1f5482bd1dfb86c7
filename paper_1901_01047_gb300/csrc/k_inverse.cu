// k_inverse.cu -- FP64 in-place Gauss-Jordan inverse, one thread-block
// cluster per matrix (the from-scratch N of the initial build and of the
// periodic recompute, Eq. Zk: N = [e^V - g0 (e^V - 1)]^-1).
//
// A cluster of GJ_CTAS blocks shares one n x n matrix in global memory.  Rows
// are owned cyclically (row r by block r % GJ_CTAS).  Per column c:
//   1. every block finds the largest |A[r][c]|, r >= c, among its rows and
//      posts it in shared memory; cluster barrier; every block reads all
//      posts through distributed shared memory and takes the same pivot p;
//   2. rows c and p are swapped and row c is scaled by 1/d (column c of the
//      working matrix becomes column c of the inverse: A[c][c] := 1/d), each
//      block doing a slice of the columns; cluster barrier;
//   3. every block eliminates column c from its own rows (one warp per row).
// The row interchanges are undone at the end as column interchanges in
// reverse order.  The sign of det A comes from the pivots.
#include <cooperative_groups.h>

#include <cstdint>

#include "device_util.cuh"
#include "kernels.h"
#include "state.h"

namespace cg = cooperative_groups;

namespace dca {

constexpr int GJ_CTAS = 8;
constexpr int GJ_THREADS = 1024;

struct GjPost {
  double val;    // signed pivot candidate
  double mag;    // |val|, -1 if the block has no row >= c
  int idx;
  int pad;
};

__device__ __forceinline__ bool gj_better(double m1, int i1, double m2, int i2) {
  return m1 > m2 || (m1 == m2 && i1 < i2);
}

__device__ void gj_matrix(const Config& cfg, int mode, int mat, int* sgn_out, cg::cluster_group& cluster);

__device__ __forceinline__ bool gj_wants(const Config& cfg, int mode, int mat) {
  const WalkerDev& w = cfg.W[mat >> 1];
  if (mode == 0) return true;
  if (mode == 2) return w.rebuild_pending && w.status == ST_OK;
  return w.active && w.recompute_pending && w.status == ST_OK;
}

// mode 0: initial build / standalone; mode 1: periodic recompute (into the
// other buffer); mode 2: rebuild after a change of the bare propagator.
// Persistent grid of clusters fed by a work queue: the rank-0 block of a
// cluster takes the next matrix (walker * 2 + spin) from cfg.gj_next (reset to
// 0 by k_build_A before every launch), so clusters that drew small matrices
// take more of them.  Dynamic shared memory: one int per row (pivot rows).
__global__ void __cluster_dims__(GJ_CTAS, 1, 1) __launch_bounds__(GJ_THREADS)
    k_gj_cluster(Config cfg, int mode, int* sgn_out) {
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ int s_next;
  // Nothing to do in most windows: every block sees the same records, so the
  // decision is uniform over the cluster.
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int m = threadIdx.x; m < 2 * cfg.n_walkers && !s_any; m += blockDim.x)
    if (gj_wants(cfg, mode, m)) s_any = 1;
  __syncthreads();
  if (!s_any) return;
  const int rank = (int)cluster.block_rank();
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_next = atomicAdd(cfg.gj_next, 1);
    cluster.sync();
    const int mat = *cluster.map_shared_rank(&s_next, 0);
    cluster.sync();  // every block has read s_next before it changes
    if (mat >= 2 * cfg.n_walkers) break;
    if (!gj_wants(cfg, mode, mat)) continue;
    gj_matrix(cfg, mode, mat, sgn_out, cluster);
    cluster.sync();  // the next matrix reuses the shared posts and pivots
  }
}

__device__ void gj_matrix(const Config& cfg, int mode, int mat, int* sgn_out, cg::cluster_group& cluster) {
  const int rank = (int)cluster.block_rank();
  const int wi = mat >> 1, sp = mat & 1;
  WalkerDev& w = cfg.W[wi];
  const int n = w.n, ld = w.cap;
  double* A = (cfg.prec == PREC_MIXED) ? w.Ascr[sp] : (double*)w.N[mode == 1 ? w.parity ^ 1 : w.parity][sp];
  extern __shared__ int s_piv[];
  __shared__ GjPost s_post;
  __shared__ GjPost s_warp[GJ_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int sign = 1;
  bool bad = false;
  for (int c = 0; c < n; ++c) {
    // 1. pivot candidates of this block's rows
    double bm = -1.0, bv = 0.0;
    int bi = 0x7fffffff;
    for (int r = c + ((rank - c % GJ_CTAS + GJ_CTAS) % GJ_CTAS) + GJ_CTAS * tid; r < n; r += GJ_CTAS * GJ_THREADS) {
      const double v = A[(size_t)r * ld + c];
      const double m = fabs(v);
      if (gj_better(m, r, bm, bi)) {
        bm = m;
        bv = v;
        bi = r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double om = __shfl_xor_sync(0xffffffffu, bm, o);
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (gj_better(om, oi, bm, bi)) {
        bm = om;
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) s_warp[warp] = GjPost{bv, bm, bi, 0};
    __syncthreads();
    if (tid == 0) {
      GjPost b = s_warp[0];
      for (int k = 1; k < GJ_THREADS / 32; ++k)
        if (gj_better(s_warp[k].mag, s_warp[k].idx, b.mag, b.idx)) b = s_warp[k];
      s_post = b;
    }
    cluster.sync();
    // every block picks the same pivot from all posts
    GjPost best{0.0, -1.0, 0x7fffffff, 0};
    for (int k = 0; k < GJ_CTAS; ++k) {
      const GjPost* q = cluster.map_shared_rank(&s_post, k);
      const GjPost pk = *q;
      if (gj_better(pk.mag, pk.idx, best.mag, best.idx)) best = pk;
    }
    if (!(best.mag > 0.0)) {
      bad = true;
      break;  // every block reaches the same decision
    }
    const int p = best.idx;
    const double d = best.val;
    if (tid == 0) s_piv[c] = p;
    if (p != c) sign = -sign;
    if (d < 0.0) sign = -sign;
    const double rd = 1.0 / d;
    // 2. swap rows c and p, scale the new row c (column slice per block)
    const int j0 = (int)(((long long)n * rank) / GJ_CTAS), j1 = (int)(((long long)n * (rank + 1)) / GJ_CTAS);
    for (int j = j0 + tid; j < j1; j += GJ_THREADS) {
      const double rowc = A[(size_t)c * ld + j];
      const double rowp = A[(size_t)p * ld + j];
      if (p != c) A[(size_t)p * ld + j] = rowc;
      A[(size_t)c * ld + j] = (j == c) ? rd : rowp * rd;
    }
    // the posts are re-read by other blocks above: the barrier also protects s_post
    cluster.sync();
    // 3. eliminate column c from this block's rows, one warp per row
    const double* Ac = A + (size_t)c * ld;
    for (int r = rank + GJ_CTAS * warp; r < n; r += GJ_CTAS * (GJ_THREADS / 32)) {
      if (r == c) continue;
      double* Ar = A + (size_t)r * ld;
      double f = 0.0;
      if (lane == 0) f = Ar[c];
      f = __shfl_sync(0xffffffffu, f, 0);
      if (f == 0.0) continue;
      for (int j = lane; j < n; j += 32) {
        const double a = (j == c) ? 0.0 : Ar[j];
        Ar[j] = a - f * Ac[j];
      }
    }
    __syncthreads();
  }
  if (bad) {
    cluster.sync();  // no block leaves while another may still read its post
    if (rank == 0 && tid == 0) {
      set_status(w, ST_ERR_NUMERIC);
      sgn_out[mat] = 0;
    }
    return;
  }
  // The other blocks must finish their eliminations before columns move.
  cluster.sync();
  // undo the row interchanges as column interchanges, last first (own rows)
  for (int c = n - 1; c >= 0; --c) {
    const int p = s_piv[c];
    if (p == c) continue;
    for (int r = rank + GJ_CTAS * tid; r < n; r += GJ_CTAS * GJ_THREADS) {
      double* Ar = A + (size_t)r * ld;
      const double t = Ar[c];
      Ar[c] = Ar[p];
      Ar[p] = t;
    }
  }
  if (rank == 0 && tid == 0) sgn_out[mat] = sign;
}

int gj_smem_bytes(int max_n) { return (int)sizeof(int) * (max_n > 0 ? max_n : 1); }

void launch_gj(const Config& cfg, int mode, int max_n, int* d_sgn, cudaStream_t st) {
  const int smem = gj_smem_bytes(max_n);
  static int configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaFuncSetAttribute(k_gj_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = smem;
  }
  // one cluster of GJ_CTAS blocks per GJ_CTAS SMs, at most one per matrix
  const int mats = 2 * cfg.n_walkers, fit = device_sm_count() / GJ_CTAS > 0 ? device_sm_count() / GJ_CTAS : 1;
  const int clusters = mats < fit ? mats : fit;
  k_gj_cluster<<<GJ_CTAS * clusters, GJ_THREADS, smem, st>>>(cfg, mode, d_sgn);
}

}  // namespace dca
