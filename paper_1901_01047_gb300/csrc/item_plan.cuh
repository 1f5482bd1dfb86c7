// item_plan.cuh -- the work list of a persistent warp-specialised kernel.
//
// A persistent CTA takes the global items blockIdx.x, blockIdx.x + gridDim.x,
// ... of a list made of sets (walker-spins) with count(s) items each.  All
// threads of the CTA plan that list once, before the roles split: the counts
// are evaluated in parallel and scanned in shared memory, chunk by chunk, and
// the CTA's own items are written in order as (set, sub-item) pairs.  Every
// role (TMA producer, MMA issuer, converters) then walks the same list.  A
// serial walk over the walker records, one dependent global load per set and
// role, is left only for the items past the list's capacity.
#pragma once

#include <cstdint>

namespace dca {

// sub-item field of a list entry (items of a set < 65536); the set index takes
// the 15 bits above it, so a list serves fewer than 32768 sets (walker-spins)
constexpr int PLAN_SUB_BITS = 16;

// ITEMS listed items per CTA; CHUNK sets counted and scanned per pass.
template <int ITEMS, int CHUNK>
struct ItemPlanT {
  static constexpr int kItems = ITEMS, kChunk = CHUNK;
  int pre[CHUNK + 1];  // exclusive prefix of the chunk's counts
  int warp_tot[32];
  int item[ITEMS];     // set << PLAN_SUB_BITS | sub-item
  int n;               // items of this CTA (may exceed ITEMS)
};
using ItemPlan = ItemPlanT<2048, 512>;
using ItemPlanSmall = ItemPlanT<192, 128>;  // for kernels with little shared memory left

// Called by every thread of the CTA (blockDim.x a multiple of 32); ends with a
// barrier, after which P.n and P.item are valid.
template <typename Plan, typename Count>
__device__ void plan_items(Plan& P, int nsets, Count count) {
  constexpr int PLAN_CHUNK = Plan::kChunk, PLAN_ITEMS = Plan::kItems;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const long long G = gridDim.x;
  long long base = 0;  // items of the earlier chunks
  int mine = 0;        // items of this CTA in the earlier chunks
  for (int s0 = 0; s0 < nsets; s0 += PLAN_CHUNK) {
    const int m = min(PLAN_CHUNK, nsets - s0);
    __syncthreads();  // readers of the previous chunk are done
    const int per = (m + nthr - 1) / nthr;
    const int k0 = min(m, tid * per), k1 = min(m, k0 + per);
    int own = 0;
    for (int k = k0; k < k1; ++k) {
      const int c = (int)count(s0 + k);
      P.pre[k] = c;
      own += c;
    }
    int incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) P.warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int v = lane < nw ? P.warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (lane < nw) P.warp_tot[lane] = v;
    }
    __syncthreads();
    int run = incl - own + (warp > 0 ? P.warp_tot[warp - 1] : 0);
    for (int k = k0; k < k1; ++k) {
      const int c = P.pre[k];
      P.pre[k] = run;
      run += c;
    }
    const int total = P.warp_tot[nw - 1];
    if (tid == 0) P.pre[m] = total;
    __syncthreads();
    // this CTA's items of the chunk: local index f, f + G, ... < total
    const long long f = ((((long long)blockIdx.x - base) % G) + G) % G;
    const int cnt = f < total ? (int)((total - 1 - f) / G + 1) : 0;
    for (int k = tid; k < cnt; k += nthr) {
      const int at = mine + k;
      if (at >= PLAN_ITEMS) break;
      const int local = (int)(f + (long long)k * G);
      int lo = 0, hi = m;  // pre[lo] <= local < pre[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P.pre[mid] <= local) lo = mid;
        else hi = mid;
      }
      P.item[at] = ((s0 + lo) << PLAN_SUB_BITS) | (local - P.pre[lo]);
    }
    mine += cnt;
    base += total;
  }
  if (tid == 0) P.n = mine;
  __syncthreads();
}

// One role's walk over the CTA's items (the same sequence in every role).
template <typename Plan>
struct PlanWalk {
  static constexpr int PLAN_ITEMS = Plan::kItems;
  const Plan* P = nullptr;
  int k = 0;                           // next list entry
  int s = -1;                          // serial walk past the list
  long long base = 0, cnt = 0, item = 0;
  __device__ void start(const Plan& p) {
    P = &p;
    k = 0;
    s = -1;
  }
  template <typename Count>
  __device__ bool next(int nsets, Count count, int& set, int& sub) {
    const int n = P->n;
    if (k < n && k < PLAN_ITEMS) {
      const int v = P->item[k++];
      set = v >> PLAN_SUB_BITS;
      sub = v & ((1 << PLAN_SUB_BITS) - 1);
      return true;
    }
    if (k >= n || nsets <= 0) return false;
    if (s < 0) {  // items past the list: global item blockIdx.x + PLAN_ITEMS * gridDim.x onwards
      s = 0;
      base = 0;
      cnt = count(0);
      item = (long long)blockIdx.x + (long long)PLAN_ITEMS * gridDim.x;
    }
    while (item >= base + cnt) {
      base += cnt;
      if (++s >= nsets) return false;
      cnt = count(s);
    }
    set = s;
    sub = (int)(item - base);
    item += gridDim.x;
    return true;
  }
};

}  // namespace dca
