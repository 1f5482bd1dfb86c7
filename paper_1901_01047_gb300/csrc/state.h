// state.h -- device-side data layout of the CT-AUX walker library.
//
// One WalkerDev record per walker lives in device memory; it holds the
// walker's scalars and pointers into the library-owned pools.  Every kernel
// reads the record to find out how much work this window has (the order n
// changes every submatrix update), so the host launches a fixed kernel
// sequence per window without reading anything back.
//
// Notation (DCA++ paper Sec. 2.3 and the submatrix-update paragraph there):
//   vertex p = (site r_p, time tau_p, auxiliary spin s_p);
//   V_p^sigma = sigma gamma s_p if p interacts, 0 otherwise (sigma = +1 up, -1 down);
//   g0 = -G0;  N_sigma^-1 = e^{V} - g0 (e^{V} - 1);  G = N g0.
// A window ("submatrix update") evaluates up to k_s proposals against the
// N of the window start: insertion candidates are appended as
// non-interacting rows n, n+1, ... of the extended matrices, accepted
// flips are collected in the ordered set P with a_p = e^{V'_p - V_p} - 1,
// and B_P = I + (I - G_PP) diag(a_P) is grown by bordering (its inverse
// Binv).  At the end N <- N + (G[:,P] - E_P) diag(a_P) Binv N[P,:] on the
// extended configuration: in place on the existing rows / columns, plus the
// rows and columns of the accepted insertions appended at n, n+1, ...
//
// Dead rows.  A removed vertex becomes non-interacting (V = 0, stored s = 0)
// and keeps its row and column until a compaction pass.  Its column of N is
// e_y, its row never enters a ratio, an update factor or a measurement, so the
// live rows (in order) are exactly the configuration of a single-spin chain.
// Compaction gathers the live rows / columns into the other buffer when dead
// rows exceed a fraction of n, when n + k_s would exceed the capacity, and
// before every recompute.
#pragma once
#include <cstdint>

namespace dca {

constexpr int KS_MAX = 128;     // largest submatrix size (App. B default is 128)

enum : int32_t {
  ST_OK = 0,
  ST_ERR_TIMEOUT = -4,  // a bounded wait inside a kernel gave up
  ST_ERR_NUMERIC = -5,
  ST_ERR_CAPACITY = -7,
};

enum : int32_t {
  PREC_FP64 = 0,   // N stored and updated in FP64
  PREC_MIXED = 1,  // N stored in FP32, products in FP32; ratios, B^-1, recompute in FP64
};

struct ProblemDev {
  int32_t nc, n_tau;
  double beta, K, gamma, tau_scale;   // tau_scale = n_tau / beta
  double expV[2][2];                  // e^{sigma gamma s}: [spin][s > 0]
  double rexpVm1[2][2];               // 1 / (e^{sigma gamma s} - 1) (inf when gamma = 0; never used then)
  const int32_t* site_sub;            // [nc*nc]
  const int32_t* site_add;            // [nc*nc]: site_add[y*nc + d] = x with site_sub[x*nc + y] = d
  const double* g0;                   // [2][nc][n_tau+1], g0 = -G0
  const float* g0f;                   // FP32 copy of g0 (mixed-precision interpolation)
  // Measurement grid tau_a = (a + 1/2) beta / n_tau_meas on the g0 grid when
  // n_tau = q n_tau_meas with q even (mixed path; else meas_q = 0): the grid
  // offset of tau_a - tau_i is q a + c_i, so each vertex reads one phase
  // p = c_i mod q of the table.  g0m[sp][p][d][m] = g0f[sp][d][q m + p],
  // m = 0 .. n_tau_meas (0 past the table end).
  const float* g0m;
  int32_t meas_q;
  // Two-particle measurement: K_a . r_s / 2 pi modulo 1 as 56-bit fractions
  // [nc][nc], and the index of Q - K for every K [nc] (null when off).
  const unsigned long long* kr56;
  const int32_t* k_dn;
};

struct Proposal {
  double tau;      // insert: new vertex time
  double u;        // Metropolis uniform
  int32_t type;    // 0 insert, 1 remove, 2 auxiliary-spin flip
  int32_t s;       // insert: +1 / -1
  int32_t site;    // insert: site
  uint32_t word;   // remove / flip: index word, index = floor(word * k / 2^32)
  int32_t slot;    // insert: candidate slot c, extended row n + c
  int32_t pad;
};

struct WalkerDev {
  // ---- configuration and chain state ----
  int32_t n;                 // rows of N (live + dead)
  int32_t n_live;            // interacting vertices: the expansion order k
  int32_t n_dead;            // dead rows awaiting compaction
  int32_t compact_pending;
  int32_t cap;               // matrix capacity (rows / leading dimension)
  int32_t problem;           // index into the problem table
  int32_t status;            // ST_OK or an error code; a walker in error stops
  int32_t parity;            // which of the two buffers is current
  int32_t windows_since_recompute;
  uint32_t key0, key1;       // Philox key
  uint64_t q;                // next proposal number
  int64_t sweeps_done, sweeps_target, sweep_pos, sweep_len_cur, sweep_len, warm_k_sum;
  int64_t sweeps_base;       // sweeps_done when the current lockstep call began
  double sign;

  // ---- current window ----
  int32_t active;            // this window does work
  int32_t win_len;           // proposals generated
  int32_t n_cand;            // insertion candidates generated
  int32_t n_acc;             // accepted flips l
  int32_t n_removed;         // accepted removals (existing rows)
  int32_t n_eval;            // proposals evaluated (win_len unless aborted)
  int32_t aborted;
  int32_t n_ins;             // accepted insertions (appended rows)
  int32_t measure_pending;
  int32_t recompute_pending;
  int32_t rebuild_pending;   // the bare propagator changed: N is rebuilt from scratch (Gauss-Jordan) before the next window
  int32_t first_window;      // this window starts a sweep

  // ---- counters ----
  int64_t n_prop, n_accept, n_ties, n_aborts, n_windows, n_meas, n_recomputes;
  double sign_sum, k_sum, max_drift;
  unsigned long long drift_bits[2];  // max |N_old - N_new| and max |N_new| of a recompute (bits of doubles >= 0)
  // algorithmic work (both spins): N update flop / bytes, candidate extension flop / bytes
  double flops, upd_bytes, ext_flops, ext_bytes, rec_flops;

  // ---- decision log / replay ----
  int64_t log_cap, forced_n;
  uint8_t* log;              // [log_cap]
  const uint8_t* forced;     // [forced_n]

  // ---- pools (device pointers) ----
  int32_t* vsite[2];         // [parity][cap]
  double* vtau[2];
  int32_t* vs[2];            // +1 / -1 interacting, 0 dead (non-interacting)
  void* N[2][2];             // [parity][spin] cap x cap, row-major, ld = cap; FP64 or FP32
  double* Ascr[2];           // [spin] cap x cap FP64 work matrix of the recompute (mixed only)
  void* OzA[2];              // [spin][5][cap][cap] FP16 digit planes of the rows of A (sliced residual)
  void* OzN[2];              // [spin][4][cap][cap] FP16 digit planes of the columns of N, transposed
  int32_t* OzE[2];           // [spin][2][cap] their exponents: rows of A, columns of N
  int32_t* live_idx;         // [cap] rows of the live vertices, ascending
  int32_t* surv_tmp;         // [cap] scratch for rebuilding live_idx
  Proposal* prop;            // [KS_MAX]
  double* Gc[2];             // [spin][KS_MAX][cap]: G_ext[:, n + c] stored per candidate c
  double* Xr[2];             // [spin][KS_MAX][cap]: X[c, :] = g0[c,:] (e^V - 1) N, stored in the type of N
                             // (FP32 on the mixed path, where X is an FP32 product: read it through xrows())
  // V, U, gR and bvec hold the arithmetic type of the products: FP64 on the
  // FP64 path, FP32 (first half of the buffer, same indexing) on the mixed path.
  double* Vb[2];             // [spin][KS_MAX][cap]: V[c, j] = g0(r_j - r_c, tau_j - tau_c) (0 if j dead)
  double* Ub[2];             // [spin][KS_MAX][cap]: U[c, i] = g0(r_c - r_i, tau_c - tau_i) (e^{V_i} - 1)
  double* Binv[2];           // [spin][KS_MAX][KS_MAX]
  double* aP[2];             // [spin][KS_MAX]
  int32_t* P;                // [KS_MAX] extended index of accepted flips, in order
  int32_t* removed;          // [KS_MAX] live ranks removed this window, ascending
  int32_t* flipped;          // [KS_MAX] live ranks whose auxiliary spin was flipped this window
  int32_t n_flipped;         // accepted flips this window
  int32_t pad_flip;
  int64_t n_neglected;       // proposals rejected by the neglect rule
  int32_t* acc_slot;         // [KS_MAX] candidate slot of the m-th accepted insertion
  int32_t* acc_p;            // [KS_MAX] its position in P
  double* Lrow[2];           // [spin][cap][KS_MAX] rows of L at extended row index
  double* Lp[2];             // [spin][cap][KS_MAX] rows of L Binv at extended row index
  void* Rr[2];               // [spin][KS_MAX][cap] rows of R = N_ext[P, 0:n) (arithmetic type)
  float* Aop[2];             // [spin][hi, lo][cap][KS_MAX] split L' rows (tensor-core update)
  float* Bop[2];             // [spin][hi, lo][cap][KS_MAX] split R^T rows (tensor-core update)
  double* Gacc;              // [2][nc][n_tau_meas]
  double* Gtmp;              // [2][nc][n_tau_meas] correction term of one measurement
  double* gR;                // [2][nc][cap]
  double* bvec;              // [2][nc][cap]
  double* Mgrid;             // [2][nc][nfft_L] delayed-NFFT grid of M (frequency measurement), or null
  double* Mfreq;             // [2][nc][n_omega][re, im] dense-DFT accumulator of M, or null
  unsigned long long* vx;    // [cap] frequency measurement: per vertex (floor(tau/beta 2^56) << 8) | (site + 1), 0 if dead
  void* g4E;                 // [2][cap][S] complex pairs of T: e^{i (w_s tau_j - K_s.r_j)} (two-particle measurement)
  void* g4T;                 // [2][cap][S] complex pairs of T: f_i sum_j N_ij conj(E(j, s))
  double* g4A;               // [S][S][re, im] sum of sign M_up(s1, s2) M_dn(q - s1, q - s2)
  double* g4D;               // [2][S][re, im] sum of sign M_sigma(s, s)
  int32_t* perm;             // [cap] live columns sorted by site (dense DFT)
  int32_t* goff;             // [nc + 1] their site-group offsets
};

#ifdef __CUDACC__
// A walker keeps its first error: later kernels of the same window may meet
// the consequences of the first failure, which would hide its cause.
__device__ __forceinline__ void set_status(WalkerDev& w, int32_t code) { atomicCAS(&w.status, (int32_t)ST_OK, code); }
#endif

// Iteration state of the device-side window loop.  iters and max_iters are
// reset by every sweep call; total_iters only grows and timed_out stays set
// until the host has read it (the calls are stream-ordered and the host
// checks at its next synchronisation).
struct LoopState {
  int64_t iters;
  int64_t max_iters;
  int64_t total_iters;
  int32_t timed_out;
  int32_t pad;
};

// Pooled schedule: the walkers together run until their summed sweep count
// reaches `target`; `go` (recomputed before every window) says whether it has
// not yet.
struct PoolState {
  int64_t target;
  int64_t sum;
  int32_t go;
  int32_t pad;
};

// TMA tensor maps per walker and spin: update operands A and B, N of parity 0
// and 1 (128-row boxes), the candidate tables V and U of the tensor-core
// extension, N of parity 0 and 1 in 32-row boxes (MN-major operand), the
// digit planes of the sliced recompute residual (N: 128-row boxes, A: 64).
constexpr int TMAPS_PER_SPIN = 10;

// Opaque copy of a TMA tensor map (CUtensorMap: 128 bytes, 64-byte aligned).
struct alignas(64) TmapDev {
  uint64_t opaque[16];
};

// N-update kernel of the mixed-precision path.
enum : int32_t {
  UPD_CUDA_CORE = 1,  // FP32 CUDA-core tiles
  UPD_TCGEN05 = 2,    // 3xTF32 tcgen05.mma fed by TMA
};

struct Config {
  int32_t n_walkers;
  int32_t ks;                // k_sub
  int32_t warmup;
  int32_t recompute_every;
  int32_t recompute_sweeps;  // batched schedule: recompute every walker every this many sweeps
  int32_t recompute_gj;      // mixed path: Gauss-Jordan inverse instead of the Newton step
  int32_t recompute_oz;      // mixed path: Newton residual by digit slicing on the tensor cores
  int32_t n_tau_meas;
  int32_t prec;              // PREC_FP64 or PREC_MIXED
  double tie_eps;
  WalkerDev* W;              // [n_walkers]
  const ProblemDev* P;       // [n_problems]
  int32_t* active_count;     // [1]
  int32_t upd_kernel;        // UPD_CUDA_CORE or UPD_TCGEN05 (mixed precision)
  int32_t upd_bn;            // column tile of the tcgen05 N update: 32 or 64 (64 only for k_s <= 64)
  const TmapDev* tmaps;      // [n_walkers][2 spins][TMAPS_PER_SPIN]
  int32_t ext_tc;            // mixed path: candidate products G_ext and X on tcgen05
  int32_t* gj_next;          // [1] next matrix of the Gauss-Jordan work queue (reset by k_build_A)
  int32_t pooled;            // pooled schedule (else lockstep sweeps)
  PoolState* pool;           // [1] target and go flag of the pooled schedule (all walkers)
  int32_t gamma_fp64;        // mixed path: B^-1 and the Schur complements in FP64 (else double-float)
  int32_t tf32_terms;        // products per K step of the tensor-core kernels: 3 (3xTF32) or 1 (TF32)
  long long wait_cycles;     // bound of every mbarrier wait in the tensor-core kernels (SM clocks)
  int32_t recompute_at_measure;  // recompute N in the window of every measurement (before it)
  uint32_t flip_thr;         // a proposal is an auxiliary-spin flip when (word0 >> 2) < flip_thr (0 = none)
  int32_t dup_rule;          // spin changed twice in a window: 0 end the window, 1 reject the proposal,
                             // 2 apply the change within the window
  int32_t n_omega;           // frequency measurement: positive Matsubara frequencies (0 = off)
  int32_t nfft_L;            // its grid points over [0, beta)
  int32_t nfft_msp;          // its window half-width in grid points
  int32_t freq_dft;          // frequency measurement as the dense contraction (else delayed NFFT)
  int32_t n_w4;              // two-particle measurement: fermionic frequencies per sign (0 = off)
  int32_t m4;                // its bosonic transfer index
};

}  // namespace dca
