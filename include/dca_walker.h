/*
 * dca_walker.h -- C ABI of the GB300 CT-AUX walker library (libdcawalker.so).
 *
 * The library runs continuous-time auxiliary-field QMC walkers (DCA++ paper,
 * Sec. 2.3) on one GPU: submatrix (delayed) updates of the per-spin N
 * matrices (Sec. 2.3, "Submatrix updates"), sign tracking, periodic
 * recomputation of N, and accumulation of the measured Green's function G(tau)
 * (Sec. 2.3, the equation for <G> in terms of M), of M(i w_n) by the delayed
 * NFFT or a dense transform (Sec. 2.3, Eq. nfft) and of the two-particle
 * Green's function (Sec. 2.5); and the steps of the outer DCA loop (Sec. 2.1)
 * that turn the measured M into the next bare propagator.  Every step runs in
 * CUDA kernels built for sm_103a; there is no CPU fallback.
 *
 * Problem statement (Sec. 2.3, Eq. generalized_hubbard and the decoupling
 * equations): a single-band Hubbard cluster of Nc sites with on-site U,
 * inverse temperature beta, expansion constant K > 0 and the bare cluster
 * propagator G0(r, tau) of H0 (which carries the +U/2 shift of
 * Eq. generalized_hubbard).  cosh(gamma) = 1 + U beta Nc / (2K).
 *
 * Conventions
 *   - Every function returns DCA_OK (0) or a negative DCA_ERR_* code; nothing
 *     throws across the ABI.  dca_walker_last_error() gives a message.
 *   - Host arrays passed in are caller-owned and copied during the call.
 *     Output buffers are caller-owned host memory.  Device memory is owned by
 *     the library (allocated in dca_walker_create, freed in destroy).
 *   - Work is ordered on the CUDA stream given at create (NULL = the legacy
 *     default stream).  dca_walker_sweep only enqueues work on that stream
 *     (unless kernel-group timing is on, see dca_walker_set_timing);
 *     dca_walker_sync, measure_G, stats, get_state, get_decision_log, save and
 *     load synchronise it.  Errors a walker meets while its sweeps run (its
 *     status) are reported by the next dca_walker_sync.
 *   - Matrices are row-major.  Spin index 0 = up, 1 = down.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *     (lo32(seed), hi32(seed) ^ walker_index) and counter
 *     (lo32(j), hi32(j), tag, 0); tag 0 = proposal words, 1 = acceptance
 *     uniform, 2 = initial configuration.  Proposal q from its words w0..w3:
 *     a flip when (w0 >> 2) < floor(flip_fraction * 2^30), else an insertion
 *     (w0 bit 0 clear: spin from bit 1, site floor(w1 nc / 2^32), time
 *     beta u53(w2, w3)) or a removal; removal and flip pick the vertex
 *     floor(w1 k / 2^32) of the current order k.
 */
#ifndef DCA_WALKER_H
#define DCA_WALKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DCA_API __attribute__((visibility("default")))
#else
#define DCA_API
#endif

#define DCA_OK 0
#define DCA_ERR_ARG (-1)      /* invalid argument */
#define DCA_ERR_CUDA (-2)     /* a CUDA call failed */
#define DCA_ERR_OOM (-3)      /* device or host allocation failed */
#define DCA_ERR_TIMEOUT (-4)  /* a bounded device wait or poll gave up */
#define DCA_ERR_NUMERIC (-5)  /* NaN / Inf in a ratio, singular recompute */
#define DCA_ERR_STATE (-6)    /* call not valid in the current state */
#define DCA_ERR_CAPACITY (-7) /* a walker's order outgrew its matrix capacity */

/* Arithmetic of the N matrices and their updates.
 *   FP64:   N stored and updated in FP64; every product, ratio and inverse in FP64.
 *   MIXED (= TF32X3): N stored in FP32.  The three N-sized products (the rank-l
 *           update and both candidate products of the extension) run as 3xTF32 on
 *           the tensor cores (or FP32 CUDA cores, DCA_UPD_CUDA_CORE) with FP32
 *           accumulation; the update factors L B^-1 and the rows of accepted
 *           insertions in double-float (FP32 pairs, about 44 bits); Gamma (B^-1) and
 *           the determinant ratios in FP64 (DCA_GAMMA_FP64) or double-float
 *           (DCA_GAMMA_DOUBLE_FLOAT); the recompute from an FP64 A = N^-1 with a
 *           double-float residual.  The FP32 storage of N bounds the accuracy: the
 *           measured errors of N and G against the FP64 walker on the same trajectory
 *           are 1e-6..1e-4 relative, growing with the conditioning of N^-1 and with
 *           the updates since the last recompute; with N recomputed before every
 *           measurement (recompute_at_measure) the accumulated G is within about
 *           3e-7.
 *   TF32:   as MIXED with one TF32 product per K step instead of three (the
 *           tensor-core kernels only); about 11 bits per product. */
#define DCA_PREC_FP64 0
#define DCA_PREC_MIXED 1
#define DCA_PREC_TF32X3 1
#define DCA_PREC_TF32 2

/* Arithmetic of Gamma (B^-1) and the determinant ratios on the mixed paths. */
#define DCA_GAMMA_FP64 0          /* FP64 (default) */
#define DCA_GAMMA_DOUBLE_FLOAT 1  /* FP32 pairs, about 44 bits, on the FP32 pipes */

/* One physical problem (a cluster with its bare propagator). */
typedef struct {
  int32_t nc;              /* cluster sites, 1..64; N_corr = Nc (single band, Sec. 2.3) */
  const int32_t* site_sub; /* host [nc*nc]: index of r_i - r_j folded into the cluster;
                              rows must be permutations of 0..nc-1 */
  double U;                /* on-site interaction, >= 0 */
  double beta;             /* inverse temperature, > 0 */
  double K;                /* expansion constant, > 0 (App. B "expansion-parameter-K") */
  int32_t n_tau;           /* G0 grid intervals, samples at l*beta/n_tau, l = 0..n_tau */
  const double* G0;        /* host [2][nc][n_tau+1] in the paper's sign convention
                              (negative on (0, beta)); l = 0 holds G0(r, 0+),
                              l = n_tau holds G0(r, beta-).  Linear interpolation in
                              between, antiperiodic continuation to (-beta, 0). */
  const double* k_dot_r;   /* host [nc][nc] K_a . r_s (cluster momentum a, site s); read
                              only by the two-particle measurement (n_w4 > 0), else NULL */
  const int32_t* k_sub;    /* host [nc][nc] index of K_a - K_b modulo the reciprocal lattice;
                              same use */
} dca_problem;

typedef struct {
  int32_t n_problems;              /* >= 1 */
  const dca_problem* problems;     /* host [n_problems] */
  int32_t n_walkers;               /* 1 .. 16383 */
  const int32_t* walker_problem;   /* host [n_walkers] problem index per walker, or NULL
                                      for walker w -> problem w % n_problems */
  int32_t k_sub;                   /* proposals per submatrix update, 1..128
                                      (App. B "max-submatrix-size") */
  int32_t recompute_every;         /* recompute N from scratch every this many
                                      submatrix updates; 0 = never */
  int32_t warmup_sweeps;           /* App. B "warm-up-sweeps" */
  int32_t n_tau_meas;              /* measurement grid: tau_a = (a + 1/2) beta / n_tau_meas */
  int32_t precision;               /* DCA_PREC_* */
  int32_t init_config_size;        /* App. B "initial-configuration-size" */
  int32_t capacity;                /* max order per walker (matrix size); 0 = automatic */
  uint64_t seed;                   /* App. B "seed" */
  double tie_eps;                  /* near-tie band on | |R| - u |; 0 = 1e-10 */
  int64_t log_capacity;            /* decision-log bytes per walker; 0 = no log */
  int32_t update_kernel;           /* N-update kernel of DCA_PREC_MIXED: DCA_UPD_* */
  int32_t recompute_sweeps;        /* batched schedule: every walker recomputes N after the
                                      first window of every this-many-th sweep (all walkers in
                                      the same window, so the inverses share the GPU); 0 = off.
                                      Independent of recompute_every. */
  int32_t recompute_method;        /* DCA_RECOMPUTE_* */
  int32_t schedule;                /* DCA_SCHEDULE_*: how dca_walker_sweep shares the windows */
  int32_t gamma_precision;         /* DCA_GAMMA_*: B^-1 and ratios of the mixed paths */
  int32_t recompute_at_measure;    /* 1: recompute N in the window that ends every measured
                                      sweep, before its measurement (the measurement then sees a
                                      from-scratch N instead of one carrying the drift of the
                                      updates since the last recompute); 0: off */
  int32_t n_omega_meas;            /* frequency measurement of M (delayed NFFT, read by
                                      dca_walker_measure_M): positive fermionic Matsubara
                                      frequencies, 8..4096; 0 = off */
  double flip_fraction;            /* probability that a proposal is an auxiliary-spin flip of
                                      a uniformly chosen vertex (Sec. 2.3, the third single-spin
                                      update; R = rho_up rho_dn), in [0, 1]; else insert / remove
                                      with probability 1/2 each.  0 = no flips */
  int32_t duplicate_rule;          /* DCA_DUP_*: a removal or flip that picks a spin already
                                      changed in the current submatrix update */
  int32_t freq_method;             /* DCA_FREQ_*: how the frequency measurement is evaluated */
  int32_t n_w4;                    /* two-particle measurement (dca_walker_measure_G4), particle-
                                      particle up-down channel: fermionic frequencies per sign
                                      (App. B "four-point-fermionic-frequencies"), 1..32; 0 = off */
  int32_t w4_transfer;             /* its bosonic transfer index m, nu_m = 2 pi m / beta
                                      (App. B four-point "frequency-transfer"), |m| <= 64 */
  int32_t q4_transfer;             /* its momentum transfer Q as a cluster-momentum index
                                      (App. B four-point "momentum-transfer"), 0..nc-1 of every problem */
} dca_walker_params;

/* The frequency measurement of M (dca_walker_measure_M):
 *   NFFT: the delayed NFFT of Sec. 2.3 (Eq. nfft): every measurement spreads its
 *         n^2 samples onto an oversampled grid with a Gaussian window; one
 *         transform at read-out;
 *   DFT:  the same sums evaluated directly, as a contraction of N with the
 *         phase factors e^{-i w_n tau_j} (n^2 n_omega multiply-adds per spin;
 *         no window error). */
#define DCA_FREQ_NFFT 0
#define DCA_FREQ_DFT 1

/* Spins changed twice in one submatrix update (Sec. 2.3, "Submatrix updates"):
 *   ABORT:   end the update before that proposal and evaluate it first in the
 *            next one (exact: the chain of single-spin updates);
 *   NEGLECT: reject the proposal (no performance loss; breaks detailed
 *            balance, as the paper notes);
 *   UPDATE:  apply the second change within the update (the paper's first
 *            option, which it carries out with Bennett's factor updating; here
 *            the change of one column of the window's matrix B gives the ratio
 *            1 + c (1 - (B^-1)_qq), and B^-1 follows by a rank-1 Sherman-Morrison
 *            correction): the chain of single-spin updates without ending the
 *            window. */
#define DCA_DUP_ABORT 0
#define DCA_DUP_NEGLECT 1
#define DCA_DUP_UPDATE 2

/* Scheduling of the walkers by dca_walker_sweep(n).  The chains do not depend
 * on it: each walker's windows, recomputes and measurements follow from its
 * own proposal counter and sweep count only.
 *   LOCKSTEP: every walker runs exactly n more sweeps, and all walkers start
 *             each sweep in the same window (a walker with a shorter sweep
 *             waits for the others).
 *   POOLED:   the walkers together run n * n_walkers more sweeps, every walker
 *             taking part in every window until that total is reached (the
 *             measurement budget is shared, as independent walkers of uneven
 *             expansion order do; a walker may stop part-way through a sweep
 *             and resumes it on the next call). */
#define DCA_SCHEDULE_LOCKSTEP 0
#define DCA_SCHEDULE_POOLED 1

/* Recompute of N (the inverse of A = e^V - g0 (e^V - 1), Eq. Zk, formed
 * from scratch in FP64 for the current configuration):
 *   AUTO:      DCA_PREC_FP64 inverts it by Gauss-Jordan with partial
 *              pivoting; the mixed paths apply one Newton step
 *              N <- N + N (I - A N) whose residual I - A N is formed on the
 *              tensor cores from exponent-aligned 9-bit digit planes of A (5)
 *              and N (4), the leading plane products summed exactly (Ozaki
 *              et al., Numer. Algorithms 59, 2012): about 2^-40 of the row /
 *              column maxima, so the step brings the FP32 N back to its
 *              rounding level.  Needs 18 cap^2 bytes per spin and walker.
 *   GJ:        Gauss-Jordan on both paths.
 *   NEWTON_DF: the mixed paths' Newton step with the residual in double-float
 *              arithmetic on the CUDA cores (about 2^-44 of sum |A| |N|). */
#define DCA_RECOMPUTE_AUTO 0
#define DCA_RECOMPUTE_GJ 1
#define DCA_RECOMPUTE_NEWTON_DF 2

/* N-update kernels of the mixed-precision path (ignored by DCA_PREC_FP64). */
#define DCA_UPD_AUTO 0       /* DCA_UPD_TCGEN05 */
#define DCA_UPD_CUDA_CORE 1  /* FP32 CUDA-core tiles */
#define DCA_UPD_TCGEN05 2    /* 3xTF32 tcgen05.mma, operands and N tiles moved by TMA */

/* Vertex of a configuration: site index, imaginary time, auxiliary spin. */
typedef struct {
  int32_t site;
  int32_t s;      /* +1 or -1 */
  double tau;     /* in [0, beta) */
} dca_vertex;

typedef struct {
  int64_t proposals;        /* decided proposals (accepted + rejected) */
  int64_t accepts;
  int64_t near_ties;        /* decisions with | |R| - u | < tie_eps */
  int64_t aborts;           /* submatrix updates ended early by the duplicate-spin rule */
  int64_t windows;          /* submatrix updates done */
  int64_t sweeps;           /* sweeps done (including warm-up) */
  int64_t measurements;
  int64_t recomputes;
  int64_t sweep_length;     /* frozen proposals per measured sweep (0 before set) */
  int32_t order;            /* current expansion order k */
  int32_t status;           /* DCA_OK or the walker's error code */
  double sign;              /* current configuration sign */
  double k_sum;             /* sum of sign * k over measurements (<k> = k_sum / sign_sum) */
  double max_drift;         /* largest max|N - N_fresh| / max|N_fresh| seen at recomputes */
  double n_update_flops;    /* algorithmic flop of the N updates (2 n^2 l + 2 n l^2 per spin) */
  double n_update_bytes;    /* algorithmic bytes of the N updates (read + write n^2, n x l factors) */
  double extend_flops;      /* flop of the candidate extension (4 n^2 c per spin) */
  double extend_bytes;      /* algorithmic bytes of the candidate extension (one read of N per spin) */
  double recompute_flops;   /* flop of the from-scratch inverses (2 n^3 per spin) */
  int64_t neglected;        /* proposals rejected by DCA_DUP_NEGLECT */
} dca_walker_stats_t;

typedef struct dca_walker dca_walker;

/*
 * Bare propagator of an isolated cluster for the CT-AUX H0 (effective
 * chemical potential mu - U/2, Eq. generalized_hubbard):
 *   G0(r, tau) = -(1/Nc) sum_K cos(K.r) e^{-tau xi_K} / (1 + e^{-beta xi_K}),
 *   xi_K = eps_K - (mu - U/2),
 * evaluated on the GPU.  eps_K: host [nc]; k_dot_r: host [nc][nc] (K index,
 * site index); G0_out: host [2][nc][n_tau+1] (both spins equal).
 */
DCA_API int dca_g0_isolated_cluster(int32_t nc, const double* eps_K, const double* k_dot_r, double mu,
                            double U, double beta, int32_t n_tau, double* G0_out);

/* Validate parameters, upload problems, draw each walker's initial
 * configuration (init_config_size interacting vertices, counter tag 2) and
 * build its N matrices from scratch.  cuda_stream: a cudaStream_t or NULL. */
DCA_API int dca_walker_create(const dca_walker_params* params, void* cuda_stream, dca_walker** out);

/* Run n_sweeps more sweeps on every walker (DCA_SCHEDULE_LOCKSTEP), or
 * n_sweeps * n_walkers more sweeps over all walkers together
 * (DCA_SCHEDULE_POOLED).  A warm-up sweep is max(k, 1)
 * proposals (k at its start); after warm-up the sweep length is frozen to the
 * rounded mean of those k (max(k,1) when warmup_sweeps = 0).  Every sweep at
 * or past warm-up ends with one measurement.  The submatrix updates run as a
 * device-side loop (a CUDA graph with a conditional WHILE node, captured on
 * the first call) until the sweeps are done: the call enqueues a target
 * kernel and one graph launch on the walker's stream and returns without
 * waiting.  Walker errors (DCA_ERR_NUMERIC, DCA_ERR_CAPACITY, DCA_ERR_TIMEOUT
 * of a bounded wait in a kernel, or of the loop's iteration bound) surface at
 * the next dca_walker_sync.  With kernel-group timing on (dca_walker_set_timing)
 * the host drives the same kernels instead, synchronising the stream between
 * chunks of windows, and the call returns the walkers' errors itself. */
DCA_API int dca_walker_sweep(dca_walker* w, int32_t n_sweeps);

/* Wait for the work enqueued on the walker's stream and report the first
 * error of the sweeps since the last check: DCA_ERR_TIMEOUT if a window loop
 * reached its iteration bound, else the error code of the first walker whose
 * status is not DCA_OK (a walker in error stops; the others go on), else
 * DCA_OK.  The handle stays usable after an error: stats, measure_G,
 * get_state and save work, and dca_walker_load restores every walker. */
DCA_API int dca_walker_sync(dca_walker* w);

/* Switch the schedule (DCA_SCHEDULE_*) between sweeps; the chains do not
 * change.  Synchronises the stream. */
DCA_API int dca_walker_set_schedule(dca_walker* w, int32_t schedule);

/* Bounds of the device-side waits: max_windows caps the windows of one
 * dca_walker_sweep call (0 = the automatic bound, which normal runs never
 * reach); wait_cycles bounds every mbarrier wait inside the tensor-core
 * kernels in SM clock cycles (0 = the default of 4e9, about two seconds).  A
 * bound that runs out stops the affected walkers with DCA_ERR_TIMEOUT, the
 * kernel lets its copies in flight land, frees its tensor memory and returns,
 * so the context stays usable.  Used to exercise the failure paths.
 * Synchronises the stream. */
DCA_API int dca_walker_set_limits(dca_walker* w, int64_t max_windows, int64_t wait_cycles);

/* Checkpoint of every walker's chain (App. B "seed" and the Monte-Carlo
 * parameters make a run reproducible; this makes it resumable): the
 * configuration (vertex list in live order), the sign, the proposal counter
 * (the Philox counter: the random stream continues exactly), the sweep state
 * (position, frozen length, warm-up sums, recompute phase), the counters and
 * the G accumulators.  N is not stored: dca_walker_load rebuilds it from
 * scratch (the periodic recompute, Eq. Zk).  buf may be NULL (or cap too
 * small) to query the size in *n; a non-NULL buf with cap < the size returns
 * DCA_ERR_ARG.  Synchronises the stream. */
DCA_API int dca_walker_save(dca_walker* w, void* buf, size_t cap, size_t* n);

/* Restore a checkpoint written by dca_walker_save into a handle created with
 * the same parameters (walker count, problems, precision and measurement grid
 * are checked): each walker's configuration, sign, counters and accumulators
 * are set, its status reset to the saved one, and N rebuilt from scratch in
 * FP64 (rounded to FP32 on the mixed paths).  The decision log and any forced
 * decisions are left as they are.  Returns DCA_ERR_ARG for a malformed or
 * mismatching buffer (the handle is left unchanged then) and
 * DCA_ERR_NUMERIC if a rebuilt matrix is singular or its determinant sign
 * disagrees with the saved sign.  Synchronises the stream. */
DCA_API int dca_walker_load(dca_walker* w, const void* buf, size_t n);

/* Copy the accumulated sum over measurements of sign * G(dr, tau_a) (paper
 * convention) to G_out [n_walkers][2][nc][n_tau_meas] (nc of each walker's
 * problem; walkers laid out back to back), the sign sums to sign_sum_out
 * [n_walkers] and the measurement counts to n_meas_out [n_walkers].  Any of
 * the outputs may be NULL.  Synchronises the stream. */
DCA_API int dca_walker_measure_G(dca_walker* w, double* G_out, double* sign_sum_out, int64_t* n_meas_out);

/* Accumulated frequency-domain measurement (Sec. 2.3: the Fourier
 * coefficients of M are accumulated; Eq. nfft with the transform delayed to
 * the read-out).  For every walker, spin, cluster difference dr and
 * w_n = (2n + 1) pi / beta, n < n_omega_meas:
 *   sum over measurements of sign * M(dr, i w_n),
 *   M(dr, i w_n) = 1/(beta Nc) sum_{i,j : r_i - r_j = dr} (e^{V_i} - 1) N_ij e^{i w_n (tau_i - tau_j)},
 * so that G(K, i w_n) = G0(K, i w_n) - G0(K, i w_n)^2 <M(K, i w_n)> with
 * M(K) = sum_dr e^{-i K.dr} M(dr) (paper sign convention).  M_out: host
 * [n_walkers][2][nc][n_omega_meas][re, im] (walkers back to back, nc of each
 * walker's problem); sign_sum_out [n_walkers] and n_meas_out [n_walkers] as
 * in dca_walker_measure_G; any output may be NULL.  With DCA_FREQ_NFFT the
 * spreading onto the oversampled grid uses a truncated Gaussian window with a
 * relative error of about 1e-12 (FP64) or 1e-8 (mixed paths); DCA_FREQ_DFT
 * evaluates the sums directly.  Returns DCA_ERR_STATE if the frequency
 * measurement is off.  Synchronises the stream. */
DCA_API int dca_walker_measure_M(dca_walker* w, double* M_out, double* sign_sum_out, int64_t* n_meas_out);

/* Two-particle measurement of the particle-particle up-down channel
 * (Sec. 2.5, Eq. bse_cluster; App. B four-point type PARTICLE_PARTICLE_UP_DOWN).
 * Per configuration the spins are independent, so
 *   G2(K, K', q) = < G_up(K, K') G_dn(q - K, q - K') >,
 *   G_sigma(k1, k2) = G0(k1) delta_{k1 k2} - G0(k1) M_sigma(k1, k2) G0(k2),
 *   M_sigma(k1, k2) = 1/(beta Nc) sum_ij e^{i (w1 tau_i - K1.r_i)} [(e^V - 1) N]_ij e^{-i (w2 tau_j - K2.r_j)},
 * with the combined index k = (K, i w_n) and q = (Q, i nu_m) (q4_transfer,
 * w4_transfer).  The measured points are s = K * 2 n_w4 + n + n_w4 for the
 * cluster momenta K and n = -n_w4 .. n_w4 - 1; the spin-down factor is taken
 * at q - s = (Q - K, i w_{m - n - 1}).  After every measured sweep each walker
 * adds, with S = nc * 2 n_w4,
 *   A(s1, s2) = sign M_up(s1, s2) M_dn(q - s1, q - s2)   [S][S]
 *   D(up, s) = sign M_up(s, s),  D(dn, s) = sign M_dn(q - s, q - s)   [2][S]
 * (M_sigma as dense products on the GPU, FP64 on the FP64 path, FP32 products
 * with FP64 accumulators on the mixed path); G2 for a given G0 follows from
 * them by dca_g4_assemble.  Outputs (host, may be NULL):
 * A_out [W][S_w][S_w][re, im], D_out [W][2][S_w][re, im] concatenated over
 * walkers (S_w of the walker's problem), sign_sum_out [W], n_meas_out [W].
 * Returns DCA_ERR_STATE if the measurement is off.  Synchronises the stream. */
DCA_API int dca_walker_measure_G4(dca_walker* w, double* A_out, double* D_out, double* sign_sum_out,
                                  int64_t* n_meas_out);

/* G2(s1, s2) [S][S][re, im] from one set of accumulators (A [S][S][re, im],
 * D [2][S][re, im], their sign sum) and the bare propagator at the measured
 * points, G0_up [S][re, im] at s and G0_dn [S][re, im] at q - s (paper sign):
 *   G2 sign_sum = G0u(s1) G0d(s1) [ delta_{s1 s2} (sign_sum - D_up(s1) G0u(s1) - D_dn(s1) G0d(s1))
 *                                   + A(s1, s2) G0u(s2) G0d(s2) ].
 * Host arrays; evaluated on the current device.  Returns DCA_ERR_NUMERIC if
 * sign_sum is zero. */
DCA_API int dca_g4_assemble(int32_t S, const double* A, const double* D, double sign_sum, const double* G0_up,
                            const double* G0_dn, double* G2_out);

/* Zero the G accumulators, sign sums and measurement counters. */
DCA_API int dca_walker_reset_measurements(dca_walker* w);

/* Per-walker counters, out [n_walkers].  Synchronises the stream. */
DCA_API int dca_walker_stats(dca_walker* w, dca_walker_stats_t* out);

/* Current configuration of walker wi: verts [capacity], *k = order, and both
 * N matrices as FP64 k x k row-major into N_up / N_dn (each may be NULL). */
DCA_API int dca_walker_get_state(dca_walker* w, int32_t wi, dca_vertex* verts, int32_t* k, double* N_up,
                         double* N_dn);

/* Decision log of walker wi: one byte per proposal number q (bit 0 accepted,
 * bit 1 near tie), out [cap]; *n = number of proposals logged so far. */
DCA_API int dca_walker_get_decision_log(dca_walker* w, int32_t wi, uint8_t* out, int64_t cap, int64_t* n);

/* Replay mode: walker wi takes the accept bit of log[q] instead of its own
 * Metropolis decision for proposal q < n (used to compare arithmetic on an
 * identical trajectory).  n = 0 switches replay off. */
DCA_API int dca_walker_set_forced_decisions(dca_walker* w, int32_t wi, const uint8_t* log, int64_t n);

/* N_sigma = [e^{V_sigma} - g0_sigma (e^{V_sigma} - 1)]^-1 from scratch for a
 * given configuration (all n vertices interacting): the periodic recompute of
 * a walker (Eq. Zk) as a standalone operation.  problem: as in
 * dca_walker_create; verts: host [n] (site in 0..nc-1, s = +-1, 0 <= tau < beta);
 * N_up, N_dn: host n x n row-major outputs (either may be NULL); det_sign:
 * sign of det N_up^-1 det N_dn^-1 (may be NULL).  Runs on the current device
 * and default stream, allocating device memory for the call and freeing it;
 * returns DCA_ERR_NUMERIC if a matrix is singular. */
DCA_API int dca_fresh_N(const dca_problem* problem, int32_t n, const dca_vertex* verts, double* N_up,
                        double* N_dn, int32_t* det_sign);

/* Same operation and outputs as dca_fresh_N, for callers that cannot allocate
 * device memory: processes whose device memory belongs to another allocator
 * (a framework's caching pool that must see every byte), and services that
 * are sized for a fixed device footprint and may not grow it at run time.
 * The paper has no counterpart: it is a deployment variant of the recompute.
 * It calls no cudaMalloc, cudaFree or other allocating routine; all device
 * memory is one fixed file-scope __device__ array (about 3.2 MB, held by
 * every GPU that loads the library until exit).  Limits: n <=
 * DCA_NOALLOC_MAX_ORDER, nc <= DCA_NOALLOC_MAX_SITES, 2 * nc * (n_tau + 1) <=
 * DCA_NOALLOC_MAX_TABLE; larger sizes return DCA_ERR_ARG with a message in
 * dca_walker_last_error(NULL).  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: a cudaDeviceReset invalidates it, so do not call
 * this function again after resetting the device.  Every call reuses the
 * same array and leaves its contents behind; calls are serialised on the
 * host, but GPU work that overlaps a call and touches the array races with
 * it.  It runs on the current device and the legacy default stream with
 * synchronous copies. */
#define DCA_NOALLOC_MAX_ORDER 256
#define DCA_NOALLOC_MAX_SITES 64
#define DCA_NOALLOC_MAX_TABLE 262144
DCA_API int dca_fresh_N_noalloc(const dca_problem* problem, int32_t n, const dca_vertex* verts,
                                double* N_up, double* N_dn, int32_t* det_sign);

/* ---------------------------------------------------------------------------
 * Outer DCA loop (Sec. 2.1): the steps that turn the walkers' measured M into
 * the next bare propagator of the cluster, for the single-band Hubbard model
 * on the square lattice, eps_k = -2t (cos kx + cos ky) - 4t' cos kx cos ky,
 * paramagnetic.  Frequency arrays are host [nc][n_omega][re, im] over the
 * cluster momenta K and w_n = (2n + 1) pi / beta, n < n_omega; everything
 * runs in FP64 on the current device (device memory allocated for the call
 * and freed).  The lattice must be inversion symmetric (G(-K) = G(K)).
 * One iteration:
 *   dca_sigma_update   (after the walkers ran on calG0')   new Sigma
 *   dca_coarse_grain   Gbar, calG0, calG0', xi from Sigma
 *   dca_g0_table_from_freq   the table for dca_walker_update_G0
 * Start with Sigma = 0 (dca_coarse_grain then gives the first bath).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t nc;             /* cluster sites = cluster momenta, 1..64 */
  const double* kpts;     /* host [nc][2] cluster momenta K */
  const double* k_dot_r;  /* host [nc][nc] K . r (K index, site index) */
  double recip[4];        /* reciprocal superlattice vectors b1 = (recip[0], recip[1]),
                             b2 = (recip[2], recip[3]): a_i . b_j = 2 pi delta_ij */
  double t, tp, mu, U, beta;
  int32_t n_fine;         /* patch integration: n_fine x n_fine midpoints per patch, 1..64 */
} dca_lattice;

/* Eqs. sigma_dca and G_coarsegrained, then Eq. cluster-exclusion:
 *   Gbar(K, i w_n) = mean over the patch of K (the reciprocal-superlattice cell
 *                    centred on K) of [i w_n + mu - eps(K + k~) - Sigma(K, i w_n)]^-1,
 *   calG0 = [Gbar^-1 + Sigma]^-1, and the CT-AUX bare propagator of H0 with the
 *   +U/2 shift of Eq. generalized_hubbard, calG0'^-1 = calG0^-1 - U/2;
 *   xi_shifted [nc] = patch mean of eps - mu + U/2 (the high-frequency form
 *   1/(i w_n - xi) of calG0' to second order).  Outputs may be NULL. */
DCA_API int dca_coarse_grain(const dca_lattice* lat, int32_t n_omega, const double* sigma, double* Gbar,
                             double* G0w, double* G0w_shifted, double* xi_shifted);

/* Eq. dyson_sigma and Eq. self-energy-mixing from measurements taken with the
 * bare propagator calG0' (G0w_shifted): M_dr holds n_sets accumulators as
 * written by dca_walker_measure_M for walkers of this problem ([n_sets][2][nc]
 * [n_omega][re, im], sums of sign * M(dr, i w_n)), sign_sum their sign sums;
 *   <M(K)> = sum over sets and spins of sum_dr e^{-i K.dr} M(dr) / (2 sum sign_sum),
 *   <G> = calG0' - calG0'^2 <M>,  Sigma_QMC = calG0'^-1 + U/2 - <G>^-1,
 *   sigma_out = alpha Sigma_QMC + (1 - alpha) sigma_old,  0 < alpha <= 1.
 * Returns DCA_ERR_NUMERIC if the sign sum is zero. */
DCA_API int dca_sigma_update(const dca_lattice* lat, int32_t n_omega, const double* G0w_shifted, int32_t n_sets,
                             const double* M_dr, const double* sign_sum, const double* sigma_old, double alpha,
                             double* sigma_out);

/* The walker table [2][nc][n_tau + 1] (paper sign convention, both spins, as
 * dca_problem.G0 and dca_walker_update_G0 take it) from calG0'(K, i w_n):
 * G0(r, tau_l) = (1/Nc) sum_K cos(K.r) G0(K, tau_l), tau_l = l beta / n_tau,
 * with the tail 1/(i w_n - xi_K) summed in closed form and the remainder over
 * n < n_omega (the remainder falls off as 1/w_n^3). */
DCA_API int dca_g0_table_from_freq(const dca_lattice* lat, int32_t n_omega, const double* G0w_shifted,
                                   const double* xi_shifted, int32_t n_tau, double* G0_table);

/* Replace the bare propagator of problem `problem` (host [2][nc][n_tau+1],
 * same layout and convention as dca_problem.G0), e.g. for the next iteration
 * of an outer DCA loop.  Stream-ordered: the table is copied to a staging
 * buffer on the walker's stream (pass pinned host memory for an asynchronous
 * copy) and sweeps launched afterwards use it.  The table is checked on the
 * device: one with a non-finite entry is not taken (the previous table stays)
 * and the next dca_walker_sync returns DCA_ERR_ARG.  A table that differs
 * from the current one changes N^-1 = e^V - g0 (e^V - 1) of every walker on
 * that problem, so their N is rebuilt from scratch (Gauss-Jordan, FP64) for
 * their current configurations, and their signs are taken from the new
 * determinants; an unchanged table leaves the walkers as they are. */
DCA_API int dca_walker_update_G0(dca_walker* w, int32_t problem, const double* G0);

/* Replace the bare propagators of all problems at once: G0_all is the host
 * concatenation of every problem's table in problem order (problem p:
 * [2][nc_p][n_tau_p + 1], as for dca_walker_update_G0).  One copy to the
 * staging buffers (pinned host memory makes it asynchronous) and three
 * kernels for all problems, stream-ordered like dca_walker_update_G0: the
 * copy itself runs on a stream of the handle, so it overlaps the sweeps
 * enqueued before the call, and the kernels that take the tables wait for it
 * on the walker's stream (with pinned memory the host array must stay
 * unchanged until the stream has passed the copy, e.g. until the next
 * dca_walker_sync); a
 * problem whose table has a non-finite entry keeps its previous table (the
 * others are taken) and the next dca_walker_sync returns DCA_ERR_ARG. */
DCA_API int dca_walker_update_G0_all(dca_walker* w, const double* G0_all);

/* Change the submatrix size (1..128) and the N-update kernel (DCA_UPD_*,
 * mixed precision only) between sweeps.  The submatrix method reaches the
 * same Markov chain as single-spin updates for every k_sub (Sec. 2.3,
 * "Submatrix updates"), so both are pure performance parameters; used by the
 * autotuner.  Synchronises the stream. */
DCA_API int dca_walker_set_tuning(dca_walker* w, int32_t k_sub, int32_t update_kernel);

/* Column tile of the tensor-core N update (DCA_UPD_TCGEN05): 32 or 64
 * columns of N per tile, 0 for the default (64).  With k_sub > 64 the tile is
 * 32 whatever is asked (the operands of the larger K extent leave room for no
 * more).  A performance parameter like k_sub (the results differ only by the
 * order of FP32 additions); used by the autotuner.  DCA_ERR_ARG for another
 * value.  Synchronises the stream. */
DCA_API int dca_walker_set_update_tile(dca_walker* w, int32_t tile_n);

/* Change the recompute schedule between sweeps (the fields of the same names
 * in dca_walker_params): recompute_every (windows, 0 = off), recompute_sweeps
 * (batched schedule, 0 = off) and recompute_at_measure (0 or 1).  N is a
 * function of the configuration, so the chains do not change; only the
 * rounding carried by N between recomputes does.  Synchronises the stream. */
DCA_API int dca_walker_set_recompute(dca_walker* w, int32_t recompute_every, int32_t recompute_sweeps,
                                     int32_t recompute_at_measure);

/* Kernel groups for timing: bit g of the mask times group g with CUDA events
 * recorded on the walker's stream around every launch of that group.
 *   0 proposals, 1 candidate extension (G columns / X rows), 2 Metropolis
 *   with the Gamma (B^-1) growth, 3 the rank-l N update kernel alone,
 *   4 measurement, 5 the from-scratch inverse kernel alone, 6 the factors of
 *   the N update (L B^-1, N[P,:]), 7 the rest of the update (rows of accepted
 *   insertions, dead marking, compaction), 8 the matrix build before the
 *   inverse, 9 the drift check and adoption after it. */
#define DCA_N_GROUPS 10
DCA_API int dca_walker_set_timing(dca_walker* w, uint32_t group_mask);

/* Accumulated milliseconds and kernel launches per group (arrays of
 * DCA_N_GROUPS, either may be NULL) and the total number of kernels the
 * library launched; reset != 0 zeroes the counters.  Synchronises the stream. */
DCA_API int dca_walker_get_timing(dca_walker* w, double* group_ms, int64_t* group_launches,
                                  int64_t* total_launches, int32_t reset);

/* Device buffer sizes and capacity of walker wi (for diagnostics). */
DCA_API int dca_walker_capacity(dca_walker* w, int32_t wi, int32_t* capacity);

DCA_API void dca_walker_destroy(dca_walker* w);

/* Message of the last error on this handle (or of the last failed create
 * when w is NULL).  The string stays valid until the next call on w. */
DCA_API const char* dca_walker_last_error(dca_walker* w);

#ifdef __cplusplus
}
#endif
#endif /* DCA_WALKER_H */
