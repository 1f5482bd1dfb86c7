// kernels.h -- host-side launchers of the walker kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "state.h"

namespace dca {

// Kernel groups of one window (and the per-window extras), timed separately.
enum Group : int {
  GROUP_PROPOSE = 0,         // k_begin
  GROUP_EXTEND = 1,          // k_cand_zero, k_cand_ext (mixed: k_ext_g, k_ext_x), k_cand_cc
  GROUP_METROPOLIS = 2,      // k_metropolis
  GROUP_UPDATE = 3,          // the rank-l update of N
  GROUP_MEASURE = 4,         // k_meas_*
  GROUP_RECOMPUTE = 5,       // k_gj_cluster
  GROUP_UPDATE_PRE = 6,      // k_upd_factors (tcgen05 path) or k_upd_lrow, k_upd_lp_rr
  GROUP_UPDATE_POST = 7,     // k_upd_border, k_window_end, k_compact_N, k_compact_end
  GROUP_RECOMPUTE_PRE = 8,   // k_build_A
  GROUP_RECOMPUTE_POST = 9,  // (k_store_fp32), k_recompute_drift, k_recompute_adopt
  N_GROUPS = 10,
};

// Launch order of the groups in one window.  The recompute (when a period
// is set) comes before the measurement, so a sweep whose last window also
// recomputes N is measured on the recomputed N.
constexpr int WINDOW_GROUPS[] = {GROUP_PROPOSE,       GROUP_EXTEND,    GROUP_METROPOLIS,     GROUP_UPDATE_PRE,
                                 GROUP_UPDATE,        GROUP_UPDATE_POST, GROUP_RECOMPUTE_PRE, GROUP_RECOMPUTE,
                                 GROUP_RECOMPUTE_POST, GROUP_MEASURE};
constexpr int N_WINDOW_GROUPS = (int)(sizeof(WINDOW_GROUPS) / sizeof(int));
inline bool is_recompute_group(int g) {
  return g == GROUP_RECOMPUTE_PRE || g == GROUP_RECOMPUTE || g == GROUP_RECOMPUTE_POST;
}

// Kernel attributes (dynamic shared memory limits); call once per process
// and device before any launch or stream capture.
cudaError_t setup_window_kernels();

// Each launcher returns the number of kernels it launched.
int launch_window_group(int group, const Config& cfg, int max_cap, cudaStream_t st);
void launch_count_active(const Config& cfg, cudaStream_t st);
void launch_loop_control(const Config& cfg, cudaGraphConditionalHandle handle, LoopState* ls, cudaStream_t st);
void launch_loop_reset(LoopState* ls, int64_t max_iters, cudaStream_t st);
void launch_add_target(const Config& cfg, int64_t n_sweeps, cudaStream_t st);
void launch_init(const Config& cfg, int n0, int max_cap, int* d_sgn, cudaStream_t st);
// N of every walker from scratch for the vertex list of its current buffer
// (live rows 0 .. n-1), and the configuration sign.
void launch_rebuild(const Config& cfg, int max_n, int* d_sgn, cudaStream_t st);
void launch_fresh_inverse(const Config& cfg, int max_n, int* d_sgn, cudaStream_t st);
// Gauss-Jordan inverse of the FP64 work matrices, one 8-block cluster each.
void launch_gj(const Config& cfg, int mode, int max_n, int* d_sgn, cudaStream_t st);
// Mixed-precision recompute by one Newton step against the FP64 A = N^-1:
// the two products (R = I - A N0 in FP64, N1 = N0 + N0 R in FP32), then the
// drift measurement and the copy of N1 into the other buffer.
void launch_refine_gemms(const Config& cfg, int max_cap, cudaStream_t st);
// N1 = N0 + N0 R (FP32), R from either residual.
void launch_refine_correct(const Config& cfg, int max_cap, cudaStream_t st);
// The residual R = I - A N0 by exponent-aligned digit slicing on the tensor
// cores (four kernels).
void launch_refine_oz(const Config& cfg, int max_cap, cudaStream_t st);
cudaError_t setup_refine_tc();
void launch_refine_adopt(const Config& cfg, int max_cap, cudaStream_t st);
// part: GROUP_RECOMPUTE_PRE, GROUP_RECOMPUTE or GROUP_RECOMPUTE_POST.
int launch_recompute(int part, const Config& cfg, int max_cap, int* d_sgn, cudaStream_t st);
int launch_measure(const Config& cfg, int max_cap, int max_nc, cudaStream_t st);

// Streaming multiprocessors of the current device (queried once per device;
// 1 if the query fails, which only makes the persistent grids smaller).
int device_sm_count();
// Grid of a persistent kernel without an occupancy query: `per_sm` blocks per
// SM of the current device, at most `items`.
int sm_grid(long long items, int per_sm);

// Grid of a persistent item kernel (for_each_item): as many blocks as the SMs
// hold at once (occupancy of `fn` at `block` threads and `smem` dynamic bytes,
// cached per kernel), at most `items`.
int persist_grid(const void* fn, long long items, int block, size_t smem = 0);
// Candidate extension of the mixed path: the two streaming passes over N.
int launch_ext_mixed(const Config& cfg, int max_cap, cudaStream_t st);
// Tensor-core N update (mixed precision): kernel attributes, tile width for
// a submatrix size, tensor maps of one walker ([spin][A, B, N0, N1]), the
// operand split and the update itself.
cudaError_t setup_update_tc();
// Column tile of the tcgen05 N update for k_s and the requested tile (0 = default 64).
int tc_tile_n(int ks, int bn);
int ext_tile_c(int ks);  // candidate tile (N extent) of the tensor-core extension
bool encode_update_maps(const WalkerDev& w, int ks, int upd_bn, TmapDev* out);
cudaError_t setup_ext_tc();
void launch_ext_g_tc(const Config& cfg, cudaStream_t st);
void launch_ext_x_tc(const Config& cfg, cudaStream_t st);
// L, L' and both split operands of the tensor-core update in one kernel.
void launch_upd_factors(const Config& cfg, int max_cap, cudaStream_t st);
void launch_upd_tc(const Config& cfg, cudaStream_t st);
// g0 = -G0 (FP64 and FP32) from a staged G0, unless an entry is not finite:
// then *bad = 1 and the old table is kept.
void launch_negate(const double* src, double* dst, float* dstf, size_t n, int* bad, int* changed, cudaStream_t st);
// Delayed-NFFT frequency measurement: kernel attributes, the spreading of one
// measurement (launched with the other measurement kernels) and the
// transform of the accumulated grids at read-out (out at per-walker offsets
// d_base, [2][nc][n_omega][re, im] each).
cudaError_t setup_nfft();
int launch_meas_nfft(const Config& cfg, int max_cap, int max_nc, cudaStream_t st);
void launch_nfft_finish(const Config& cfg, int max_nc, const long long* d_base, double* d_out, cudaStream_t st);
// The dense-DFT variant: per measurement the site sort and the contraction;
// at read-out a copy of the accumulators (same output layout).
int launch_meas_ndft(const Config& cfg, int max_cap, int max_nc, cudaStream_t st);
// Two-particle measurement (k_g4.cu): returns the number of kernels launched.
int launch_meas_g4(const Config& cfg, int max_cap, int max_nc, cudaStream_t st);
void launch_g4_assemble(int S, const double* A, const double* D, double sign_sum, const double* Gu, const double* Gd,
                        double* out, cudaStream_t st);
void launch_ndft_copy(const Config& cfg, int max_nc, const long long* d_base, double* d_out, cudaStream_t st);
// Every walker's tau-grid accumulator to d_out + d_base[walker] (one read-out copy).
void launch_gather_G(const Config& cfg, int max_nc, const long long* d_base, double* d_out, cudaStream_t st);
// Phase table of the measurement grid (ProblemDev::g0m) from the FP32 table g0f.
void launch_meas_table(const ProblemDev& pd, int n_tau_meas, cudaStream_t st);
// Every problem's staged table checked, committed (where finite) and its
// measurement phase table rebuilt: three kernels.
void launch_g0_update_all(const ProblemDev* d_P, int np, int ntm, const double* stage, const long long* off, int* bad,
                          int* bad_any, int* changed, cudaStream_t st);
// N rebuilt from scratch (in place) for the walkers whose problem has
// changed[problem] != 0; returns the number of kernels launched.
int launch_rebuild_changed(const Config& cfg, int max_cap, const int* changed, int* d_sgn, cudaStream_t st);
void launch_g0_isolated(int nc, const double* d_eps, const double* d_kr, double mu_eff, double beta, int n_tau,
                        double* d_out, cudaStream_t st);

}  // namespace dca
