// kernels.h -- host-side launchers of the walker kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "state.h"

namespace dca {

// Kernel groups of one window (and the per-window extras), timed separately.
enum Group : int {
  GROUP_PROPOSE = 0,     // k_begin
  GROUP_EXTEND = 1,      // k_cand_g, k_cand_x, k_cand_cc
  GROUP_METROPOLIS = 2,  // k_metropolis
  GROUP_UPDATE = 3,      // k_upd_lrow, k_upd_lp_rr, k_upd_apply, k_upd_border, k_window_end,
                         // k_compact_N, k_compact_end
  GROUP_MEASURE = 4,     // k_meas_*
  GROUP_RECOMPUTE = 5,   // k_build_A, k_gj_cluster, (k_store_fp32), k_recompute_finish
  N_GROUPS = 6,
};

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
void launch_fresh_inverse(const Config& cfg, int max_n, int* d_sgn, cudaStream_t st);
// Gauss-Jordan inverse of the FP64 work matrices, one 8-block cluster each.
void launch_gj(const Config& cfg, int mode, int max_n, int* d_sgn, cudaStream_t st);
int launch_recompute(const Config& cfg, int max_cap, int* d_sgn, cudaStream_t st);
int launch_measure(const Config& cfg, int max_cap, int max_nc, cudaStream_t st);
void launch_negate(const double* src, double* dst, size_t n, cudaStream_t st);
void launch_g0_isolated(int nc, const double* d_eps, const double* d_kr, double mu_eff, double beta, int n_tau,
                        double* d_out, cudaStream_t st);

}  // namespace dca
