// kernels.h -- host-side launchers of the walker kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "state.h"

namespace dca {

void launch_window(const Config& cfg, int max_cap, cudaStream_t st);
void launch_count_active(const Config& cfg, cudaStream_t st);
void launch_add_target(const Config& cfg, int64_t n_sweeps, cudaStream_t st);
void launch_init(const Config& cfg, int n0, int max_cap, int* d_sgn, cudaStream_t st);
void launch_recompute(const Config& cfg, int max_cap, int* d_sgn, cudaStream_t st);
void launch_measure(const Config& cfg, int max_cap, int max_nc, cudaStream_t st);
void launch_g0_isolated(int nc, const double* d_eps, const double* d_kr, double mu_eff, double beta, int n_tau,
                        double* d_out, cudaStream_t st);

}  // namespace dca
