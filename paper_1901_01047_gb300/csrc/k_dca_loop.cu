// k_dca_loop.cu -- the outer DCA self-consistency loop around the walkers
// (DCA++ paper Sec. 2.1): coarse-graining, cluster exclusion, the Dyson
// equation for the cluster self-energy from the measured M, mixing, and the
// imaginary-time table of the new bare propagator that dca_walker_update_G0
// takes.  All in FP64 on the GPU; single band, paramagnetic, square lattice
// eps_k = -2t (cos kx + cos ky) - 4t' cos kx cos ky.
//
//   Eq. sigma_dca / G_coarsegrained  Gbar(K, i w_n) = mean over the patch of K of
//                                    [i w_n + mu - eps(K + k~) - Sigma(K, i w_n)]^-1
//   Eq. cluster-exclusion            calG0 = [Gbar^-1 + Sigma]^-1
//   CT-AUX bare propagator           calG0'^-1 = calG0^-1 - U/2 (the +U/2 of H0 in
//                                    Eq. generalized_hubbard)
//   Eq. dyson_sigma                  Sigma = calG0^-1 - <G>^-1, <G> = calG0' - calG0'^2 <M>
//                                    (the walker measured with calG0'; calG0^-1 = calG0'^-1 + U/2)
//   Eq. self-energy-mixing           Sigma <- alpha Sigma + (1 - alpha) Sigma_old
//   table                            G0(r, tau_l) = (1/Nc) sum_K cos(K.r) G0(K, tau_l),
//                                    G0(K, tau) = -e^{-tau xi}/(1 + e^{-beta xi})
//                                      + (2/beta) sum_{n < n_omega} Re[e^{-i w_n tau} R(K, i w_n)],
//                                    R = calG0' - 1/(i w_n - xi_K), xi_K = patch mean of eps - mu + U/2.
// The patch of K is the cell of the reciprocal superlattice centred on K, on
// a midpoint mesh of n_fine x n_fine points.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dca_walker.h"
#include "kernels.h"
#include "problem_host.h"

namespace dca {

constexpr int CG_MAX_POINTS = 4096;  // n_fine <= 64

struct Cplx {
  double re, im;
};

__device__ __forceinline__ Cplx cinv(Cplx z) {
  const double d = z.re * z.re + z.im * z.im;
  return Cplx{z.re / d, -z.im / d};
}
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return Cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

__device__ __forceinline__ double eps_of(double kx, double ky, double t, double tp) {
  const double cx = cos(kx), cy = cos(ky);
  return -2.0 * t * (cx + cy) - 4.0 * tp * cx * cy;
}

// grid (frequency blocks, K); the patch dispersion of K tabulated in shared memory.
__global__ void __launch_bounds__(256) k_coarse_grain(int nc, const double* kpts, double b00, double b01, double b10,
                                                      double b11, int n_fine, double t, double tp, double mu,
                                                      double U, double beta, int n_omega, const double* sigma,
                                                      double* Gbar, double* G0w, double* G0ws, double* xi) {
  __shared__ double s_eps[CG_MAX_POINTS];
  __shared__ double s_red[256];
  const int K = blockIdx.y;
  const int np = n_fine * n_fine;
  const double kx = kpts[2 * K], ky = kpts[2 * K + 1];
  double part = 0.0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const int m1 = p / n_fine, m2 = p - m1 * n_fine;
    const double u1 = ((double)m1 + 0.5) / (double)n_fine - 0.5, u2 = ((double)m2 + 0.5) / (double)n_fine - 0.5;
    const double e = eps_of(kx + u1 * b00 + u2 * b10, ky + u1 * b01 + u2 * b11, t, tp);
    s_eps[p] = e;
    part += e;
  }
  s_red[threadIdx.x] = part;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s_red[threadIdx.x] += s_red[threadIdx.x + o];
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) xi[K] = s_red[0] / (double)np - mu + 0.5 * U;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_omega) return;
  const size_t o = ((size_t)K * n_omega + n) * 2;
  const double w = (2.0 * n + 1.0) * 3.14159265358979323846 / beta;
  const Cplx sg{sigma[o], sigma[o + 1]};
  double gr = 0.0, gi = 0.0;
  for (int p = 0; p < np; ++p) {
    const Cplx g = cinv(Cplx{mu - s_eps[p] - sg.re, w - sg.im});
    gr += g.re;
    gi += g.im;
  }
  const Cplx gb{gr / (double)np, gi / (double)np};
  const Cplx gi_ = cinv(gb);
  const Cplx g0 = cinv(Cplx{gi_.re + sg.re, gi_.im + sg.im});                  // [Gbar^-1 + Sigma]^-1
  const Cplx g0i = cinv(g0);
  const Cplx g0s = cinv(Cplx{g0i.re - 0.5 * U, g0i.im});                      // Hartree-shifted
  Gbar[o] = gb.re;
  Gbar[o + 1] = gb.im;
  G0w[o] = g0.re;
  G0w[o + 1] = g0.im;
  G0ws[o] = g0s.re;
  G0ws[o + 1] = g0s.im;
}

// Sigma(K, i w_n) from the accumulated M of n_sets walkers: <M(K)> =
// [sum_sets sum_spins sum_dr e^{-i K.dr} M(dr)] / (2 sum_sets sign_sum).
// One thread per (K, n).
__global__ void __launch_bounds__(256) k_sigma_update(int nc, int n_omega, const double* k_dot_r, double U,
                                                      const double* G0ws, int n_sets, const double* M_dr,
                                                      double inv_norm, const double* sigma_old, double alpha,
                                                      double* sigma_out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc * n_omega) return;
  const int K = e / n_omega, n = e - K * n_omega;
  double mr = 0.0, mi = 0.0;
  for (int s = 0; s < n_sets; ++s)
    for (int sp = 0; sp < 2; ++sp)
      for (int d = 0; d < nc; ++d) {
        const size_t o = ((((size_t)s * 2 + sp) * nc + d) * n_omega + n) * 2;
        double sn, cs;
        sincos(k_dot_r[(size_t)K * nc + d], &sn, &cs);
        // e^{-i K.dr} M
        mr += cs * M_dr[o] + sn * M_dr[o + 1];
        mi += cs * M_dr[o + 1] - sn * M_dr[o];
      }
  const Cplx M{mr * inv_norm, mi * inv_norm};
  const size_t o = (size_t)e * 2;
  const Cplx g0{G0ws[o], G0ws[o + 1]};
  const Cplx g0g0m = cmul(cmul(g0, g0), M);
  const Cplx G{g0.re - g0g0m.re, g0.im - g0g0m.im};
  const Cplx g0i = cinv(g0), Gi = cinv(G);
  const double sr = g0i.re + 0.5 * U - Gi.re, si = g0i.im - Gi.im;             // calG0^-1 - G^-1
  sigma_out[o] = alpha * sr + (1.0 - alpha) * sigma_old[o];
  sigma_out[o + 1] = alpha * si + (1.0 - alpha) * sigma_old[o + 1];
}

// G0(K, tau_l) for l = 0 .. n_tau: closed-form tail plus the Matsubara sum of
// the remainder.  One thread per (K, l); the phases (2n + 1) l / n_tau are
// reduced exactly modulo 2 before sincospi.
__global__ void __launch_bounds__(256) k_g0_tau(int nc, int n_omega, double beta, int n_tau, const double* G0ws,
                                                const double* xi, double* GK) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc * (n_tau + 1)) return;
  const int K = e / (n_tau + 1), l = e - K * (n_tau + 1);
  const double x = xi[K];
  double acc = 0.0;
  for (int n = 0; n < n_omega; ++n) {
    const double w = (2.0 * n + 1.0) * 3.14159265358979323846 / beta;
    const size_t o = ((size_t)K * n_omega + n) * 2;
    const Cplx tail = cinv(Cplx{-x, w});
    const double rr = G0ws[o] - tail.re, ri = G0ws[o + 1] - tail.im;
    const long long ph = ((2LL * n + 1) * (long long)l) % (2LL * n_tau);
    double sn, cs;
    sincospi((double)ph / (double)n_tau, &sn, &cs);
    acc += cs * rr + sn * ri;  // Re[e^{-i phi} R]
  }
  const double tau = (double)l * beta / (double)n_tau;
  const double tl = x >= 0.0 ? -exp(-tau * x) / (1.0 + exp(-beta * x)) : -exp((beta - tau) * x) / (exp(beta * x) + 1.0);
  GK[e] = tl + 2.0 * acc / beta;
}

// table[sp][r][l] = (1/Nc) sum_K cos(K.r) GK[K][l], both spins.
__global__ void __launch_bounds__(256) k_g0_table(int nc, int n_tau, const double* k_dot_r, const double* GK,
                                                  double* table) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = nc * (n_tau + 1);
  if (e >= m) return;
  const int r = e / (n_tau + 1), l = e - r * (n_tau + 1);
  double acc = 0.0;
  for (int K = 0; K < nc; ++K) acc += cos(k_dot_r[(size_t)K * nc + r]) * GK[(size_t)K * (n_tau + 1) + l];
  acc /= (double)nc;
  table[e] = acc;
  table[m + e] = acc;
}

}  // namespace dca

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

int loop_fail(int code, const std::string& msg) {
  dca::set_handleless_error(msg);
  return code;
}

int check_lattice(const dca_lattice* lat, int32_t n_omega, const char* who) {
  if (!lat || lat->nc < 1 || lat->nc > 64 || !lat->kpts || !lat->k_dot_r || !(lat->beta > 0.0) || lat->n_fine < 1 ||
      lat->n_fine * lat->n_fine > dca::CG_MAX_POINTS || !(lat->U >= 0.0) || n_omega < 1)
    return loop_fail(DCA_ERR_ARG, std::string(who) + ": invalid lattice or frequency count");
  return DCA_OK;
}

// Device scratch of one call, freed on scope exit.
struct Scratch {
  std::vector<void*> p;
  ~Scratch() {
    for (void* q : p) cudaFree(q);
  }
  double* get(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(double) * (n ? n : 1)) != cudaSuccess) return nullptr;
    p.push_back(q);
    return (double*)q;
  }
};

}  // namespace

extern "C" DCA_API int dca_coarse_grain(const dca_lattice* lat, int32_t n_omega, const double* sigma, double* Gbar,
                                        double* G0w, double* G0w_shifted, double* xi_shifted) {
  int rc = check_lattice(lat, n_omega, "dca_coarse_grain");
  if (rc != DCA_OK) return rc;
  if (!sigma) return loop_fail(DCA_ERR_ARG, "dca_coarse_grain: sigma is NULL");
  const int nc = lat->nc;
  const size_t fw = (size_t)nc * n_omega * 2;
  Scratch s;
  double *d_k = s.get(2 * (size_t)nc), *d_sig = s.get(fw), *d_gb = s.get(fw), *d_g0 = s.get(fw), *d_g0s = s.get(fw),
         *d_xi = s.get(nc);
  if (!d_k || !d_sig || !d_gb || !d_g0 || !d_g0s || !d_xi) return loop_fail(DCA_ERR_OOM, "dca_coarse_grain: device memory");
  cudaError_t e = cudaMemcpy(d_k, lat->kpts, sizeof(double) * 2 * nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_sig, sigma, sizeof(double) * fw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    dca::k_coarse_grain<<<dim3((n_omega + 255) / 256, nc), 256>>>(
        nc, d_k, lat->recip[0], lat->recip[1], lat->recip[2], lat->recip[3], lat->n_fine, lat->t, lat->tp, lat->mu,
        lat->U, lat->beta, n_omega, d_sig, d_gb, d_g0, d_g0s, d_xi);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && Gbar) e = cudaMemcpy(Gbar, d_gb, sizeof(double) * fw, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && G0w) e = cudaMemcpy(G0w, d_g0, sizeof(double) * fw, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && G0w_shifted) e = cudaMemcpy(G0w_shifted, d_g0s, sizeof(double) * fw, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && xi_shifted) e = cudaMemcpy(xi_shifted, d_xi, sizeof(double) * nc, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return loop_fail(DCA_ERR_CUDA, std::string("dca_coarse_grain: ") + cudaGetErrorString(e));
  return DCA_OK;
}

extern "C" DCA_API int dca_sigma_update(const dca_lattice* lat, int32_t n_omega, const double* G0w_shifted,
                                        int32_t n_sets, const double* M_dr, const double* sign_sum,
                                        const double* sigma_old, double alpha, double* sigma_out) {
  int rc = check_lattice(lat, n_omega, "dca_sigma_update");
  if (rc != DCA_OK) return rc;
  if (!G0w_shifted || n_sets < 1 || !M_dr || !sign_sum || !sigma_old || !sigma_out || !(alpha > 0.0) || alpha > 1.0)
    return loop_fail(DCA_ERR_ARG, "dca_sigma_update: invalid argument");
  double ss = 0.0;
  for (int i = 0; i < n_sets; ++i) ss += sign_sum[i];
  if (!(ss != 0.0)) return loop_fail(DCA_ERR_NUMERIC, "dca_sigma_update: the sign sum is zero");
  const int nc = lat->nc;
  const size_t fw = (size_t)nc * n_omega * 2, mw = (size_t)n_sets * 2 * fw;
  Scratch s;
  double *d_kr = s.get((size_t)nc * nc), *d_g0s = s.get(fw), *d_m = s.get(mw), *d_old = s.get(fw), *d_out = s.get(fw);
  if (!d_kr || !d_g0s || !d_m || !d_old || !d_out) return loop_fail(DCA_ERR_OOM, "dca_sigma_update: device memory");
  cudaError_t e = cudaMemcpy(d_kr, lat->k_dot_r, sizeof(double) * nc * nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_g0s, G0w_shifted, sizeof(double) * fw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_m, M_dr, sizeof(double) * mw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_old, sigma_old, sizeof(double) * fw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    dca::k_sigma_update<<<(nc * n_omega + 255) / 256, 256>>>(nc, n_omega, d_kr, lat->U, d_g0s, n_sets, d_m,
                                                             1.0 / (2.0 * ss), d_old, alpha, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(sigma_out, d_out, sizeof(double) * fw, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return loop_fail(DCA_ERR_CUDA, std::string("dca_sigma_update: ") + cudaGetErrorString(e));
  return DCA_OK;
}

extern "C" DCA_API int dca_g0_table_from_freq(const dca_lattice* lat, int32_t n_omega, const double* G0w_shifted,
                                              const double* xi_shifted, int32_t n_tau, double* G0_table) {
  int rc = check_lattice(lat, n_omega, "dca_g0_table_from_freq");
  if (rc != DCA_OK) return rc;
  if (!G0w_shifted || !xi_shifted || !G0_table || n_tau < 1)
    return loop_fail(DCA_ERR_ARG, "dca_g0_table_from_freq: invalid argument");
  const int nc = lat->nc;
  const size_t fw = (size_t)nc * n_omega * 2, nt = (size_t)nc * (n_tau + 1);
  Scratch s;
  double *d_kr = s.get((size_t)nc * nc), *d_g0s = s.get(fw), *d_xi = s.get(nc), *d_gk = s.get(nt), *d_tab = s.get(2 * nt);
  if (!d_kr || !d_g0s || !d_xi || !d_gk || !d_tab) return loop_fail(DCA_ERR_OOM, "dca_g0_table_from_freq: device memory");
  cudaError_t e = cudaMemcpy(d_kr, lat->k_dot_r, sizeof(double) * nc * nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_g0s, G0w_shifted, sizeof(double) * fw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_xi, xi_shifted, sizeof(double) * nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    dca::k_g0_tau<<<(unsigned)((nt + 255) / 256), 256>>>(nc, n_omega, lat->beta, n_tau, d_g0s, d_xi, d_gk);
    dca::k_g0_table<<<(unsigned)((nt + 255) / 256), 256>>>(nc, n_tau, d_kr, d_gk, d_tab);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(G0_table, d_tab, sizeof(double) * 2 * nt, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return loop_fail(DCA_ERR_CUDA, std::string("dca_g0_table_from_freq: ") + cudaGetErrorString(e));
  return DCA_OK;
}

extern "C" DCA_API int dca_g4_assemble(int32_t S, const double* A, const double* D, double sign_sum,
                                       const double* G0_up, const double* G0_dn, double* G2_out) {
  if (S < 1 || S > 4096 || !A || !D || !G0_up || !G0_dn || !G2_out)
    return loop_fail(DCA_ERR_ARG, "dca_g4_assemble: invalid argument");
  if (!(sign_sum != 0.0) || !std::isfinite(sign_sum)) return loop_fail(DCA_ERR_NUMERIC, "dca_g4_assemble: sign sum is zero");
  const size_t sq = (size_t)S * S * 2;
  Scratch s;
  double *d_a = s.get(sq), *d_d = s.get(4 * (size_t)S), *d_u = s.get(2 * (size_t)S), *d_n = s.get(2 * (size_t)S),
         *d_o = s.get(sq);
  if (!d_a || !d_d || !d_u || !d_n || !d_o) return loop_fail(DCA_ERR_OOM, "dca_g4_assemble: device memory");
  cudaError_t e = cudaMemcpy(d_a, A, sizeof(double) * sq, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_d, D, sizeof(double) * 4 * S, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_u, G0_up, sizeof(double) * 2 * S, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_n, G0_dn, sizeof(double) * 2 * S, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    dca::launch_g4_assemble(S, d_a, d_d, sign_sum, d_u, d_n, d_o, 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(G2_out, d_o, sizeof(double) * sq, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return loop_fail(DCA_ERR_CUDA, std::string("dca_g4_assemble: ") + cudaGetErrorString(e));
  return DCA_OK;
}
