// problem_host.cu -- host-side validation and table preparation of a problem.
#include <cmath>

#include "problem_host.h"

namespace dca {

int check_problem(const dca_problem& pr, std::string& err) {
  if (pr.nc < 1 || !pr.site_sub || !pr.G0 || pr.n_tau < 1 || !(pr.beta > 0.0) || !(pr.K > 0.0) || !(pr.U >= 0.0) ||
      !std::isfinite(pr.U) || !std::isfinite(pr.beta) || !std::isfinite(pr.K)) {
    err = "invalid scalar or NULL array";
    return DCA_ERR_ARG;
  }
  for (int r = 0; r < pr.nc; ++r) {
    std::vector<int> seen(pr.nc, 0);
    for (int c = 0; c < pr.nc; ++c) {
      const int v = pr.site_sub[r * pr.nc + c];
      if (v < 0 || v >= pr.nc || seen[v]++) {
        err = "site_sub row is not a permutation";
        return DCA_ERR_ARG;
      }
    }
  }
  std::vector<int32_t> add(pr.nc * pr.nc, -1);
  for (int x = 0; x < pr.nc; ++x)
    for (int y = 0; y < pr.nc; ++y) add[y * pr.nc + pr.site_sub[x * pr.nc + y]] = x;
  for (int v : add)
    if (v < 0) {
      err = "site_sub does not define a group difference table";
      return DCA_ERR_ARG;
    }
  const size_t tsz = (size_t)2 * pr.nc * (pr.n_tau + 1);
  for (size_t t = 0; t < tsz; ++t)
    if (!std::isfinite(pr.G0[t])) {
      err = "G0 has a non-finite entry";
      return DCA_ERR_ARG;
    }
  return DCA_OK;
}

void prepare_problem(const dca_problem& pr, ProblemDev& d, std::vector<int32_t>& add, std::vector<double>& g0) {
  d = ProblemDev{};
  d.nc = pr.nc;
  d.n_tau = pr.n_tau;
  d.beta = pr.beta;
  d.K = pr.K;
  // cosh(gamma) = 1 + U beta N_corr / (2K), N_corr = Nc (Sec. 2.3)
  d.gamma = std::acosh(1.0 + pr.U * pr.beta * (double)pr.nc / (2.0 * pr.K));
  d.tau_scale = (double)pr.n_tau / pr.beta;
  for (int sp = 0; sp < 2; ++sp) {
    const double sigma = sp == 0 ? 1.0 : -1.0;
    d.expV[sp][0] = std::exp(-sigma * d.gamma);
    d.expV[sp][1] = std::exp(sigma * d.gamma);
    for (int k = 0; k < 2; ++k) d.rexpVm1[sp][k] = 1.0 / (d.expV[sp][k] - 1.0);
  }
  add.assign(pr.nc * pr.nc, -1);
  for (int x = 0; x < pr.nc; ++x)
    for (int y = 0; y < pr.nc; ++y) add[y * pr.nc + pr.site_sub[x * pr.nc + y]] = x;
  const size_t tsz = (size_t)2 * pr.nc * (pr.n_tau + 1);
  g0.resize(tsz);
  for (size_t t = 0; t < tsz; ++t) g0[t] = -pr.G0[t];
}

}  // namespace dca
