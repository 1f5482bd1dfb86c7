// problem_host.h -- host-side validation and table preparation of a problem.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dca_walker.h"
#include "state.h"

namespace dca {

// DCA_OK, or DCA_ERR_ARG with a message: scalars in range, arrays present,
// rows of site_sub permutations that form a difference table, G0 finite.
int check_problem(const dca_problem& pr, std::string& err);

// Scalars of the device record (pointers left null), the site-addition
// table site_add[y*nc + d] = x with site_sub[x*nc + y] = d, and g0 = -G0.
void prepare_problem(const dca_problem& pr, ProblemDev& d, std::vector<int32_t>& add, std::vector<double>& g0);

// Message returned by dca_walker_last_error(NULL) on this thread.
void set_handleless_error(const std::string& msg);

}  // namespace dca
