// DACG (Algorithm 3) and IRLM (Algorithm 1 right) on the device kernels.
#include "internal.h"

namespace lapeig {

int solve_dacg(lap_graph*, int, double, const lap_opts&, bool, SolveOut&) {
  set_error("DACG is not available in this build");
  return LAP_EINVAL;
}

int solve_irlm(lap_graph*, int, double, const lap_opts&, bool, SolveOut&) {
  set_error("IRLM is not available in this build");
  return LAP_EINVAL;
}

}  // namespace lapeig
