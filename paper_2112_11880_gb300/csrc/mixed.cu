// Mixed-precision solve: complex64 inner BiCGStab inside complex128
// iterative refinement.  (Built in the next step; rejects the request until
// then.)
#include "internal.hpp"

namespace helm {

helm_status solve_mixed(helm_csr, const double2*, double2*, const helm_opts&, helm_info*, cudaStream_t) {
  return HELM_ERR_INVALID;
}

}  // namespace helm
