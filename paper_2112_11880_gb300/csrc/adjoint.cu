// Adjoint of u = A^{-1} b.  (Built in a later step; rejects the request until
// then.)
#include "internal.hpp"

extern "C" helm_status helm_adjoint(helm_csr, const void*, const void*, const helm_opts*, void*, void*,
                                    helm_info*, helm_stream_t) {
  return HELM_ERR_INVALID;
}
