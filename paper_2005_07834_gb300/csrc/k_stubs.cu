// Entry points of stages that are not available in this build.
#include "lrs_internal.h"

namespace lrs {

int backward_site(lrs_ctx* ctx, Site& s, const double*, const double*, double*, double2*) {
  (void)ctx; (void)s;
  return set_error(LRS_ERR_UNSUPPORTED, "adjoint not built");
}

}  // namespace lrs
