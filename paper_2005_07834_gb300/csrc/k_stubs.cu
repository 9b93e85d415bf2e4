// Entry points of stages that are not available in this build.
#include "lrs_internal.h"

namespace lrs {

int project_mixed(lrs_ctx* ctx, Site& s) {
  (void)ctx; (void)s;
  return set_error(LRS_ERR_UNSUPPORTED, "mixed-precision projection not built");
}

int chi0_mixed(lrs_ctx* ctx, Site& s) {
  (void)ctx; (void)s;
  return set_error(LRS_ERR_UNSUPPORTED, "mixed-precision chi0 not built");
}

int backward_site(lrs_ctx* ctx, Site& s, const double*, const double*, double*, double2*) {
  (void)ctx; (void)s;
  return set_error(LRS_ERR_UNSUPPORTED, "adjoint not built");
}

}  // namespace lrs
