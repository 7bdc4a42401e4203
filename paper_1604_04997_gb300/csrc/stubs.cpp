// Entry points whose kernels are not built yet report PM_ERR_UNSUPPORTED.
#include "pm.h"
#include "pm_internal.h"

extern "C" pm_status pm_serve_set_weights(pm_ctx *, const double *, int32_t) {
  return pm_set_error(PM_ERR_UNSUPPORTED, "serving is not available in this build");
}
extern "C" pm_status pm_serve_start(pm_ctx *, const pm_serve_config *) {
  return pm_set_error(PM_ERR_UNSUPPORTED, "serving is not available in this build");
}
extern "C" pm_status pm_serve_submit(pm_ctx *, const pm_query *, uint64_t *) {
  return pm_set_error(PM_ERR_UNSUPPORTED, "serving is not available in this build");
}
extern "C" pm_status pm_serve_poll(pm_ctx *, uint64_t, int32_t) {
  return pm_set_error(PM_ERR_UNSUPPORTED, "serving is not available in this build");
}
extern "C" pm_status pm_serve_stop(pm_ctx *) { return PM_OK; }
