// Entry points whose kernels are not built yet: they report LQ_ERR_UNSUPPORTED.
#include "lq_internal.h"
using namespace lq;
extern "C" lq_status lq_stout_backward(const lq_field*, double, int, unsigned, const lq_field*, double, lq_field*,
                                       lq_field*, const lq_backward_opts*, void*) {
  set_error("lq_stout_backward: not available in this build");
  return LQ_ERR_UNSUPPORTED;
}
extern "C" lq_status lq_stout_smear_batch(lq_field* const*, int, double, int, unsigned, const lq_stout_opts*, void*) {
  set_error("lq_stout_smear_batch: not available in this build");
  return LQ_ERR_UNSUPPORTED;
}
