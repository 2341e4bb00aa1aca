// Tensor-core Gram for full PID (placeholder until the tcgen05 kernel lands).
#include "capi_internal.h"

namespace pidh {

pid_status plan_gram(pid_handle h, const EnsInput&, GramPlan*) {
  return fail(h, PID_ERR_UNSUPPORTED, "tensor-core Gram not built yet; use PID_FP32");
}

pid_status launch_gram_one(pid_handle h, const EnsInput&, const GramPlan&, EnsPlan&, float*,
                           cudaStream_t) {
  return fail(h, PID_ERR_UNSUPPORTED, "tensor-core Gram not built yet");
}

pid_status launch_gram_batch(pid_handle h, const GramPlan&, const pidk::EnsDesc*, int, int, double,
                             double, cudaStream_t) {
  return fail(h, PID_ERR_UNSUPPORTED, "tensor-core Gram not built yet");
}

}  // namespace pidh
