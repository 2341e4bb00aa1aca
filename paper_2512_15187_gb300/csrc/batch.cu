// Batched execution of many ensembles (placeholder until the persistent batch lands).
#include "capi_internal.h"

namespace pidh {

void destroy_batch_cache(pid_handle) {}

}  // namespace pidh

extern "C" pid_status pid_batch(pid_handle h, const pid_ensemble*, int32_t, void*) {
  return pidh::fail(h, PID_ERR_UNSUPPORTED, "pid_batch not built yet");
}
