// pid_selftest_wait_timeout: exercises the bounded-wait path of the kernels. One thread
// waits on an mbarrier that nothing arrives at; the bounded wait gives up after the given
// time and the kernel reports ERR_TIMEOUT in the handle's error word, which the next
// pid_sync returns as PID_ERR_TIMEOUT. The context stays usable: nothing faults or traps.
#include <cuda.h>
#include <cuda_runtime.h>

#include "capi_internal.h"
#include "device.cuh"
#include "internal.h"

namespace pidk {

__global__ void wait_timeout_kernel(uint32_t* err, uint64_t timeout_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, timeout_ns)) atomicOr(err, ERR_TIMEOUT);
  __syncthreads();
}

}  // namespace pidk

using namespace pidk;
using namespace pidh;

extern "C" pid_status pid_selftest_wait_timeout(pid_handle h, double seconds, void* stream) {
  if (!h) return PID_ERR_INVALID_ARG;
  if (!(seconds > 0.0 && seconds <= 2.0))
    return fail(h, PID_ERR_INVALID_ARG, "seconds must be in (0, 2]");
  DeviceGuard g(h->device);
  wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
      h->err_word, static_cast<uint64_t>(seconds * 1e9));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "wait-timeout kernel launch");
  return PID_OK;
}
