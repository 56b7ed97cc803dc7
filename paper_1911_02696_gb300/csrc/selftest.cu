// Self-test of the bounded mbarrier wait: one warp waits on a barrier whose
// phase never completes, gives up after the limit, records the timeout in
// the device error word and returns.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace ppc {

__global__ void selftest_timeout_kernel(unsigned* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival that never comes
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = __all_sync(FULL_MASK, mbar_wait_bounded(&bar, 0, limit_ns));
  if (!ok && threadIdx.x == 0) atomicOr(err, ERR_BIT_TIMEOUT_FULL);
}

}  // namespace ppc

extern "C" int pospopcnt_selftest_timeout(uint64_t limit_ns, cudaStream_t stream) {
  if (limit_ns > 1000000000ull) return POSPOPCNT_ERR_INVALID;
  int rc = POSPOPCNT_OK;
  ppc::DeviceState* st = ppc::current_state(&rc);
  if (!st) return rc;
  ppc::selftest_timeout_kernel<<<1, 32, 0, stream>>>(st->d_err, limit_ns);
  ppc::note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? POSPOPCNT_OK : ppc::cuda_fail(e);
}
