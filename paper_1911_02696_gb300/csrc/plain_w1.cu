// The array popcount (K = 1): the carry-save circuit with one counter.
#include "plain_kernels.cuh"

namespace ppc {
template int launch_plain_k<1>(const DeviceState&, const pospopcnt_config&, const void*, size_t,
                               unsigned long long*, bool, cudaStream_t, const PlainAcc&);
}  // namespace ppc
