// Single-stream kernels instantiated for 32-bit words.
#include "plain_kernels.cuh"

namespace ppc {
template int launch_plain_k<32>(const DeviceState&, const pospopcnt_config&, const void*, size_t,
                               unsigned long long*, bool, cudaStream_t, const PlainAcc&);
template int launch_plain_sysmem_k<32>(const DeviceState&, const void*, size_t, unsigned long long*,
                                       cudaStream_t);
}  // namespace ppc
