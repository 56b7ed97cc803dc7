// Single-stream kernel instantiated for 64-bit words.
#include "plain_kernels.cuh"

namespace ppc {
template int launch_plain_k<64>(const DeviceState&, const pospopcnt_config&, const void*, size_t,
                                unsigned long long*, bool, cudaStream_t, const PlainAcc&);
}  // namespace ppc
