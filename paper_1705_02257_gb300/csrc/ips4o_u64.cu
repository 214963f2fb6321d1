// Instantiation of the distribution-step driver for one element type.
#include "ips4o_driver.cuh"

namespace ips4o {
ips4o_status sort_u64(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part) {
    return sort_t<TU64>(st, d, n, s, part);
}
size_t workspace_bytes_u64(size_t n, int sms) { return workspace_bytes_t<TU64>(n, sms); }
}  // namespace ips4o
