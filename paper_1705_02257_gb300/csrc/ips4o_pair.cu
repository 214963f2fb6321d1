// Instantiation of the distribution-step driver for one element type.
#include "ips4o_driver.cuh"

namespace ips4o {
ips4o_status sort_pair(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part) {
    return sort_t<TPair>(st, d, n, s, part);
}
size_t workspace_bytes_pair(size_t n, int sms) { return workspace_bytes_t<TPair>(n, sms); }
}  // namespace ips4o
