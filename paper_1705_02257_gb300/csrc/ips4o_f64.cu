// Instantiation of the distribution-step driver for one element type.
#include "ips4o_driver.cuh"

namespace ips4o {
ips4o_status sort_f64(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part) {
    return sort_t<TF64>(st, d, n, s, part);
}
size_t workspace_bytes_f64(size_t n, int sms) { return workspace_bytes_t<TF64>(n, sms); }
}  // namespace ips4o
