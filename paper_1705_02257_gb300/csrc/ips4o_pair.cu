// Every instantiation of the kernels and drivers for one element type: the
// plain, segmented and no-allocation sorts.  Keeping them in one translation
// unit means the kernel attributes that a driver sets apply to the very
// kernels it launches.
#include "ips4o_noalloc_driver.cuh"

namespace ips4o {
ips4o_status sort_pair(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part) {
    return sort_t<TPair>(st, d, n, s, part);
}
ips4o_status sort_from_pair(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out) {
    return sort_from_t<TPair>(st, d, src, n, s, out);
}
ips4o_status sort_segments_pair(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s) {
    return sort_segments_t<TPair>(st, d, segs, s);
}
ips4o_status enqueue_segments_pair(DeviceState& st, void* d, const uint64_t* d_off, uint64_t count, cudaStream_t s) {
    return enqueue_segments_t<TPair>(st, d, (const u64*)d_off, count, s);
}
ips4o_status upload_class_table_pair(const ips4o_class_params* t) { return upload_class_table_t<TPair>(t); }
ips4o_status sort_noalloc_pair(DeviceState& st, void* d, size_t n, cudaStream_t s, Task* tasks) {
    return noalloc_sort_t<TPair>(st, d, n, s, tasks);
}
ips4o_status reserve_pair(DeviceState& st, size_t n, size_t num_segments) {
    return reserve_t<TPair>(st, n, num_segments);
}
size_t workspace_bytes_pair(size_t n, int sms) { return workspace_bytes_t<TPair>(n, sms); }
ips4o_status sort_strict_pair(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    return strict_sort_t<TPair>(st, d, n, s);
}
size_t strict_workspace_bytes_pair(size_t n, int sms) { return strict_workspace_bytes_t<TPair>(n, sms); }
}  // namespace ips4o
