// Every instantiation of the kernels and drivers for quartets (Section 5:
// three 64-bit key words compared lexicographically, one payload word): the
// plain and segmented sorts.  Keeping them in one translation unit means the
// kernel attributes that a driver sets apply to the very kernels it launches.
#include "ips4o_driver.cuh"

namespace ips4o {
ips4o_status sort_quartet(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part) {
    return sort_t<TQuartet>(st, d, n, s, part);
}
ips4o_status sort_from_quartet(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out) {
    return sort_from_t<TQuartet>(st, d, src, n, s, out);
}
ips4o_status sort_segments_quartet(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s) {
    return sort_segments_t<TQuartet>(st, d, segs, s);
}
ips4o_status enqueue_segments_quartet(DeviceState& st, void* d, const uint64_t* d_off, uint64_t count,
                                      cudaStream_t s) {
    return enqueue_segments_t<TQuartet>(st, d, (const u64*)d_off, count, s);
}
ips4o_status upload_class_table_quartet(const ips4o_class_params* t) { return upload_class_table_t<TQuartet>(t); }
ips4o_status reserve_quartet(DeviceState& st, size_t n, size_t num_segments) {
    return reserve_t<TQuartet>(st, n, num_segments);
}
size_t workspace_bytes_quartet(size_t n, int sms) { return workspace_bytes_t<TQuartet>(n, sms); }
ips4o_status sort_strict_quartet(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    return strict_sort_t<TQuartet>(st, d, n, s);
}
size_t strict_workspace_bytes_quartet(size_t n, int sms) { return strict_workspace_bytes_t<TQuartet>(n, sms); }
}  // namespace ips4o
