// Every instantiation of the kernels and drivers for one element type: the
// plain, segmented and no-allocation sorts.  Keeping them in one translation
// unit means the kernel attributes that a driver sets apply to the very
// kernels it launches.
#include "ips4o_noalloc_driver.cuh"

namespace ips4o {
ips4o_status sort_f64(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part) {
    return sort_t<TF64>(st, d, n, s, part);
}
ips4o_status sort_from_f64(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out) {
    return sort_from_t<TF64>(st, d, src, n, s, out);
}
ips4o_status sort_segments_f64(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s) {
    return sort_segments_t<TF64>(st, d, segs, s);
}
ips4o_status enqueue_segments_f64(DeviceState& st, void* d, const uint64_t* d_off, uint64_t count, cudaStream_t s) {
    return enqueue_segments_t<TF64>(st, d, (const u64*)d_off, count, s);
}
ips4o_status upload_class_table_f64(const ips4o_class_params* t) { return upload_class_table_t<TF64>(t); }
ips4o_status sort_noalloc_f64(DeviceState& st, void* d, size_t n, cudaStream_t s, Task* tasks) {
    return noalloc_sort_t<TF64>(st, d, n, s, tasks);
}
ips4o_status reserve_f64(DeviceState& st, size_t n, size_t num_segments) {
    return reserve_t<TF64>(st, n, num_segments);
}
size_t workspace_bytes_f64(size_t n, int sms) { return workspace_bytes_t<TF64>(n, sms); }
ips4o_status sort_strict_f64(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    return strict_sort_t<TF64>(st, d, n, s);
}
size_t strict_workspace_bytes_f64(size_t n, int sms) { return strict_workspace_bytes_t<TF64>(n, sms); }
}  // namespace ips4o
