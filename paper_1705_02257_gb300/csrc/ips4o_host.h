// ips4o_host.h — host-side state shared by the per-type drivers and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/ips4o.h"

namespace ips4o {

struct DeviceState {
    int device = -1;
    int sms = 0;
    void* d_ws = nullptr;           // workspace (device)
    size_t ws_bytes = 0;
    void* h_stage = nullptr;        // pinned host staging for descriptors / readback
    size_t h_stage_bytes = 0;
    void* d_host_copy = nullptr;    // device buffer for ips4o_sort_host
    size_t d_host_copy_bytes = 0;
    void* d_aux = nullptr;          // 100-byte records: pairs, input copy, run bounds
    size_t aux_bytes = 0;
    unsigned* d_status = nullptr;   // status word of the last enqueue-only call on this stream
    bool attrs_ready[5] = {false, false, false, false, false};   // kernel attributes set, per element type
    int permute_grid[5] = {0, 0, 0, 0, 0};
    // largest n and segment count the workspace was reserved for, per element
    // type (ips4o_reserve_workspace): the enqueue-only segmented sort sizes
    // its level queues from them
    uint64_t reserved_n[5] = {0, 0, 0, 0, 0};
    uint64_t reserved_segments[5] = {0, 0, 0, 0, 0};
    std::vector<cudaEvent_t> events;
    struct Timed { int phase; int ev; };
    std::vector<Timed> timed;       // profiled launches whose events have not been read yet
    int next_event = 0;
    // a device-planned (asynchronous) call whose statistics and status have
    // not been read back yet: its loop state and stream
    bool pending = false;
    const void* pending_ls = nullptr;
    cudaStream_t pending_stream = nullptr;
    std::mutex mtx;
    ips4o_stats stats{};
};

// Completes the statistics of the last asynchronous call on this state
// (waits for its stream; reads the device loop state and the profiling
// events) and returns the device-side status it recorded.  Callers hold
// st.mtx.
ips4o_status finalize_pending(DeviceState& st);
// Kernel times of the profiled launches whose events were recorded on the
// state (params.profile), added to its statistics.  The events must have
// completed (the caller has synchronised the stream).
ips4o_status collect_profile_events(DeviceState& st);

// The library's default parameters (what ips4o_set_params(NULL) restores).
constexpr ips4o_params kDefaultParams = {256, 0, 0, 1, 0, 0x2545F4914F6CDD1Dull, 0, 0, 0, 0};

DeviceState* stream_state(void* stream, cudaError_t* err);   // state of (current device, stream)
DeviceState* current_device_state(cudaError_t* err);          // state of (current device, NULL stream)
ips4o_params& global_params();
void set_last_cuda_error(cudaError_t e, const char* where);
void set_last_message(const char* msg);
ips4o_status ensure_device_buffer(void** ptr, size_t* have, size_t need);
ips4o_status ensure_host_pinned(void** ptr, size_t* have, size_t need);

// Per-type entry points (defined in ips4o_<type>.cu).
struct PartitionOut {
    uint64_t* bounds;
    size_t* num_buckets;
    uint64_t* splitters;
    size_t* num_splitters;
    int* eq;
};

ips4o_status sort_u64(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part);
ips4o_status sort_f64(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part);
ips4o_status sort_pair(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part);
// d = the sorted elements of src (device-accessible, only read; n elements)
ips4o_status sort_from_u64(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out);
ips4o_status sort_from_f64(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out);
ips4o_status sort_from_pair(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out);
struct Task;
ips4o_status sort_segments_u64(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s);
ips4o_status enqueue_segments_u64(DeviceState& st, void* d, const uint64_t* d_off, uint64_t count, cudaStream_t s);
ips4o_status enqueue_segments_f64(DeviceState& st, void* d, const uint64_t* d_off, uint64_t count, cudaStream_t s);
ips4o_status enqueue_segments_pair(DeviceState& st, void* d, const uint64_t* d_off, uint64_t count, cudaStream_t s);
ips4o_status sort_segments_f64(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s);
ips4o_status sort_segments_pair(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s);
// Per size class leaves / alpha (0 = the default rule), indexed by floor(log2 n).
const ips4o_class_params* class_table();
ips4o_status upload_class_table_u64(const ips4o_class_params* t);
ips4o_status upload_class_table_f64(const ips4o_class_params* t);
ips4o_status upload_class_table_pair(const ips4o_class_params* t);

// ips4o_sort_noalloc: its fixed scratch and limits, and its level loop
// (tasks = 2 * kNoAllocMaxTasks entries)
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // device scratch, 16 MiB
constexpr size_t kNoAllocHostBytes = (size_t)1 << 20;       // host staging, 1 MiB
constexpr size_t kNoAllocMaxN = (size_t)1 << 20;            // largest array, in elements
constexpr size_t kNoAllocMaxTasks = 256;                    // subproblems per level
ips4o_status sort_noalloc_u64(DeviceState& st, void* d, size_t n, cudaStream_t s, Task* tasks);
ips4o_status sort_noalloc_f64(DeviceState& st, void* d, size_t n, cudaStream_t s, Task* tasks);
ips4o_status sort_noalloc_pair(DeviceState& st, void* d, size_t n, cudaStream_t s, Task* tasks);
ips4o_status reserve_u64(DeviceState& st, size_t n, size_t num_segments);
ips4o_status reserve_f64(DeviceState& st, size_t n, size_t num_segments);
ips4o_status reserve_pair(DeviceState& st, size_t n, size_t num_segments);
ips4o_status sort_quartet(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part);
ips4o_status sort_from_quartet(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out);
ips4o_status sort_segments_quartet(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s);
ips4o_status enqueue_segments_quartet(DeviceState& st, void* d, const uint64_t* d_off, uint64_t count,
                                      cudaStream_t s);
ips4o_status upload_class_table_quartet(const ips4o_class_params* t);
ips4o_status reserve_quartet(DeviceState& st, size_t n, size_t num_segments);
size_t workspace_bytes_quartet(size_t n, int sms);
ips4o_status sort_rec100(DeviceState& st, void* d, size_t n, cudaStream_t s);
size_t rec100_aux_bytes(size_t n);
size_t workspace_bytes_u64(size_t n, int sms);
// the strictly in-place sort (Section 4.6) per element type, and its workspace
ips4o_status sort_strict_u64(DeviceState& st, void* d, size_t n, cudaStream_t s);
ips4o_status sort_strict_f64(DeviceState& st, void* d, size_t n, cudaStream_t s);
ips4o_status sort_strict_pair(DeviceState& st, void* d, size_t n, cudaStream_t s);
ips4o_status sort_strict_quartet(DeviceState& st, void* d, size_t n, cudaStream_t s);
ips4o_status sort_strict_rec100(DeviceState& st, void* d, size_t n, cudaStream_t s);
size_t strict_workspace_bytes_u64(size_t n, int sms);
size_t strict_workspace_bytes_f64(size_t n, int sms);
size_t strict_workspace_bytes_pair(size_t n, int sms);
size_t strict_workspace_bytes_quartet(size_t n, int sms);
size_t strict_workspace_bytes_rec100(size_t n, int sms);
size_t workspace_bytes_f64(size_t n, int sms);
size_t workspace_bytes_pair(size_t n, int sms);

}  // namespace ips4o
