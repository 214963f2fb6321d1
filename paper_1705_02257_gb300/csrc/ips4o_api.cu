// ips4o_api.cu — the extern "C" entry points declared in include/ips4o.h.
//
// Argument checking, per-device state (workspace, pinned staging, stats),
// and dispatch on the element type to the per-type drivers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "ips4o_common.cuh"
#include "ips4o_host.h"

namespace ips4o {

// Failure-path self-check: a flag that nothing sets and a status word.
static __device__ unsigned g_probe[2];

static __global__ void k_wait_probe(unsigned* words, unsigned spin_limit) {
    if (threadIdx.x == 0 && !wait_flag_set(&words[0], spin_limit)) atomicOr(&words[1], kStatusTimeout);
}

// Copies between device memory and pinned host memory by a kernel: the GPU
// reads and writes pinned host memory directly (over NVLink-C2C on a
// Grace-Blackwell node, over PCIe elsewhere), and a grid of SMs keeps more
// requests in flight than one copy engine.
static __global__ void k_copy16(uint4* __restrict__ dst, const uint4* __restrict__ src, size_t n) {
    // four independent 16-byte loads per thread in flight before the stores
    constexpr int U = 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < n; i += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = src[i + u * stride];
#pragma unroll
        for (int u = 0; u < U; ++u) dst[i + u * stride] = v[u];
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

static __global__ void k_copy4(unsigned* __restrict__ dst, const unsigned* __restrict__ src, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// dst and src are device-accessible addresses; false if the alignment does
// not allow a kernel copy (the caller then uses cudaMemcpyAsync).
static bool kernel_copy(void* dst, const void* src, size_t bytes, cudaStream_t s, int sms, cudaError_t* err) {
    const uintptr_t a = (uintptr_t)dst | (uintptr_t)src | (uintptr_t)bytes;
    const int grid = sms * 16;
    if (a % 16 == 0) k_copy16<<<grid, 256, 0, s>>>((uint4*)dst, (const uint4*)src, bytes / 16);
    else if (a % 4 == 0) k_copy4<<<grid, 256, 0, s>>>((unsigned*)dst, (const unsigned*)src, bytes / 4);
    else return false;
    *err = cudaGetLastError();
    return true;
}

namespace {
std::mutex g_mtx;
// one state (workspace, staging, stats) per (device, stream): calls on
// different streams run side by side, calls on one stream are serialised
std::map<std::pair<int, uintptr_t>, DeviceState*> g_states;
ips4o_stats g_last_stats[64];
ips4o_params g_params = kDefaultParams;
thread_local char g_last_err[256] = {0};
ips4o_class_params g_classes[IPS4O_NUM_CLASSES] = {};
}  // namespace

const ips4o_class_params* class_table() { return g_classes; }

ips4o_params& global_params() { return g_params; }

void set_last_message(const char* msg) { std::snprintf(g_last_err, sizeof g_last_err, "%s", msg); }

void set_last_cuda_error(cudaError_t e, const char* where) {
    std::snprintf(g_last_err, sizeof g_last_err, "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
}

DeviceState* stream_state(void* stream, cudaError_t* err) {
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) { *err = cudaErrorInvalidDevice; return nullptr; }
    std::lock_guard<std::mutex> lk(g_mtx);
    DeviceState*& slot = g_states[std::make_pair(dev, (uintptr_t)stream)];
    if (!slot) {
        DeviceState* s = new DeviceState();
        s->device = dev;
        *err = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
        if (*err != cudaSuccess) { delete s; return nullptr; }
        slot = s;
    }
    return slot;
}

DeviceState* current_device_state(cudaError_t* err) { return stream_state(nullptr, err); }

static DeviceState* g_last_state[64];

static void publish_stats(DeviceState& st) {
    std::lock_guard<std::mutex> lk(g_mtx);
    g_last_stats[st.device] = st.stats;
    g_last_state[st.device] = &st;
}

ips4o_status collect_profile_events(DeviceState& st) {
    for (const DeviceState::Timed& t : st.timed) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, st.events[t.ev], st.events[t.ev + 1]);
        if (e != cudaSuccess) {
            set_last_cuda_error(e, "cudaEventElapsedTime");
            st.timed.clear();
            st.next_event = 0;
            return IPS4O_ERR_CUDA;
        }
        st.stats.phase_ms[t.phase] += ms;
        st.stats.phase_launches[t.phase]++;
    }
    st.timed.clear();
    st.next_event = 0;
    return IPS4O_OK;
}

ips4o_status finalize_pending(DeviceState& st) {
    if (!st.pending) return IPS4O_OK;
    st.pending = false;
    cudaError_t e = cudaStreamSynchronize(st.pending_stream);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaStreamSynchronize");
        return IPS4O_ERR_CUDA;
    }
    LoopState h;
    e = cudaMemcpy(&h, st.pending_ls, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaMemcpy(loop state)");
        return IPS4O_ERR_CUDA;
    }
    st.stats.levels = h.levels;
    st.stats.chunks = (uint32_t)h.chunks;
    st.stats.subproblems = h.subproblems;
    st.stats.blocks_moved = h.blocks_moved;
    st.stats.blocks_skipped = h.blocks_skipped;
    st.stats.fix_blocks_moved = h.fix_blocks;
    st.stats.base_case_buckets = h.base_buckets;
    st.stats.elements_distributed = h.elements_distributed;
    ips4o_status rc = collect_profile_events(st);
    publish_stats(st);
    if (h.guard_hits) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "device bounds guard failed %u time(s); first at kernels line %u (%llu, %llu)",
                      h.guard_hits, h.guard_line, (unsigned long long)h.guard_a, (unsigned long long)h.guard_b);
        set_last_message(msg);
    }
    if (h.status & kStatusTimeout) return IPS4O_ERR_TIMEOUT;
    if (h.status) return IPS4O_ERR_INTERNAL;
    return rc;
}

ips4o_status ensure_device_buffer(void** ptr, size_t* have, size_t need) {
    if (*ptr && *have >= need) return IPS4O_OK;
    if (*ptr) {
        cudaError_t e = cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
        if (e != cudaSuccess) { set_last_cuda_error(e, "cudaFree"); return IPS4O_ERR_CUDA; }
    }
    cudaError_t e = cudaMalloc(ptr, need);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        set_last_cuda_error(e, "cudaMalloc(workspace)");
        return e == cudaErrorMemoryAllocation ? IPS4O_ERR_OOM : IPS4O_ERR_CUDA;
    }
    *have = need;
    return IPS4O_OK;
}

ips4o_status ensure_host_pinned(void** ptr, size_t* have, size_t need) {
    if (*ptr && *have >= need) return IPS4O_OK;
    if (*ptr) {
        cudaFreeHost(*ptr);
        *ptr = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMallocHost(ptr, need);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        set_last_cuda_error(e, "cudaMallocHost(staging)");
        return IPS4O_ERR_OOM;
    }
    *have = need;
    return IPS4O_OK;
}

static size_t elem_size(int kt) {
    switch (kt) {
    case IPS4O_U64: return 8;
    case IPS4O_F64: return 8;
    case IPS4O_PAIR_U64: return 16;
    case IPS4O_REC100_K10: return 100;
    case IPS4O_QUARTET_U64: return 32;
    default: return 0;
    }
}

static size_t elem_align(int kt) {
    return kt == IPS4O_REC100_K10 ? 4 : (kt == IPS4O_QUARTET_U64 ? 16 : elem_size(kt));
}

static ips4o_status check_args(const void* p, size_t n, int kt) {
    if (kt < 0 || kt > IPS4O_QUARTET_U64) return IPS4O_ERR_UNSUPPORTED_TYPE;
    if (elem_size(kt) == 0) return IPS4O_ERR_UNSUPPORTED_TYPE;
    if (n > 1 && !p) return IPS4O_ERR_INVALID_ARG;
    // one bucket region of the block permutation holds at most 2^25 - 2^16 - 2
    // blocks of 512 bytes (the packed pointer word): 16 GiB per call
    if (n > ((size_t)16 << 30) / elem_size(kt)) return IPS4O_ERR_TOO_LARGE;
    if (p && ((uintptr_t)p % elem_align(kt)) != 0) return IPS4O_ERR_MISALIGNED;
    return IPS4O_OK;
}

static ips4o_status dispatch(DeviceState& st, void* d, size_t n, int kt, cudaStream_t s, PartitionOut* part) {
    ips4o_status rc;
    switch (kt) {
    case IPS4O_U64: rc = sort_u64(st, d, n, s, part); break;
    case IPS4O_F64: rc = sort_f64(st, d, n, s, part); break;
    case IPS4O_PAIR_U64: rc = sort_pair(st, d, n, s, part); break;
    case IPS4O_QUARTET_U64: rc = sort_quartet(st, d, n, s, part); break;
    case IPS4O_REC100_K10:
        if (part) return IPS4O_ERR_UNSUPPORTED_TYPE;   // records are sorted through key + index pairs
        rc = sort_rec100(st, d, n, s);
        break;
    default: return IPS4O_ERR_UNSUPPORTED_TYPE;
    }
    publish_stats(st);
    return rc;
}

static ips4o_status dispatch_segments(DeviceState& st, void* d, const std::vector<Task>& segs, int kt,
                                      cudaStream_t s) {
    ips4o_status rc;
    switch (kt) {
    case IPS4O_U64: rc = sort_segments_u64(st, d, segs, s); break;
    case IPS4O_F64: rc = sort_segments_f64(st, d, segs, s); break;
    case IPS4O_PAIR_U64: rc = sort_segments_pair(st, d, segs, s); break;
    case IPS4O_QUARTET_U64: rc = sort_segments_quartet(st, d, segs, s); break;
    default: return IPS4O_ERR_UNSUPPORTED_TYPE;
    }
    publish_stats(st);
    return rc;
}

// Reads `count` 8-byte values from host or device memory (unified addressing).
static ips4o_status read_u64s(const void* src, size_t count, std::vector<uint64_t>* out, cudaStream_t s) {
    out->resize(count);
    if (count == 0) return IPS4O_OK;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, src);
    cudaGetLastError();   // a plain host pointer may leave a query error behind
    const bool on_device = e == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    if (!on_device) {
        std::memcpy(out->data(), src, count * 8);
        return IPS4O_OK;
    }
    e = cudaMemcpyAsync(out->data(), src, count * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaMemcpyAsync(segment table)"); return IPS4O_ERR_CUDA; }
    return IPS4O_OK;
}

// Per-segment limits: the same as one ips4o_sort call.
static ips4o_status check_segment(size_t n, int kt) {
    if (n > ((size_t)16 << 30) / elem_size(kt)) return IPS4O_ERR_TOO_LARGE;
    return IPS4O_OK;
}

}  // namespace ips4o

using namespace ips4o;

extern "C" {

ips4o_status ips4o_sort(void* d_ptr, size_t n, int key_type, void* stream) {
    ips4o_status rc = check_args(d_ptr, n, key_type);
    if (rc != IPS4O_OK) return rc;
    if (n < 2) return IPS4O_OK;
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    return dispatch(*st, d_ptr, n, key_type, (cudaStream_t)stream, nullptr);
}

ips4o_status ips4o_sort_strict(void* d_ptr, size_t n, int key_type, void* stream) {
    ips4o_status rc = check_args(d_ptr, n, key_type);
    if (rc != IPS4O_OK) return rc;
    if (n < 2) return IPS4O_OK;
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaStreamIsCapturing"); return IPS4O_ERR_CUDA; }
    if (cap != cudaStreamCaptureStatusNone) {
        set_last_message("ips4o_sort_strict synchronises between batches: not while the stream is being captured");
        return IPS4O_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    switch (key_type) {
    case IPS4O_U64: rc = sort_strict_u64(*st, d_ptr, n, s); break;
    case IPS4O_F64: rc = sort_strict_f64(*st, d_ptr, n, s); break;
    case IPS4O_PAIR_U64: rc = sort_strict_pair(*st, d_ptr, n, s); break;
    case IPS4O_QUARTET_U64: rc = sort_strict_quartet(*st, d_ptr, n, s); break;
    case IPS4O_REC100_K10: rc = sort_strict_rec100(*st, d_ptr, n, s); break;
    default: return IPS4O_ERR_UNSUPPORTED_TYPE;
    }
    publish_stats(*st);
    if (rc != IPS4O_OK) {
        st->pending = false;
        return rc;
    }
    return finalize_pending(*st);
}

size_t ips4o_workspace_bytes_strict(size_t n, int key_type) {
    int sms = 152;
    cudaError_t e;
    DeviceState* st = current_device_state(&e);
    if (st) sms = st->sms;
    else cudaGetLastError();
    switch (key_type) {
    case IPS4O_U64: return strict_workspace_bytes_u64(n, sms);
    case IPS4O_F64: return strict_workspace_bytes_f64(n, sms);
    case IPS4O_PAIR_U64: return strict_workspace_bytes_pair(n, sms);
    case IPS4O_QUARTET_U64: return strict_workspace_bytes_quartet(n, sms);
    case IPS4O_REC100_K10: return strict_workspace_bytes_rec100(n, sms);
    default: return 0;
    }
}

ips4o_status ips4o_sort_segmented(void* d_base, const uint64_t* offsets, size_t num_segments, int key_type,
                                  void* stream) {
    if (key_type < 0 || key_type > IPS4O_QUARTET_U64 || elem_size(key_type) == 0) return IPS4O_ERR_UNSUPPORTED_TYPE;
    if (num_segments == 0) return IPS4O_OK;
    if (!offsets) return IPS4O_ERR_INVALID_ARG;
    if (d_base && ((uintptr_t)d_base % elem_size(key_type)) != 0) return IPS4O_ERR_MISALIGNED;
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    std::vector<uint64_t> off;
    ips4o_status rc = read_u64s(offsets, num_segments + 1, &off, (cudaStream_t)stream);
    if (rc != IPS4O_OK) return rc;
    std::vector<Task> segs(num_segments);
    for (size_t i = 0; i < num_segments; ++i) {
        if (off[i + 1] < off[i]) return IPS4O_ERR_INVALID_ARG;
        rc = check_segment(off[i + 1] - off[i], key_type);
        if (rc != IPS4O_OK) return rc;
        segs[i] = Task{off[i], off[i + 1] - off[i]};
    }
    if (off[num_segments] > off[0] && !d_base) return IPS4O_ERR_INVALID_ARG;
    return dispatch_segments(*st, d_base, segs, key_type, (cudaStream_t)stream);
}

ips4o_status ips4o_sort_segmented_async(void* d_base, const uint64_t* d_offsets, size_t num_segments, int key_type,
                                        void* stream) {
    if (key_type < 0 || key_type > IPS4O_QUARTET_U64 || key_type == IPS4O_REC100_K10) return IPS4O_ERR_UNSUPPORTED_TYPE;
    if (num_segments == 0) return IPS4O_OK;
    if (!d_offsets || !d_base) return IPS4O_ERR_INVALID_ARG;
    if (((uintptr_t)d_base % elem_align(key_type)) != 0) return IPS4O_ERR_MISALIGNED;
    if (num_segments >= (1ull << 32)) return IPS4O_ERR_TOO_LARGE;
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    cudaStream_t s = (cudaStream_t)stream;
    switch (key_type) {
    case IPS4O_U64: return enqueue_segments_u64(*st, d_base, d_offsets, num_segments, s);
    case IPS4O_F64: return enqueue_segments_f64(*st, d_base, d_offsets, num_segments, s);
    case IPS4O_QUARTET_U64: return enqueue_segments_quartet(*st, d_base, d_offsets, num_segments, s);
    default: return enqueue_segments_pair(*st, d_base, d_offsets, num_segments, s);
    }
}

ips4o_status ips4o_sort_batched(void* const* ptrs, const uint64_t* lens, size_t count, int key_type, void* stream) {
    if (key_type < 0 || key_type > IPS4O_QUARTET_U64 || elem_size(key_type) == 0) return IPS4O_ERR_UNSUPPORTED_TYPE;
    if (count == 0) return IPS4O_OK;
    if (!ptrs || !lens) return IPS4O_ERR_INVALID_ARG;
    const size_t es = elem_size(key_type);
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    std::vector<uint64_t> p, n;
    ips4o_status rc = read_u64s(ptrs, count, &p, (cudaStream_t)stream);
    if (rc == IPS4O_OK) rc = read_u64s(lens, count, &n, (cudaStream_t)stream);
    if (rc != IPS4O_OK) return rc;
    // the arrays as segments of one address range starting at the lowest of them
    std::vector<std::pair<uint64_t, uint64_t>> arr;
    arr.reserve(count);
    for (size_t i = 0; i < count; ++i) {
        if (n[i] == 0) continue;
        if (!p[i]) return IPS4O_ERR_INVALID_ARG;
        if (p[i] % es) return IPS4O_ERR_MISALIGNED;
        rc = check_segment(n[i], key_type);
        if (rc != IPS4O_OK) return rc;
        arr.emplace_back(p[i], n[i]);
    }
    if (arr.empty()) return IPS4O_OK;
    std::sort(arr.begin(), arr.end());
    for (size_t i = 0; i + 1 < arr.size(); ++i)
        if (arr[i].first + arr[i].second * es > arr[i + 1].first) return IPS4O_ERR_INVALID_ARG;   // overlap
    const uint64_t base = arr[0].first;
    std::vector<Task> segs(arr.size());
    for (size_t i = 0; i < arr.size(); ++i) segs[i] = Task{(arr[i].first - base) / es, arr[i].second};
    return dispatch_segments(*st, (void*)(uintptr_t)base, segs, key_type, (cudaStream_t)stream);
}

ips4o_status ips4o_sort_host(void* h_ptr, size_t n, int key_type, void* stream) {
    ips4o_status rc = check_args(h_ptr, n, key_type);
    if (rc != IPS4O_OK) return rc;
    if (n < 2) return IPS4O_OK;
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    const size_t bytes = n * elem_size(key_type);
    rc = ensure_device_buffer(&st->d_host_copy, &st->d_host_copy_bytes, bytes);
    if (rc != IPS4O_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // pinned host memory is read and written by kernels through its device address
    cudaPointerAttributes attr;
    void* h_dev = nullptr;
    if (cudaPointerGetAttributes(&attr, h_ptr) == cudaSuccess && attr.type == cudaMemoryTypeHost)
        h_dev = attr.devicePointer;
    cudaGetLastError();   // a plain pageable pointer may leave a query error behind
    bool by_kernel = false, written = false;
    if (h_dev && key_type != IPS4O_REC100_K10 && (uintptr_t)h_dev % elem_align(key_type) == 0) {
        // pinned host memory and an element type sorted in place: the first
        // distribution level reads the host buffer itself and writes its
        // blocks into the device copy (no separate copy pass), and the base
        // case writes each sorted bucket straight back into the host buffer;
        // the ranges it does not write (equality buckets, single elements,
        // subproblems of the segment scheduler) are copied back by a kernel
        by_kernel = true;
        written = true;
        switch (key_type) {
        case IPS4O_U64: rc = sort_from_u64(*st, st->d_host_copy, h_dev, n, s, h_dev); break;
        case IPS4O_F64: rc = sort_from_f64(*st, st->d_host_copy, h_dev, n, s, h_dev); break;
        case IPS4O_QUARTET_U64: rc = sort_from_quartet(*st, st->d_host_copy, h_dev, n, s, h_dev); break;
        default: rc = sort_from_pair(*st, st->d_host_copy, h_dev, n, s, h_dev); break;
        }
        publish_stats(*st);
        if (rc != IPS4O_OK) return rc;
    } else {
        if (h_dev) {
            by_kernel = kernel_copy(st->d_host_copy, h_dev, bytes, s, st->sms, &e);
            if (by_kernel && e != cudaSuccess) { set_last_cuda_error(e, "copy kernel (H2D)"); return IPS4O_ERR_CUDA; }
        }
        if (!by_kernel) {
            e = cudaMemcpyAsync(st->d_host_copy, h_ptr, bytes, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) { set_last_cuda_error(e, "cudaMemcpyAsync(H2D)"); return IPS4O_ERR_CUDA; }
        }
        rc = dispatch(*st, st->d_host_copy, n, key_type, s, nullptr);
        if (rc != IPS4O_OK) return rc;
    }
    if (written) {
        // the result is already in the host buffer
    } else if (by_kernel && kernel_copy(h_dev, st->d_host_copy, bytes, s, st->sms, &e)) {
        if (e != cudaSuccess) { set_last_cuda_error(e, "copy kernel (D2H)"); return IPS4O_ERR_CUDA; }
    } else {
        e = cudaMemcpyAsync(h_ptr, st->d_host_copy, bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) { set_last_cuda_error(e, "cudaMemcpyAsync(D2H)"); return IPS4O_ERR_CUDA; }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaStreamSynchronize"); return IPS4O_ERR_CUDA; }
    return finalize_pending(*st);
}

ips4o_status ips4o_partition(void* d_ptr, size_t n, int key_type, void* stream, uint64_t* h_bounds,
                             size_t* num_buckets, uint64_t* h_splitters, size_t* num_splitters, int* eq) {
    ips4o_status rc = check_args(d_ptr, n, key_type);
    if (rc != IPS4O_OK) return rc;
    if (n < 2 || !h_bounds || !num_buckets || !h_splitters || !num_splitters || !eq) return IPS4O_ERR_INVALID_ARG;
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    PartitionOut out{h_bounds, num_buckets, h_splitters, num_splitters, eq};
    return dispatch(*st, d_ptr, n, key_type, (cudaStream_t)stream, &out);
}

size_t ips4o_workspace_bytes(size_t n, int key_type) {
    int sms = 152;
    cudaError_t e;
    DeviceState* st = current_device_state(&e);
    if (st) sms = st->sms;
    else cudaGetLastError();
    switch (key_type) {
    case IPS4O_U64: return workspace_bytes_u64(n, sms);
    case IPS4O_F64: return workspace_bytes_f64(n, sms);
    case IPS4O_PAIR_U64: return workspace_bytes_pair(n, sms);
    case IPS4O_QUARTET_U64: return workspace_bytes_quartet(n, sms);
    case IPS4O_REC100_K10: return workspace_bytes_pair(n, sms) + rec100_aux_bytes(n);
    default: return 0;
    }
}

ips4o_status ips4o_reserve_workspace(size_t n, size_t num_segments, int key_type, void* stream) {
    if (key_type < 0 || key_type > IPS4O_QUARTET_U64 || elem_size(key_type) == 0) return IPS4O_ERR_UNSUPPORTED_TYPE;
    cudaError_t e;
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    switch (key_type) {
    case IPS4O_U64: return reserve_u64(*st, n, num_segments);
    case IPS4O_F64: return reserve_f64(*st, n, num_segments);
    case IPS4O_PAIR_U64: return reserve_pair(*st, n, num_segments);
    case IPS4O_QUARTET_U64: return reserve_quartet(*st, n, num_segments);
    default: {
        ips4o_status rc = reserve_pair(*st, n, num_segments);
        return rc != IPS4O_OK ? rc : ensure_device_buffer(&st->d_aux, &st->aux_bytes, rec100_aux_bytes(n));
    }
    }
}

ips4o_status ips4o_release_workspace(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::vector<DeviceState*> mine;
    {
        std::lock_guard<std::mutex> lk(g_mtx);
        for (auto& kv : g_states)
            if (kv.first.first == dev) mine.push_back(kv.second);
    }
    for (DeviceState* st : mine) {
        std::lock_guard<std::mutex> lk(st->mtx);
        if (st->d_ws) cudaFree(st->d_ws);
        if (st->d_host_copy) cudaFree(st->d_host_copy);
        if (st->d_aux) cudaFree(st->d_aux);
        if (st->h_stage) cudaFreeHost(st->h_stage);
        for (cudaEvent_t ev : st->events) cudaEventDestroy(ev);
        st->events.clear();
        st->d_ws = st->d_host_copy = st->d_aux = st->h_stage = nullptr;
        st->d_status = nullptr;
        for (int k = 0; k < 5; ++k) st->reserved_n[k] = st->reserved_segments[k] = 0;
        st->ws_bytes = st->d_host_copy_bytes = st->aux_bytes = st->h_stage_bytes = 0;
    }
    return IPS4O_OK;
}

ips4o_status ips4o_set_params(const ips4o_params* p) {
    std::lock_guard<std::mutex> lk(g_mtx);
    if (!p) {
        g_params = kDefaultParams;
        return IPS4O_OK;
    }
    if (p->k_max < 4 || p->k_max > 256 || (p->k_max & (p->k_max - 1)) != 0) return IPS4O_ERR_INVALID_ARG;
    if (p->stripes_per_sm < 1 || p->stripes_per_sm > 16) return IPS4O_ERR_INVALID_ARG;
    if (p->alpha > 4095) return IPS4O_ERR_INVALID_ARG;
    if (p->segment_scheduler < 0 || p->segment_scheduler > 2) return IPS4O_ERR_INVALID_ARG;
    if (p->record_path < 0 || p->record_path > 1) return IPS4O_ERR_INVALID_ARG;
    g_params = *p;
    return IPS4O_OK;
}

ips4o_status ips4o_set_class_params(const ips4o_class_params* table, size_t count) {
    if (count > IPS4O_NUM_CLASSES || (count > 0 && !table)) return IPS4O_ERR_INVALID_ARG;
    ips4o_class_params t[IPS4O_NUM_CLASSES] = {};
    for (size_t c = 0; table && c < count; ++c) {
        const unsigned L = table[c].leaves, a = table[c].alpha;
        if (L && (L < 4 || L > 256 || (L & (L - 1)))) return IPS4O_ERR_INVALID_ARG;
        if (a && L && a * L > 4096) return IPS4O_ERR_INVALID_ARG;
        t[c] = table[c];
    }
    {
        std::lock_guard<std::mutex> lk(g_mtx);
        std::memcpy(g_classes, t, sizeof t);
    }
    ips4o_status rc = upload_class_table_u64(t);
    if (rc == IPS4O_OK) rc = upload_class_table_f64(t);
    if (rc == IPS4O_OK) rc = upload_class_table_pair(t);
    if (rc == IPS4O_OK) rc = upload_class_table_quartet(t);
    return rc;
}

ips4o_status ips4o_get_class_params(ips4o_class_params* out, size_t count) {
    if (!out || count > IPS4O_NUM_CLASSES) return IPS4O_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mtx);
    std::memcpy(out, g_classes, count * sizeof(ips4o_class_params));
    return IPS4O_OK;
}

ips4o_status ips4o_get_params(ips4o_params* out) {
    if (!out) return IPS4O_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mtx);
    *out = g_params;
    return IPS4O_OK;
}

ips4o_status ips4o_get_stats(ips4o_stats* out) {
    if (!out) return IPS4O_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    if (dev < 0 || dev >= 64) return IPS4O_ERR_INVALID_ARG;
    DeviceState* last = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mtx);
        last = g_last_state[dev];
    }
    if (last) {
        // an asynchronous call's counters are completed here (waits for its stream)
        std::lock_guard<std::mutex> lk(last->mtx);
        finalize_pending(*last);
    }
    std::lock_guard<std::mutex> lk(g_mtx);
    *out = g_last_stats[dev];
    return IPS4O_OK;
}

size_t ips4o_base_case_capacity(int key_type) {
    switch (key_type) {
    case IPS4O_U64: return TU64::kBaseCap;
    case IPS4O_F64: return TF64::kBaseCap;
    case IPS4O_PAIR_U64: return TPair::kBaseCap;
    case IPS4O_QUARTET_U64: return TQuartet::kBaseCap;
    default: return 0;
    }
}

const char* ips4o_status_string(int s) {
    switch (s) {
    case IPS4O_OK: return "ok";
    case IPS4O_ERR_INVALID_ARG: return "invalid argument";
    case IPS4O_ERR_UNSUPPORTED_TYPE: return "unsupported key type";
    case IPS4O_ERR_MISALIGNED: return "pointer not aligned for the key type";
    case IPS4O_ERR_OOM: return "out of memory";
    case IPS4O_ERR_CUDA: return "CUDA error";
    case IPS4O_ERR_TIMEOUT: return "bounded device wait timed out";
    case IPS4O_ERR_INTERNAL: return "internal invariant violated";
    case IPS4O_ERR_TOO_LARGE: return "request exceeds a fixed capacity";
    default: return "unknown status";
    }
}

const char* ips4o_last_cuda_error(void) { return g_last_err; }

ips4o_status ips4o_check_bounded_wait(uint32_t spin_limit, void* stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_probe);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGetSymbolAddress"); return IPS4O_ERR_CUDA; }
    unsigned* words = (unsigned*)p;                 // [0] the flag nothing sets, [1] the status
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32, 0, s>>>(words, spin_limit);
        e = cudaGetLastError();
    }
    unsigned status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, words + 1, sizeof status, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_last_cuda_error(e, "ips4o_check_bounded_wait"); return IPS4O_ERR_CUDA; }
    if (status & kStatusTimeout) return IPS4O_ERR_TIMEOUT;
    return status ? IPS4O_ERR_INTERNAL : IPS4O_OK;
}

ips4o_status ips4o_stream_status(void* stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_cuda_error(e, "ips4o_stream_status"); return IPS4O_ERR_CUDA; }
    DeviceState* st = stream_state(stream, &e);
    if (!st) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    std::lock_guard<std::mutex> lk(st->mtx);
    if (st->pending) return finalize_pending(*st);
    if (!st->d_status) return IPS4O_OK;
    unsigned bits = 0;
    e = cudaMemcpy(&bits, st->d_status, sizeof bits, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_last_cuda_error(e, "ips4o_stream_status"); return IPS4O_ERR_CUDA; }
    if (bits & 1u) return IPS4O_ERR_TIMEOUT;
    if (bits) return IPS4O_ERR_INTERNAL;
    return IPS4O_OK;
}

}  // extern "C"
