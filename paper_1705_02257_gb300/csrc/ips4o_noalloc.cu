// ips4o_noalloc.cu — ips4o_sort_noalloc: the sort for callers that must not
// allocate memory.
//
// Some callers cannot call cudaMalloc when they sort: memory-budgeted
// services whose device footprint is fixed at start-up (a later allocation
// could fail or push out other tenants), or plug-ins whose host process owns
// every device allocation.  For them this entry point sorts arrays of up to
// kNoAllocMaxN elements in a fixed scratch area that is part of the library
// image: a file-scope __device__ array (kNoAllocScratchBytes, held on every
// GPU that loads the library until the process exits) and a static host
// staging buffer.  It calls no cudaMalloc, cudaMallocHost, cudaFree or other
// allocating routine; a sort whose workspace would not fit the scratch is
// refused with IPS4O_ERR_TOO_LARGE before any work is queued.
//
// The call still synchronises its stream once per recursion level (the
// next level is planned on the host), so it cannot run while the stream is
// being captured into a CUDA graph: it checks that first and returns
// IPS4O_ERR_INVALID_ARG without touching the stream.
//
// The scratch array is shared by every call: calls that overlap on the GPU
// (different streams, or different host threads) would race on it, so the
// host side serialises calls with a mutex and each call waits for its own
// work before returning.  Counters that must start at zero are cleared by
// every call; every other part of the scratch is written before it is read.
#include <cstring>
#include <mutex>

#include "ips4o_common.cuh"
#include "ips4o_host.h"

namespace ips4o {

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
alignas(256) static unsigned char g_noalloc_host[kNoAllocHostBytes];
static Task g_noalloc_tasks[2][kNoAllocMaxTasks];
static std::mutex g_noalloc_mtx;
static DeviceState g_noalloc_state[64];
static bool g_noalloc_ready[64];

}  // namespace ips4o

using namespace ips4o;

extern "C" ips4o_status ips4o_sort_noalloc(void* d_ptr, size_t n, int key_type, void* stream) {
    size_t es;
    switch (key_type) {
    case IPS4O_U64: case IPS4O_F64: es = 8; break;
    case IPS4O_PAIR_U64: es = 16; break;
    default: return IPS4O_ERR_UNSUPPORTED_TYPE;
    }
    if (n > kNoAllocMaxN) {
        set_last_message("ips4o_sort_noalloc: more elements than its fixed scratch supports (2^20)");
        return IPS4O_ERR_TOO_LARGE;
    }
    if (n > 1 && !d_ptr) return IPS4O_ERR_INVALID_ARG;
    if (d_ptr && ((uintptr_t)d_ptr % es) != 0) return IPS4O_ERR_MISALIGNED;
    if (n < 2) return IPS4O_OK;
    // the level loop synchronises the stream: refuse a stream under capture
    // before anything is queued on it (the capture stays valid)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        if (e != cudaSuccess) cudaGetLastError();
        set_last_message("ips4o_sort_noalloc: the stream is being captured; the call synchronises per level");
        return IPS4O_ERR_INVALID_ARG;
    }
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGetDevice"); return IPS4O_ERR_CUDA; }
    if (dev < 0 || dev >= 64) return IPS4O_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mtx);
    DeviceState& st = g_noalloc_state[dev];
    if (!g_noalloc_ready[dev]) {
        // once per device, with that device current: the device address of
        // the scratch array (its name in host code is only a stand-in)
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGetSymbolAddress"); return IPS4O_ERR_CUDA; }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) { set_last_cuda_error(e, "cudaDeviceGetAttribute"); return IPS4O_ERR_CUDA; }
        st.device = dev;
        st.sms = sms;
        st.d_ws = ptr;
        st.ws_bytes = kNoAllocScratchBytes;
        st.h_stage = g_noalloc_host;
        st.h_stage_bytes = kNoAllocHostBytes;
        g_noalloc_ready[dev] = true;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Task* tasks = &g_noalloc_tasks[0][0];
    switch (key_type) {
    case IPS4O_U64: return sort_noalloc_u64(st, d_ptr, n, s, tasks);
    case IPS4O_F64: return sort_noalloc_f64(st, d_ptr, n, s, tasks);
    default: return sort_noalloc_pair(st, d_ptr, n, s, tasks);
    }
}
