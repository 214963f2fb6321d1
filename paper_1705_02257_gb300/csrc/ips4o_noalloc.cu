// ips4o_noalloc.cu — ips4o_sort_noalloc: the sort for callers that must not
// allocate memory.
//
// Some callers cannot call cudaMalloc at the time they sort: code running
// while a stream is being captured into a CUDA graph (allocation is not
// allowed there), memory-budgeted services that must not grow the device
// footprint after start-up, or plug-ins whose host process owns all device
// allocations.  For them this entry point sorts arrays of up to
// kNoAllocMaxN elements using a fixed scratch area that is part of the
// library image: a file-scope __device__ array (kNoAllocScratchBytes, held on
// every GPU that loads the library until the process exits) and a static
// host staging buffer.  It calls no cudaMalloc, cudaMallocHost, cudaFree or
// other allocating routine.
//
// The scratch array is shared by every call: calls that overlap on the GPU
// (different streams, or different host threads) would race on it, so the
// host side serialises calls with a mutex and each call waits for its own
// work before returning.  Counters that must start at zero are cleared by
// every call; every other part of the scratch is written before it is read.
#include <cstring>
#include <mutex>

#include "ips4o_driver.cuh"

namespace ips4o {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // device scratch, 16 MiB
constexpr size_t kNoAllocHostBytes = (size_t)1 << 20;       // host staging, 1 MiB
constexpr size_t kNoAllocMaxN = (size_t)1 << 20;            // largest array, in elements
constexpr size_t kNoAllocMaxTasks = 256;                    // subproblems per level (n / 16Ki << 256)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
alignas(256) static unsigned char g_noalloc_host[kNoAllocHostBytes];
static Task g_noalloc_tasks[2][kNoAllocMaxTasks];
static std::mutex g_noalloc_mtx;
static DeviceState g_noalloc_state[64];
static bool g_noalloc_ready[64];

// The library defaults: the scratch is sized for them, so user parameters
// (e.g. a smaller base case, which creates more subproblems) do not apply.
static const ips4o_params kNoAllocParams = {256, 0, 0, 2, 0, 0x2545F4914F6CDD1Dull};

template <class T>
struct NoAllocDriver : Driver<T> {
    typedef typename T::elem_t E;
    using Driver<T>::st;
    using Driver<T>::prm;
    using Driver<T>::caps;
    using Driver<T>::h_subs;
    using Driver<T>::h_stripes;
    using Driver<T>::h_tasks;
    using Driver<T>::ws;
    using Driver<T>::base_cap;
    using Driver<T>::k_max;
    using Driver<T>::rec_cap;
    using Driver<T>::stream;

    NoAllocDriver(DeviceState& s, cudaStream_t strm) : Driver<T>(s, strm, kNoAllocParams) {}

    // One chunk of the level's subproblems (same plan as the allocating path,
    // over a plain array of tasks).
    size_t plan(const Task* tasks, size_t count, size_t i0, u64 level_total, u32 level, u32* nsub_out,
                u32* nstripes_out) {
        const u64 B = T::kBlock;
        const u64 target = (u64)std::max(1, prm.stripes_per_sm) * (u64)st.sms;
        u64 stripe_len = std::max<u64>((level_total + target - 1) / target, kMinStripe);
        stripe_len = (stripe_len + B - 1) / B * B;
        u32 nsub = 0, nstr = 0;
        u64 pool = 0;
        size_t i = i0;
        for (; i < count; ++i) {
            const Task t = tasks[i];
            if (nsub >= caps.max_sub) break;
            const u32 K = leaves_for(t.n, base_cap, k_max);
            u32 alpha = prm.alpha > 0 ? (u32)prm.alpha : (u32)kDefaultAlpha;
            alpha = std::max<u32>(1, std::min<u32>(alpha, 4096 / K));
            u64 ns = std::max<u64>(1, (t.n + stripe_len - 1) / stripe_len);
            ns = std::min<u64>(ns, kMaxStripesPerSub);
            u64 slen, need;
            for (;;) {
                slen = ((t.n + ns - 1) / ns + B - 1) / B * B;
                ns = (t.n + slen - 1) / slen;
                need = 0;
                for (u64 q = 0; q < ns; ++q) need += std::min<u64>((u64)kMaxBuckets * (B - 1), std::min<u64>(slen, t.n - q * slen));
                const bool fits = nstr + ns <= caps.max_stripes && pool + need <= caps.pool_cap;
                if (fits || ns == 1 || nsub > 0) break;
                ns = std::max<u64>(1, ns / 2);
            }
            if (nstr + ns > caps.max_stripes || pool + need > caps.pool_cap) break;
            SubDesc& sd = h_subs[nsub];
            std::memset(&sd, 0, sizeof sd);
            sd.begin = t.begin;
            sd.n = t.n;
            sd.stripe_begin = nstr;
            sd.num_stripes = (u32)ns;
            sd.k_target = K;
            sd.alpha = alpha;
            sd.level = level;
            for (u64 q = 0; q < ns; ++q) {
                StripeDesc& x = h_stripes[nstr + q];
                x.begin = t.begin + q * slen;
                x.end = t.begin + std::min<u64>((q + 1) * slen, t.n);
                x.pool_off = pool;
                x.pool_cap = (u32)std::min<u64>((u64)kMaxBuckets * (B - 1), x.end - x.begin);
                x.sub = nsub;
                pool += x.pool_cap;
            }
            nstr += (u32)ns;
            ++nsub;
        }
        *nsub_out = nsub;
        *nstripes_out = nstr;
        return i - i0;
    }

    ips4o_status run(E* d, u64 n) {
        // the scratch must hold this sort's workspace: refuse rather than
        // letting the workspace helpers replace it with an allocation
        const Caps<T> c = caps_for<T>(n, st.sms, prm.stripes_per_sm, recursion_cap<T>(prm));
        if (carve<T>(c, nullptr, nullptr) > st.ws_bytes || host_stage_bytes<T>(c) > st.h_stage_bytes)
            return IPS4O_ERR_TOO_LARGE;
        ips4o_status rc = this->setup(n);
        if (rc != IPS4O_OK) return rc;
        st.stats.n = n;
        if (n <= (u64)rec_cap) return this->base_only(d, n);
        Task* cur = g_noalloc_tasks[0];
        Task* nxt = g_noalloc_tasks[1];
        size_t ncur = 1;
        cur[0] = Task{0, n};
        u32 level = 0;
        while (ncur > 0) {
            size_t nnext = 0;
            u64 level_total = 0;
            for (size_t q = 0; q < ncur; ++q) level_total += cur[q].n;
            size_t i = 0;
            while (i < ncur) {
                u32 nsub = 0, nstr = 0;
                const size_t taken = plan(cur, ncur, i, level_total, level, &nsub, &nstr);
                if (taken == 0) return IPS4O_ERR_INTERNAL;
                u32 cnt = 0;
                rc = this->run_chunk(d, nsub, nstr, false, &cnt);
                if (rc != IPS4O_OK) return rc;
                if (cnt > 0) {
                    if (cnt > caps.next_cap || nnext + cnt > kNoAllocMaxTasks) return IPS4O_ERR_TOO_LARGE;
                    IPS4O_CUDA(cudaMemcpyAsync(h_tasks, ws.next_tasks, cnt * sizeof(Task), cudaMemcpyDeviceToHost,
                                               stream));
                    IPS4O_CUDA(cudaStreamSynchronize(stream));
                    for (u32 q = 0; q < cnt; ++q) nxt[nnext + q] = h_tasks[q];
                    nnext += cnt;
                }
                i += taken;
            }
            ++level;
            st.stats.levels = level;
            Task* t = cur;
            cur = nxt;
            nxt = t;
            ncur = nnext;
            if (level > 64) return IPS4O_ERR_INTERNAL;
        }
        return IPS4O_OK;
    }
};

template <class T>
static ips4o_status noalloc_sort_t(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    NoAllocDriver<T> drv(st, s);
    return drv.run((typename T::elem_t*)d, (u64)n);
}

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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
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
    switch (key_type) {
    case IPS4O_U64: return noalloc_sort_t<TU64>(st, d_ptr, n, s);
    case IPS4O_F64: return noalloc_sort_t<TF64>(st, d_ptr, n, s);
    default: return noalloc_sort_t<TPair>(st, d_ptr, n, s);
    }
}
