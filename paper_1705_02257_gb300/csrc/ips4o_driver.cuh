// ips4o_driver.cuh — host driver of the recursion (Section 4: "As long as
// problems with at least beta*n/t elements exist, we partition those ...").
//
// The driver keeps the list of subproblems of the current recursion level on
// the host.  A level is processed in chunks (groups of subproblems whose
// state fits the workspace); each chunk is one launch of the six
// distribution-step kernels on the caller's stream, after which the buckets
// larger than the base case come back as the next level's subproblems and
// the others have already been sorted in shared memory by the cleanup kernel.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "ips4o_host.h"
#include "ips4o_kernels.cuh"
#include "ips4o_strict.cuh"

namespace ips4o {

constexpr u32 kSpinLimit = 1u << 22;     // bounded waits: ~0.3 s with the sleeps
constexpr int kDefaultAlpha = 16;
// Device-planned sorts: the partial buffers of at most this many stripes per
// SM are held at once (the leftover pool, Theorem 2's O(k b t) with t a
// multiple of the SM count, independent of n), and at most this many
// subproblems form one round's chunk.
constexpr u64 kRoundStripesPerSm = 2;
constexpr u32 kRoundMaxSub = 1024;

inline u32 pow2_ceil_host(u64 x) {
    u32 p = 1;
    while (p < x && p < (1u << 30)) p <<= 1;
    return p;
}

template <class T>
struct Caps {
    u32 max_sub, max_stripes;
    u64 pool_cap, next_cap;
    u64 init_cap;       // segments that go straight to the base case (segmented calls)
    u64 stack_cap;      // segment scheduler: buckets per CTA stack (0 = not used)
    u32 stack_slots = 0;   // segment scheduler: CTA stacks
    bool rounds = false;   // device-planned levels: a second task queue and the loop state
    u64 scan_cap = 0;      // strict recursion: tiles of one scan window
    u64 copy_cap = 0;      // result written to another buffer: ranges the final copy moves
};


constexpr u64 kSegStackCap = 2048;     // per CTA; a distribution step pushes at most 256 buckets

// Workspace of the segment scheduler (one slot per CTA of its persistent grid).
template <class T>
Caps<T> caps_for_scheduler(int sms, u64 num_segments) {
    Caps<T> c;
    c.max_sub = (u32)sms;
    c.max_stripes = (u32)sms;
    c.pool_cap = (u64)sms * kMaxBuckets * (T::kBlock - 1);
    c.next_cap = 16;
    c.init_cap = num_segments;
    c.stack_cap = kSegStackCap;
    c.stack_slots = (u32)sms;
    return c;
}

// Base-case threshold in effect: buckets larger than this recurse.
template <class T>
u32 recursion_cap(const ips4o_params& p) {
    u32 rc = (u32)T::kBaseCap;
    if (p.base_case_max > 0) rc = std::min(rc, (u32)std::max(p.base_case_max, 16));
    return rc;
}

template <class T>
Caps<T> caps_for(u64 n, int sms, int stripes_per_sm, u64 cap) {
    const u64 B = T::kBlock;
    Caps<T> c;
    u64 target = (u64)std::max(1, stripes_per_sm) * (u64)std::max(1, sms);
    c.max_sub = (u32)std::min<u64>(1024, n / (cap + 1) + 1);
    c.max_stripes = (u32)std::min<u64>(4096, target + c.max_sub + 1);
    target = std::min<u64>(target, n / kMinStripe + 1);   // stripes are at least kMinStripe long
    // partial buffers: the stripes of a lower level round up per subproblem,
    // so room for 1.5 times the target number of stripes keeps a level in
    // one chunk (Theorem 2: O(k b t) extra space)
    u64 pool = std::max<u64>(n / 16, 3 * target * kMaxBuckets * (B - 1) / 2);
    pool = std::min<u64>(pool, n + kMaxBuckets * B);
    // a chunk never holds more leftovers than its stripes' buffers
    pool = std::min<u64>(pool, (u64)c.max_stripes * kMaxBuckets * (B - 1));
    c.pool_cap = std::max<u64>(pool, (u64)kMaxBuckets * B);
    c.next_cap = n / (cap + 1) + 16;
    c.init_cap = 0;
    c.stack_cap = 0;
    return c;
}

// Workspace of a device-planned sort of n elements: a leftover pool for
// kRoundStripesPerSm stripes per SM (or the whole input, when smaller), at
// most kRoundMaxSub subproblems per round, two level queues for every
// subproblem a level can have (n / (threshold + 1)), and the segment
// scheduler's per-CTA areas for subproblems left after the last round.
template <class T>
Caps<T> caps_for_rounds(u64 n, int sms, u64 cap, bool copy_out = false) {
    const u64 B = T::kBlock, per = (u64)kMaxBuckets * (B - 1);
    Caps<T> c;
    const u64 stripes = kRoundStripesPerSm * (u64)std::max(1, sms);
    c.max_sub = (u32)std::min<u64>(kRoundMaxSub, n / (cap + 1) + 1);
    c.max_stripes = (u32)std::min<u64>(4096, std::max<u64>(stripes, c.max_sub));
    c.pool_cap = std::min<u64>(stripes * per, n + (u64)kMaxBuckets * B);
    c.pool_cap = std::max<u64>(c.pool_cap, per);
    c.next_cap = n / (cap + 1) + 16;
    c.init_cap = 2 * c.next_cap;
    c.stack_cap = kSegStackCap;
    // the segment scheduler's CTAs each take one subproblem slot, stripe
    // slot, pool area and stack
    c.stack_slots = (u32)std::max<u64>(1, std::min<u64>({(u64)std::max(1, sms), (u64)c.max_sub,
                                                            (u64)c.max_stripes, c.pool_cap / per}));
    c.rounds = true;
    // a result written to another buffer: the buckets the base case does not
    // write (equality buckets, single elements: at most one chunk's buckets
    // per round) and the segment scheduler's subproblems, in chunks of at
    // most kCopyChunk elements
    if (copy_out) c.copy_cap = (u64)c.max_sub * kMaxBuckets + c.init_cap + n / kCopyChunk + 64;
    return c;
}

// Workspace of the enqueue-only segmented sort planned on the device: the
// rounds' tables and queues, a list for every segment, and the leftover pool
// of the level-by-level host driver (many segments above the base case each
// take at least one stripe and its pool area, so a larger pool keeps the
// first level in fewer chunks).
template <class T>
Caps<T> caps_for_segment_rounds(u64 n, int sms, u64 cap, u64 num_segments) {
    Caps<T> c = caps_for_rounds<T>(n, sms, cap);
    const Caps<T> h = caps_for<T>(n, sms, 1, cap);
    c.init_cap = std::max<u64>(c.init_cap, num_segments);
    c.pool_cap = std::max<u64>(c.pool_cap, h.pool_cap);
    c.max_stripes = std::max<u32>(c.max_stripes, h.max_stripes);
    return c;
}

// Elements of one window of the strict recursion's scan: about 1 GiB, a
// whole number of scan tiles; params.strict_window overrides it.
template <class T>
u64 strict_window(const ips4o_params& p) {
    typedef typename T::elem_t E;
    u64 w = p.strict_window ? (u64)p.strict_window : kScanWindowBytes / sizeof(E);
    w = std::max<u64>(kScanTile, w / kScanTile * kScanTile);
    return w;
}

// Workspace of the strict recursion: the rounds' (whose chunk limits do not
// depend on n) with a subproblem list for one window and the scan tiles;
// no level queues and no segment scheduler, so nothing grows with n.
template <class T>
Caps<T> caps_for_strict(u64 n, int sms, u64 cap, u64 window) {
    Caps<T> c = caps_for_rounds<T>(std::min<u64>(n, window), sms, cap);
    c.next_cap = window / (cap + 1) + 64;
    c.init_cap = 0;
    c.stack_cap = 0;
    c.stack_slots = 0;
    c.scan_cap = (window + kScanTile - 1) / kScanTile;
    return c;
}

// CTAs of the segment scheduler that finishes a device-planned sort.
template <class T>
u32 fallback_grid(const Caps<T>& c) {
    return c.stack_slots;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Workspace carving: returns total bytes; fills ws when base != nullptr.
template <class T>
size_t carve(const Caps<T>& c, char* base, Workspace<T>* ws) {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = align_up(off, 256);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const u64 S = c.max_sub, R = c.max_stripes;
    Workspace<T> w;
    w.subs = (SubDesc*)take(S * sizeof(SubDesc));
    w.stripes = (StripeDesc*)take(R * sizeof(StripeDesc));
    w.tree = (K*)take(S * kMaxLeaves * sizeof(K));
    w.spl = (K*)take(S * kMaxLeaves * sizeof(K));
    w.bstart = (u64*)take(S * (kMaxBuckets + 1) * 8);
    w.delim = (u32*)take(S * (kMaxBuckets + 1) * 4);
    w.wr = (u64*)take(S * kMaxBuckets * 8);
    w.flags = (u32*)take(S * kMaxBuckets * 4);
    w.exhausted = (u32*)take(S * 8 * 4);
    w.movers = (u32*)take(S * 4);
    w.region_full = (u32*)take(S * kMaxBuckets * 4);
    w.bucket_full = (u32*)take(S * kMaxBuckets * 4);
    w.counts = (u32*)take(R * kMaxBuckets * 4);
    w.lscan = (u32*)take(R * kMaxBuckets * 4);
    w.stripe_full = (u32*)take(R * 4);
    w.fix_list = (FixItem*)take(S * kMaxBuckets * sizeof(FixItem));
    w.pool = (E*)take(c.pool_cap * sizeof(E));
    w.overflow = (E*)take(S * T::kBlock * sizeof(E));
    w.next_tasks = (Task*)take(c.next_cap * sizeof(Task));
    w.base_small = (Task*)take(S * kMaxBuckets * sizeof(Task));
    w.base_tiny = (Task*)take(S * kMaxBuckets * sizeof(Task));
    w.base_large = (Task*)take(S * kMaxBuckets * sizeof(Task));
    w.init_tasks = (Task*)take(c.init_cap * sizeof(Task));
    w.init_count = (u32*)take(4 * sizeof(u32));
    w.hist = (u32*)take(65 * sizeof(u32));
    w.stacks = (Task*)take((u64)c.stack_slots * c.stack_cap * sizeof(Task));
    w.ctr = (ChunkCounters*)take(sizeof(ChunkCounters));
    w.next_tasks2 = c.rounds ? (Task*)take(c.next_cap * sizeof(Task)) : nullptr;
    w.ls = c.rounds ? (LoopState*)take(sizeof(LoopState)) : nullptr;
    w.stripe_order = c.rounds ? (u32*)take(R * sizeof(u32)) : nullptr;
    w.copy_tasks = c.copy_cap ? (Task*)take(c.copy_cap * sizeof(Task)) : nullptr;
    w.out = nullptr;
    w.scan_max = c.scan_cap ? (K*)take(c.scan_cap * sizeof(K)) : nullptr;
    w.scan_tiles = c.scan_cap ? (ScanTile*)take(c.scan_cap * sizeof(ScanTile)) : nullptr;
    if (!base) {
        w.next_tasks2 = nullptr;
        w.ls = nullptr;
    }
    w.max_sub = c.max_sub;
    w.max_stripes = c.max_stripes;
    w.pool_cap = c.pool_cap;
    w.next_cap = c.next_cap;
    w.init_cap = c.init_cap;
    w.stack_cap = c.stack_cap;
    w.scan_cap = c.scan_cap;
    w.copy_cap = c.copy_cap;
    if (ws) *ws = w;
    return align_up(off, 256);
}

// Pinned host staging: SubDesc[max_sub] + StripeDesc[max_stripes] +
// ChunkCounters + Task[next_cap].
template <class T>
size_t host_stage_bytes(const Caps<T>& c) {
    return align_up(c.max_sub * sizeof(SubDesc), 256) + align_up(c.max_stripes * sizeof(StripeDesc), 256) +
           align_up(sizeof(ChunkCounters), 256) + align_up(c.next_cap * sizeof(Task), 256);
}

template <class T>
size_t workspace_bytes_t(size_t n, int sms) {
    return carve<T>(caps_for_rounds<T>(n, sms, recursion_cap<T>(global_params())), nullptr, nullptr);
}

// Number of leaves for a subproblem of n elements (Section 4.7, adaptive
// number of buckets on the last levels).  r = 2n/T is the reduction that
// brings the average bucket to half the base-case capacity T.  One step
// with pow2(r) leaves when r <= k_max; still one step with k_max leaves when
// r <= 2*k_max (average bucket <= T; the few larger buckets take one more
// step); two balanced steps of about sqrt(r) leaves when r <= k_max^2; and
// k_max otherwise.
inline u32 leaves_for(u64 n, u64 base_cap, u32 k_max) {
    const double r = 2.0 * (double)n / (double)base_cap;
    u32 k;
    if (r <= (double)k_max) k = pow2_ceil_host((u64)std::ceil(r));
    else if (r <= 2.0 * (double)k_max) k = k_max;
    else if (r <= (double)k_max * (double)k_max) k = pow2_ceil_host((u64)std::ceil(std::sqrt(r)));
    else k = k_max;
    return std::min(std::max<u32>(k, 4), k_max);
}

// Rounds enqueued for a device-planned sort of n elements.  The recursion
// is followed on nominal sizes: a level of `subs` subproblems of m elements
// takes ceil(subs / max_sub) rounds and splits each into the number of
// leaves the planner gives that size (the class table, else leaves_for),
// down to the recursion threshold.  When the last level's nominal buckets
// come within a factor of 4 of the threshold, sampling may leave some above
// it, and one more round is added; two more rounds per nominal level (at
// most four) take levels with more subproblems than nominal and levels more
// than nominal (skewed keys, such as Exponential's); an empty round costs a
// few microseconds of launches.  Rarer stragglers, and any deeper recursion,
// go to the segment scheduler after the last round.
inline u32 rounds_for(u64 n, u64 cap, u64 base_cap, u32 k_max, u32 max_sub) {
    double subs = 1.0, m = (double)n;
    u32 r = 0, levels = 0;
    while (m > (double)cap && r < 4096) {
        ++levels;
        r += (u32)std::ceil(subs / (double)max_sub);
        const ips4o_class_params cp = class_table()[63 - __builtin_clzll((u64)m)];
        const u32 K = cp.leaves ? (u32)cp.leaves : leaves_for((u64)m, base_cap, k_max);
        subs *= K;
        m /= K;
    }
    return r + std::min<u32>(2 * levels, 4) + (m * 4.0 > (double)cap ? 1u : 0u);
}

#define IPS4O_CUDA(call)                                    \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            set_last_cuda_error(e_, #call);                 \
            return IPS4O_ERR_CUDA;                          \
        }                                                   \
    } while (0)

template <class T>
ips4o_status set_kernel_attributes(DeviceState& st) {
    IPS4O_CUDA(cudaFuncSetAttribute(k_classify<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ClassifyRegCfg<T>::smem_bytes));
    IPS4O_CUDA(cudaFuncSetAttribute(k_cleanup<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)CleanupCfg<T>::smem_bytes));
    IPS4O_CUDA(cudaFuncSetAttribute(k_cleanup_cta<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)CleanupCtaCfg<T>::smem_bytes));
    IPS4O_CUDA(cudaFuncSetAttribute(k_base<T, BaseTiny<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)BaseTiny<T>::smem_bytes));
    IPS4O_CUDA(cudaFuncSetAttribute(k_base<T, BaseSmall<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)BaseSmall<T>::smem_bytes));
    IPS4O_CUDA(cudaFuncSetAttribute(k_base<T, BaseLarge<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)BaseLarge<T>::smem_bytes));
    IPS4O_CUDA(cudaFuncSetAttribute(k_permute<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PermuteCfg<T>::smem_bytes));
    if constexpr (!std::is_same<T, TRec>::value)   // 100-byte records: host-planned levels only
        IPS4O_CUDA(cudaFuncSetAttribute(k_segments<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SegCfg<T>::smem_bytes));
    int occ = 0;
    IPS4O_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_permute<T>, PermuteCfg<T>::TPB,
                                                             PermuteCfg<T>::smem_bytes));
    st.permute_grid[T::kId] = std::max(1, occ) * st.sms;
    st.attrs_ready[T::kId] = true;
    return IPS4O_OK;
}

template <class T>
struct Driver {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;

    DeviceState& st;
    cudaStream_t stream;
    const ips4o_params prm;
    Workspace<T> ws;
    Caps<T> caps;
    SubDesc* h_subs;
    StripeDesc* h_stripes;
    ChunkCounters* h_ctr;
    Task* h_tasks;
    u32 base_cap;       // buckets average about half of this after the last step
    u32 rec_cap;        // buckets larger than this recurse; smaller go to the base case
    u32 k_max;
    int permute_grid = 0;
    u64 level_stripe_len = 0;   // stripe length of the level being planned

    Driver(DeviceState& s, cudaStream_t strm) : st(s), stream(strm), prm(global_params()) {}
    Driver(DeviceState& s, cudaStream_t strm, const ips4o_params& p) : st(s), stream(strm), prm(p) {}

    // How setup treats the buffers of the stream state:
    //   kGrow     grow the workspace and host staging as needed (may allocate);
    //   kEnqueue  use the reserved workspace, no host staging (enqueue-only calls);
    //   kFixed    use the given workspace and host staging as they are: never
    //             allocates or frees, TOO_LARGE when either is too small.
    enum WsMode { kGrow, kEnqueue, kFixed };

    ips4o_status setup(u64 n, u64 init_cap = 0, const Caps<T>* override_caps = nullptr, WsMode mode = kGrow) {
        cudaGetLastError();   // an error left by an earlier, unrelated runtime call is not this call's
        st.d_status = nullptr;  // the workspace layout changes: an earlier status word is gone
        if (override_caps) {
            caps = *override_caps;
        } else {
            caps = caps_for<T>(n, st.sms, prm.stripes_per_sm, recursion_cap<T>(prm));
            caps.init_cap = init_cap;
        }
        const size_t need = carve<T>(caps, nullptr, nullptr);
        ips4o_status rc = IPS4O_OK;
        if (mode == kGrow) rc = ensure_device_buffer(&st.d_ws, &st.ws_bytes, need);
        else if (!st.d_ws || st.ws_bytes < need) rc = IPS4O_ERR_TOO_LARGE;
        if (rc != IPS4O_OK) return rc;
        if (mode == kFixed && (!st.h_stage || st.h_stage_bytes < host_stage_bytes<T>(caps))) return IPS4O_ERR_TOO_LARGE;
        carve<T>(caps, (char*)st.d_ws, &ws);
        if (mode != kEnqueue) {
            if (mode == kGrow) rc = ensure_host_pinned(&st.h_stage, &st.h_stage_bytes, host_stage_bytes<T>(caps));
            if (rc != IPS4O_OK) return rc;
            char* h = (char*)st.h_stage;
            h_subs = (SubDesc*)h;
            h += align_up(caps.max_sub * sizeof(SubDesc), 256);
            h_stripes = (StripeDesc*)h;
            h += align_up(caps.max_stripes * sizeof(StripeDesc), 256);
            h_ctr = (ChunkCounters*)h;
            h += align_up(sizeof(ChunkCounters), 256);
            h_tasks = (Task*)h;
        } else {
            // enqueue-only calls never stage anything on the host
            h_subs = nullptr;
            h_stripes = nullptr;
            h_ctr = nullptr;
            h_tasks = nullptr;
        }
        // a smaller base case than the capacity forces deeper recursion
        rec_cap = recursion_cap<T>(prm);
        base_cap = std::min((u32)T::kBaseSmall, rec_cap);
        k_max = (u32)std::min(256, std::max(4, prm.k_max));
        k_max = pow2_ceil_host(k_max);
        if (k_max > 256) k_max = 256;
        // kernel attributes once per (stream state, element type): later calls,
        // including ones made while a stream is captured, need no such calls
        if (!st.attrs_ready[T::kId]) {
            ips4o_status arc = set_kernel_attributes<T>(st);
            if (arc != IPS4O_OK) return arc;
        }
        permute_grid = st.permute_grid[T::kId];
        st.stats = ips4o_stats{};
        st.stats.workspace_bytes = st.ws_bytes;
        // a new call supersedes the statistics of an earlier asynchronous one
        st.pending = false;
        st.timed.clear();
        st.next_event = 0;
        return IPS4O_OK;
    }

    // --- profiling helpers: events around launches when prm.profile is set
    ips4o_status ev_begin(int phase, int* slot) {
        *slot = -1;
        if (!prm.profile) return IPS4O_OK;
        while ((int)st.events.size() < st.next_event + 2) {
            cudaEvent_t e;
            IPS4O_CUDA(cudaEventCreate(&e));
            st.events.push_back(e);
        }
        *slot = st.next_event;
        st.next_event += 2;
        IPS4O_CUDA(cudaEventRecord(st.events[*slot], stream));
        st.timed.push_back(DeviceState::Timed{phase, *slot});
        return IPS4O_OK;
    }
    ips4o_status ev_end(int slot) {
        st.stats.kernel_launches++;
        if (slot < 0) return IPS4O_OK;
        IPS4O_CUDA(cudaEventRecord(st.events[slot + 1], stream));
        return IPS4O_OK;
    }
    ips4o_status collect_events() { return collect_profile_events(st); }
#define IPS4O_LAUNCH(phase, ...)                                  \
    do {                                                          \
        int slot_;                                                \
        ips4o_status rc_ = ev_begin(phase, &slot_);               \
        if (rc_ != IPS4O_OK) return rc_;                          \
        cudaError_t le_ = cudaGetLastError();                     \
        if (le_ != cudaSuccess) {                                 \
            char w_[64];                                          \
            std::snprintf(w_, sizeof w_, "before launch of phase %d (driver line %d)", phase, __LINE__); \
            set_last_cuda_error(le_, w_);                         \
            return IPS4O_ERR_CUDA;                                \
        }                                                         \
        __VA_ARGS__;                                              \
        le_ = cudaGetLastError();                                 \
        if (le_ != cudaSuccess) {                                 \
            char w_[64];                                          \
            std::snprintf(w_, sizeof w_, "launch of phase %d (driver line %d)", phase, __LINE__); \
            set_last_cuda_error(le_, w_);                         \
            return IPS4O_ERR_CUDA;                                \
        }                                                         \
        rc_ = ev_end(slot_);                                      \
        if (rc_ != IPS4O_OK) return rc_;                          \
    } while (0)

    u32 spin_limit() const { return prm.spin_limit ? prm.spin_limit : kSpinLimit; }

    ips4o_status status_from(u32 bits) {
        if (h_ctr->guard_hits) {
            char msg[160];
            std::snprintf(msg, sizeof msg, "device bounds guard failed %u time(s); first at kernels line %u (%llu, %llu)",
                          h_ctr->guard_hits, h_ctr->guard_line, (unsigned long long)h_ctr->guard_a,
                          (unsigned long long)h_ctr->guard_b);
            set_last_message(msg);
        }
        if (bits & kStatusTimeout) return IPS4O_ERR_TIMEOUT;
        if (bits & (kStatusInternal | kStatusCapacity)) return IPS4O_ERR_INTERNAL;
        return IPS4O_OK;
    }

    // Small input: one shared-memory sort.
    ips4o_status base_only(E* d, u64 n) {
        h_tasks[0] = Task{0, n};
        IPS4O_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(ChunkCounters), stream));
        const bool tiny = n <= (u64)T::kBaseTiny;
        const bool small = !tiny && n <= (u64)T::kBaseSmall;
        Task* list = tiny ? ws.base_tiny : (small ? ws.base_small : ws.base_large);
        u32* cnt = tiny ? &ws.ctr->base_tiny : (small ? &ws.ctr->base_small : &ws.ctr->base_large);
        const u32 one = 1;
        IPS4O_CUDA(cudaMemcpyAsync(list, h_tasks, sizeof(Task), cudaMemcpyHostToDevice, stream));
        IPS4O_CUDA(cudaMemcpyAsync(cnt, &one, sizeof(u32), cudaMemcpyHostToDevice, stream));
        if (tiny) {
            IPS4O_LAUNCH(6, (k_base<T, BaseTiny<T>><<<1, BaseTiny<T>::TPB, BaseTiny<T>::smem_bytes, stream>>>(
                                d, list, cnt, ws.ctr)));
        } else if (small) {
            IPS4O_LAUNCH(6, (k_base<T, BaseSmall<T>><<<1, BaseSmall<T>::TPB, BaseSmall<T>::smem_bytes, stream>>>(
                                d, list, cnt, ws.ctr)));
        } else {
            IPS4O_LAUNCH(6, (k_base<T, BaseLarge<T>><<<1, BaseLarge<T>::TPB, BaseLarge<T>::smem_bytes, stream>>>(
                                d, list, cnt, ws.ctr)));
        }
        IPS4O_CUDA(cudaMemcpyAsync(h_ctr, ws.ctr, sizeof(ChunkCounters), cudaMemcpyDeviceToHost, stream));
        IPS4O_CUDA(cudaStreamSynchronize(stream));
        IPS4O_CUDA(cudaGetLastError());
        st.stats.base_case_buckets += h_ctr->base_buckets;
        ips4o_status rc = collect_events();
        if (rc != IPS4O_OK) return rc;
        return status_from(h_ctr->status);
    }

    // Stripe length of a level: the classification CTAs (one per SM) take
    // stripes dynamically, so the number of stripes should fill whole waves
    // of SMs.  Stripes of a subproblem have equal length and never cross it,
    // so with many subproblems the count is a sum of per-subproblem
    // roundings: try 1, 2, ... stripes per SM (from the stripes_per_sm
    // parameter on) and keep the count whose last wave is fullest, with a
    // small charge for extra stripes (more partial buffers to clean up).
    u64 pick_stripe_len(const Task* tasks, size_t count, u64 level_total) const {
        const u64 B = T::kBlock;
        const u64 sms = (u64)st.sms;
        const int w0 = std::max(1, prm.stripes_per_sm);
        u64 best_len = 0;
        double best_score = -1e30;
        // a level split into several chunks anyway keeps the default
        const int w1 = count <= caps.max_sub ? w0 + 6 : w0;
        u64 nmax = 0;
        for (size_t i = 0; i < count; ++i) nmax = std::max<u64>(nmax, tasks[i].n);
        for (int wv = w0; wv <= w1; ++wv) {
            const u64 K = (u64)wv * sms;
            u64 len = std::max<u64>((level_total + K - 1) / K, kMinStripe);
            len = (len + B - 1) / B * B;
            if (K >= count && nmax > len) {
                // unequal subproblems: the smallest length (in blocks) whose
                // stripes number at most K (see k_plan)
                u64 lo = len / B, hi = (nmax + B - 1) / B;
                while (lo < hi) {
                    const u64 mid = (lo + hi) / 2;
                    u64 c = 0;
                    for (size_t i = 0; i < count; ++i) c += (tasks[i].n + mid * B - 1) / (mid * B);
                    if (c <= K) hi = mid;
                    else lo = mid + 1;
                }
                len = hi * B;
            }
            u64 total = 0, pool = 0;
            for (size_t i = 0; i < count; ++i) {
                const u64 ns = std::min<u64>(std::max<u64>(1, (tasks[i].n + len - 1) / len), kMaxStripesPerSub);
                total += ns;
                pool += ns * std::min<u64>((u64)kMaxBuckets * (B - 1), len);
            }
            // more stripes than the workspace holds would split the level
            // into more chunks: only the first candidate may do that
            if (wv > w0 && (total > caps.max_stripes || pool > caps.pool_cap)) break;
            const u64 waves = (total + sms - 1) / sms;
            const double score = (double)total / (double)(waves * sms) - 0.02 * (wv - w0);
            if (score > best_score + 1e-9) { best_score = score; best_len = len; }
            if (len == kMinStripe) break;                 // shorter stripes are not allowed
            if (total == waves * sms) break;              // full waves: later candidates cannot score higher
        }
        return best_len;
    }

    // Plan one chunk starting at tasks[i0]; returns the number of tasks taken.
    size_t plan_chunk(const Task* tasks, size_t count, size_t i0, u64 level_total, u32 level, bool partition,
                      u32* nsub_out, u32* nstripes_out) {
        const u64 B = T::kBlock;
        if (i0 == 0) level_stripe_len = pick_stripe_len(tasks, count, level_total);
        const u64 stripe_len = level_stripe_len;
        u32 nsub = 0, nstr = 0;
        u64 pool = 0;
        size_t i = i0;
        for (; i < count; ++i) {
            const Task t = tasks[i];
            if (nsub >= caps.max_sub) break;
            const ips4o_class_params cp = class_table()[63 - __builtin_clzll(t.n)];
            u32 K = partition ? k_max : (cp.leaves ? (u32)cp.leaves : leaves_for(t.n, base_cap, k_max));
            u32 alpha = prm.alpha > 0 ? (u32)prm.alpha : (u32)kDefaultAlpha;
            if (!partition && cp.alpha) alpha = cp.alpha;
            alpha = std::max<u32>(1, std::min<u32>(alpha, (u32)T::kSampleMax / K));
            u64 ns = std::max<u64>(1, (t.n + stripe_len - 1) / stripe_len);
            ns = std::min<u64>(ns, kMaxStripesPerSub);
            u64 slen, need;
            for (;;) {
                slen = ((t.n + ns - 1) / ns + B - 1) / B * B;
                ns = (t.n + slen - 1) / slen;
                need = 0;
                for (u64 s = 0; s < ns; ++s) {
                    u64 len = std::min<u64>(slen, t.n - s * slen);
                    need += std::min<u64>((u64)kMaxBuckets * (B - 1), len);
                }
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
            for (u64 s = 0; s < ns; ++s) {
                StripeDesc& x = h_stripes[nstr + s];
                x.begin = t.begin + s * slen;
                x.end = t.begin + std::min<u64>((s + 1) * slen, t.n);
                x.pool_off = pool;
                const u64 len = x.end - x.begin;
                x.pool_cap = (u32)std::min<u64>((u64)kMaxBuckets * (B - 1), len);
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

    // src: where sampling and classification read the chunk's elements (d
    // itself unless the sort starts from a copy elsewhere, see src0)
    ips4o_status run_chunk(E* d, u32 nsub, u32 nstr, bool partition, u32* next_count, const E* src = nullptr) {
        if (!src) src = d;
        IPS4O_CUDA(cudaMemcpyAsync(ws.subs, h_subs, nsub * sizeof(SubDesc), cudaMemcpyHostToDevice, stream));
        IPS4O_CUDA(cudaMemcpyAsync(ws.stripes, h_stripes, nstr * sizeof(StripeDesc), cudaMemcpyHostToDevice, stream));
        IPS4O_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(ChunkCounters), stream));
        const u64 seed = prm.seed;
        IPS4O_LAUNCH(0, (k_sample<T, 512><<<nsub, 512, 0, stream>>>(src, ws, nsub, seed)));
        const int cgrid = (int)std::min<u32>(nstr, (u32)st.sms);
        IPS4O_LAUNCH(1, (k_classify<T><<<cgrid, ClassifyRegCfg<T>::TPB, ClassifyRegCfg<T>::smem_bytes, stream>>>(
                            d, src, ws, nstr)));
        IPS4O_LAUNCH(2, (k_prefix<T, 256><<<nsub, 256, 0, stream>>>(ws, nsub)));
        IPS4O_LAUNCH(3, (k_fix<T, 256><<<st.sms * 2, 256, 0, stream>>>(d, ws)));
        IPS4O_LAUNCH(4, (k_permute<T><<<permute_grid, PermuteCfg<T>::TPB, PermuteCfg<T>::smem_bytes, stream>>>(
                            d, ws, nsub, spin_limit())));
        // one cleanup CTA per (subproblem, bucket).  A subproblem planned
        // with K >= 4 leaves has at most K buckets: without equality buckets
        // at most K leaves, with them at most K/2 leaves and K - 1 buckets.
        u32 kmax_chunk = 1;
        for (u32 q = 0; q < nsub; ++q) kmax_chunk = std::max(kmax_chunk, h_subs[q].k_target);
        const u32 bstride = std::min<u32>(kMaxBuckets, kmax_chunk >= 4 ? kmax_chunk : 2 * kmax_chunk);
        // a bucket gathers partial buffers from every stripe of its
        // subproblem: with many stripes (the top level) a CTA per bucket,
        // with few (the lower levels, many small buckets) a warp per bucket
        u32 max_ns = 1;
        for (u32 q = 0; q < nsub; ++q) max_ns = std::max(max_ns, h_subs[q].num_stripes);
        if (max_ns > 16) {
            IPS4O_LAUNCH(5, (k_cleanup_cta<T><<<nsub * bstride, CleanupCtaCfg<T>::TPB, CleanupCtaCfg<T>::smem_bytes,
                                                stream>>>(d, ws, nsub, bstride, spin_limit(), partition ? 1u : 0u,
                                                          rec_cap)));
        } else {
            const u32 clgrid = (nsub * bstride + CleanupCfg<T>::WPC - 1) / CleanupCfg<T>::WPC;
            IPS4O_LAUNCH(5, (k_cleanup<T><<<clgrid, CleanupCfg<T>::TPB, CleanupCfg<T>::smem_bytes, stream>>>(
                                d, ws, nsub, bstride, spin_limit(), partition ? 1u : 0u, rec_cap)));
        }
        if (!partition) {
            IPS4O_LAUNCH(6, (k_base<T, BaseTiny<T>><<<st.sms * 4, BaseTiny<T>::TPB, BaseTiny<T>::smem_bytes, stream>>>(
                                d, ws.base_tiny, &ws.ctr->base_tiny, ws.ctr)));
            IPS4O_LAUNCH(6, (k_base<T, BaseSmall<T>><<<st.sms * 2, BaseSmall<T>::TPB, BaseSmall<T>::smem_bytes, stream>>>(
                                d, ws.base_small, &ws.ctr->base_small, ws.ctr)));
            IPS4O_LAUNCH(6, (k_base<T, BaseLarge<T>><<<st.sms, BaseLarge<T>::TPB, BaseLarge<T>::smem_bytes, stream>>>(
                                d, ws.base_large, &ws.ctr->base_large, ws.ctr)));
        }
        IPS4O_CUDA(cudaMemcpyAsync(h_ctr, ws.ctr, sizeof(ChunkCounters), cudaMemcpyDeviceToHost, stream));
        IPS4O_CUDA(cudaStreamSynchronize(stream));
        IPS4O_CUDA(cudaGetLastError());
        ips4o_status rc = collect_events();
        if (rc != IPS4O_OK) return rc;
        st.stats.blocks_moved += h_ctr->blocks_moved;
        st.stats.blocks_skipped += h_ctr->blocks_skipped;
        st.stats.fix_blocks_moved += h_ctr->fix_blocks;
        st.stats.base_case_buckets += h_ctr->base_buckets;
        st.stats.chunks++;
        st.stats.subproblems += nsub;
        rc = status_from(h_ctr->status);
        if (rc != IPS4O_OK) return rc;
        *next_count = h_ctr->next_count;
        return IPS4O_OK;
    }

    // The input of the first level when it is not d itself: a sort from a
    // host buffer reads it there (through its device address) during the
    // first sampling and classification, which write their blocks into d,
    // so the copy to the device costs no pass of its own.
    const E* src0 = nullptr;

    ips4o_status run(E* d, u64 n, PartitionOut* part) {
        ips4o_status rc = setup(n);
        if (rc != IPS4O_OK) return rc;
        st.stats.n = n;
        if (!part && n <= (u64)rec_cap) {
            if (src0 && src0 != d)
                IPS4O_CUDA(cudaMemcpyAsync(d, src0, n * sizeof(E), cudaMemcpyDefault, stream));
            return base_only(d, n);
        }
        return levels(d, std::vector<Task>{Task{0, n}}, part);
    }

    // One round of the device-planned recursion: k_plan picks the chunk, the
    // distribution step runs it (reading src, writing d), the base case sorts
    // the small buckets it made; with mark, the larger buckets get their
    // largest element in front (the strict recursion).
    ips4o_status launch_round(E* d, const E* src, const PlanArgs& pa, bool mark) {
        const u32 sms = (u32)st.sms;
        IPS4O_LAUNCH(7, (k_plan<T><<<1, 1024, 0, stream>>>(ws, pa)));
        IPS4O_LAUNCH(0, (k_sample<T, 512><<<2 * sms, 512, 0, stream>>>(src, ws, 0, prm.seed)));
        IPS4O_LAUNCH(1, (k_classify<T><<<sms, ClassifyRegCfg<T>::TPB, ClassifyRegCfg<T>::smem_bytes, stream>>>(
                            d, src, ws, 0)));
        IPS4O_LAUNCH(2, (k_prefix<T, 256><<<4 * sms, 256, 0, stream>>>(ws, 0)));
        IPS4O_LAUNCH(3, (k_fix<T, 256><<<2 * sms, 256, 0, stream>>>(d, ws)));
        IPS4O_LAUNCH(4, (k_permute<T><<<permute_grid, PermuteCfg<T>::TPB, PermuteCfg<T>::smem_bytes, stream>>>(
                            d, ws, 0, spin_limit())));
        IPS4O_LAUNCH(5, (k_cleanup_cta<T><<<2 * sms, CleanupCtaCfg<T>::TPB, CleanupCtaCfg<T>::smem_bytes,
                                            stream>>>(d, ws, 0, 1, spin_limit(), 0u, rec_cap)));
        IPS4O_LAUNCH(5, (k_cleanup<T><<<8 * sms, CleanupCfg<T>::TPB, CleanupCfg<T>::smem_bytes, stream>>>(
                            d, ws, 0, 1, spin_limit(), 0u, rec_cap)));
        if (mark) IPS4O_LAUNCH(5, (k_mark<T, 512><<<4 * sms, 512, 0, stream>>>(d, ws, rec_cap)));
        ips4o_status rc = launch_base_lists(d);
        if (rc != IPS4O_OK) return rc;
        return launch_copies(d);
    }

    // A result written to ws.out: the ranges of the copy list.
    ips4o_status launch_copies(E* d) {
        if (!ws.out) return IPS4O_OK;
        IPS4O_LAUNCH(6, (k_copy_tasks<T><<<4 * st.sms, 256, 0, stream>>>(d, ws.out, ws.copy_tasks, &ws.ctr->copy_count,
                                                                          ws.copy_cap)));
        return IPS4O_OK;
    }

    // A sort that is one base case, with the loop state of the device-planned
    // recursion (statistics are read from it).
    ips4o_status launch_base_only(E* d, u64 n) {
        IPS4O_LAUNCH(7, (k_plan_base<T><<<1, 32, 0, stream>>>(ws, n)));
        if (n <= (u64)T::kBaseTiny) {
            IPS4O_LAUNCH(6, (k_base<T, BaseTiny<T>><<<1, BaseTiny<T>::TPB, BaseTiny<T>::smem_bytes, stream>>>(
                                d, ws.base_tiny, &ws.ctr->base_tiny, ws.ctr, ws.out)));
        } else if (n <= (u64)T::kBaseSmall) {
            IPS4O_LAUNCH(6, (k_base<T, BaseSmall<T>><<<1, BaseSmall<T>::TPB, BaseSmall<T>::smem_bytes, stream>>>(
                                d, ws.base_small, &ws.ctr->base_small, ws.ctr, ws.out)));
        } else {
            IPS4O_LAUNCH(6, (k_base<T, BaseLarge<T>><<<1, BaseLarge<T>::TPB, BaseLarge<T>::smem_bytes, stream>>>(
                                d, ws.base_large, &ws.ctr->base_large, ws.ctr, ws.out)));
        }
        IPS4O_LAUNCH(7, (k_fold<T><<<1, 32, 0, stream>>>(ws)));
        return IPS4O_OK;
    }

    // The base case of the buckets in the three base lists.
    ips4o_status launch_base_lists(E* d) {
        const u32 sms = (u32)st.sms;
        IPS4O_LAUNCH(6, (k_base<T, BaseTiny<T>><<<4 * sms, BaseTiny<T>::TPB, BaseTiny<T>::smem_bytes, stream>>>(
                            d, ws.base_tiny, &ws.ctr->base_tiny, ws.ctr, ws.out)));
        IPS4O_LAUNCH(6, (k_base<T, BaseSmall<T>><<<2 * sms, BaseSmall<T>::TPB, BaseSmall<T>::smem_bytes, stream>>>(
                            d, ws.base_small, &ws.ctr->base_small, ws.ctr, ws.out)));
        IPS4O_LAUNCH(6, (k_base<T, BaseLarge<T>><<<sms, BaseLarge<T>::TPB, BaseLarge<T>::smem_bytes, stream>>>(
                            d, ws.base_large, &ws.ctr->base_large, ws.ctr, ws.out)));
        return IPS4O_OK;
    }

    // The strictly in-place sort (Section 4.6, see ips4o_strict.cuh): the
    // host loop over batches of subproblems found by scanning the array; the
    // only state between batches is the array, the scan position and the
    // piece carried across a window edge.  Synchronises once per round and
    // once per scanned window; statistics and device-side errors are read by
    // finalize_pending (the caller's).
    ips4o_status run_strict(E* d, u64 n) {
        const u64 rc_cap = recursion_cap<T>(prm);
        const u64 window = strict_window<T>(prm);
        const Caps<T> c = n <= rc_cap ? caps_for_rounds<T>(n, st.sms, rc_cap)
                                      : caps_for_strict<T>(n, st.sms, rc_cap, window);
        ips4o_status rc = setup(n, 0, &c, kGrow);
        if (rc != IPS4O_OK) return rc;
        st.stats.n = n;
        st.d_status = &ws.ls->status;
        st.pending = true;
        st.pending_ls = ws.ls;
        st.pending_stream = stream;
        if (n <= rc_cap) return launch_base_only(d, n);      // one base case: nothing recurses
        static_assert(sizeof(LoopState) <= 64 * sizeof(Task), "loop state read back through the task staging");
        LoopState* h_ls = (LoopState*)h_tasks;
        auto read_ls = [&]() -> ips4o_status {
            IPS4O_CUDA(cudaMemcpyAsync(h_ls, ws.ls, sizeof(LoopState), cudaMemcpyDeviceToHost, stream));
            IPS4O_CUDA(cudaStreamSynchronize(stream));
            return IPS4O_OK;
        };
        const u32 sms = (u32)st.sms;
        IPS4O_LAUNCH(7, (k_strict_init<T><<<1, 32, 0, stream>>>(ws, n)));
        PlanArgs pa{};
        pa.n = n;
        pa.k_max = k_max;
        pa.alpha = prm.alpha > 0 ? (u32)prm.alpha : (u32)kDefaultAlpha;
        pa.base_cap = base_cap;
        pa.sms = sms;
        pa.w0 = (u32)std::max(1, prm.stripes_per_sm);
        const u32 scan_grid = (u32)std::min<u64>((window + kScanTile - 1) / kScanTile, 8ull * sms);
        // every batch makes progress (a subproblem that is not all equal is
        // split into smaller pieces, with a new sample each batch); a batch
        // that repeats the previous one's first subproblem, count and size
        // many times over means a bug, reported instead of looping
        u64 last_begin = ~0ull, last_elems = 0, last_delta = ~0ull;
        u32 last_count = 0, repeats = 0;
        for (u32 batch = 0;; ++batch) {
            pa.newlevel = 1;
            pa.level = batch;
            for (;;) {                                     // the rounds of the batch
                if ((rc = launch_round(d, d, pa, true)) != IPS4O_OK) return rc;
                pa.newlevel = 0;
                if ((rc = read_ls()) != IPS4O_OK) return rc;
                if (h_ls->status || h_ls->cur_pos >= h_ls->cur_count) break;
            }
            if (h_ls->status) break;
            bool done = false;
            for (;;) {                                     // scan windows until work is found
                IPS4O_LAUNCH(7, (k_scan_begin<T><<<1, 32, 0, stream>>>(ws, n, window)));
                IPS4O_LAUNCH(7, (k_scan_max<T><<<scan_grid, kScanTPB, 0, stream>>>(d, ws)));
                IPS4O_LAUNCH(7, (k_scan_prefix<T><<<1, 1024, 0, stream>>>(d, ws)));
                IPS4O_LAUNCH(7, (k_scan_heads<T><<<scan_grid, kScanTPB, 0, stream>>>(d, ws, (u32)rc_cap)));
                IPS4O_LAUNCH(7, (k_scan_link<T><<<1, 1024, 0, stream>>>(ws, n, (u32)rc_cap)));
                if ((rc = launch_base_lists(d)) != IPS4O_OK) return rc;
                if ((rc = read_ls()) != IPS4O_OK) return rc;
                if (h_ls->status || h_ls->cur_count > 0) break;
                if (h_ls->scan_pos >= n) {
                    done = true;
                    break;
                }
            }
            if (done || h_ls->status) break;
            const u64 elems = h_ls->elements_distributed, delta = elems - last_elems;
            const bool same = h_ls->batch_begin == last_begin && h_ls->cur_count == last_count && delta == last_delta;
            repeats = same ? repeats + 1 : 0;
            if (repeats >= 64) {
                set_last_message("strict recursion: a batch repeated without progress");
                return IPS4O_ERR_INTERNAL;
            }
            last_begin = h_ls->batch_begin;
            last_count = h_ls->cur_count;
            last_elems = elems;
            last_delta = delta;
        }
        IPS4O_LAUNCH(7, (k_fold<T><<<1, 32, 0, stream>>>(ws)));
        return IPS4O_OK;
    }

    // The sort as enqueued work only (Section 4's recursion planned on the
    // device, see ips4o_rounds.cuh): no host synchronisation, so the call
    // returns at once and can be captured in a CUDA graph.  Under capture
    // the workspace must have been reserved (ips4o_reserve_workspace), since
    // nothing may be allocated; otherwise it grows as needed.  Statistics and
    // device-side errors are read back later (finalize_pending).
    ips4o_status enqueue_sort(E* d, u64 n, const E* from = nullptr, E* out = nullptr) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        IPS4O_CUDA(cudaStreamIsCapturing(stream, &cap));
        const bool capturing = cap != cudaStreamCaptureStatusNone;
        const u64 rc_cap = recursion_cap<T>(prm);
        const Caps<T> c = caps_for_rounds<T>(n, st.sms, rc_cap, out != nullptr);
        ips4o_status rc = setup(n, 0, &c, capturing ? kEnqueue : kGrow);
        if (rc != IPS4O_OK) return rc;
        ws.out = out;                              // the base case and the copies write the result there
        st.stats.n = n;
        st.d_status = &ws.ls->status;
        if (!from) from = d;
        if (n <= (u64)rec_cap) {
            if (from != d) IPS4O_CUDA(cudaMemcpyAsync(d, from, n * sizeof(E), cudaMemcpyDefault, stream));
            rc = launch_base_only(d, n);
            if (rc != IPS4O_OK) return rc;
        } else {
            PlanArgs pa{};
            pa.n = n;
            pa.first = 1;
            pa.k_max = k_max;
            pa.alpha = prm.alpha > 0 ? (u32)prm.alpha : (u32)kDefaultAlpha;
            pa.base_cap = base_cap;
            pa.sms = (u32)st.sms;
            pa.w0 = (u32)std::max(1, prm.stripes_per_sm);
            const u32 R = rounds_for(n, rc_cap, base_cap, k_max, c.max_sub);
            const u32 sms = (u32)st.sms;
            for (u32 r = 0; r < R; ++r) {
                pa.first = r == 0 ? 1u : 0u;
                rc = launch_round(d, r == 0 ? from : d, pa, false);   // round 0 is the whole input (level 1)
                if (rc != IPS4O_OK) return rc;
            }
            // subproblems left after the last round: the segment scheduler
            IPS4O_LAUNCH(7, (k_rounds_done<T><<<1, 1024, 0, stream>>>(ws)));
            const SegQueue sq{ws.init_tasks, ws.init_count, ws.init_count + 1, ws.stacks, (u32)ws.stack_cap};
            IPS4O_LAUNCH(4, (k_segments<T><<<fallback_grid<T>(c), SegCfg<T>::TPB, SegCfg<T>::smem_bytes,
                                             stream>>>(d, ws, sq, prm.seed, k_max, spin_limit())));
            if ((rc = launch_copies(d)) != IPS4O_OK) return rc;
            IPS4O_LAUNCH(7, (k_fold<T><<<1, 32, 0, stream>>>(ws)));
        }
        st.pending = true;
        st.pending_ls = ws.ls;
        st.pending_stream = stream;
        return IPS4O_OK;
    }

    // Independent segments d[t.begin, t.begin + t.n) of one array, all sorted
    // by one call: the segments no larger than the base case are sorted in
    // shared memory straight away; the others enter the first distribution
    // level together, so that every level is one set of launches for all of
    // them (Section 4: subproblems of one level are processed side by side).
    ips4o_status run_segments(E* d, const std::vector<Task>& segs) {
        u64 total = 0, nbase = 0;
        for (const Task& t : segs) {
            total += t.n;
            nbase += (t.n >= 2 && t.n <= (u64)recursion_cap<T>(prm)) ? 1 : 0;
        }
        ips4o_status rc = setup(total, nbase);
        if (rc != IPS4O_OK) return rc;
        st.stats.n = total;
        std::vector<Task> tiny, small, large, big;
        for (const Task& t : segs) {
            if (t.n < 2) continue;
            if (t.n > (u64)rec_cap) big.push_back(t);
            else if (t.n <= (u64)T::kBaseTiny) tiny.push_back(t);
            else if (t.n <= (u64)T::kBaseSmall) small.push_back(t);
            else large.push_back(t);
        }
        if (nbase > 0) {
            // init_tasks = tiny, then small, then large segments
            std::vector<Task> init;
            init.reserve(nbase);
            init.insert(init.end(), tiny.begin(), tiny.end());
            init.insert(init.end(), small.begin(), small.end());
            init.insert(init.end(), large.begin(), large.end());
            const u32 cnt[4] = {(u32)tiny.size(), (u32)small.size(), (u32)large.size(), 0u};
            // pageable sources: the copies have read them when the calls return
            IPS4O_CUDA(cudaMemcpyAsync(ws.init_tasks, init.data(), init.size() * sizeof(Task), cudaMemcpyHostToDevice,
                                       stream));
            IPS4O_CUDA(cudaMemcpyAsync(ws.init_count, cnt, sizeof cnt, cudaMemcpyHostToDevice, stream));
            IPS4O_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(ChunkCounters), stream));
            const int gtiny = (int)std::min<u64>(tiny.size(), (u64)st.sms * 4);
            const int gsmall = (int)std::min<u64>(small.size(), (u64)st.sms * 2);
            const int glarge = (int)std::min<u64>(large.size(), (u64)st.sms);
            const Task* t_small = ws.init_tasks + tiny.size();
            const Task* t_large = t_small + small.size();
            if (gtiny > 0)
                IPS4O_LAUNCH(6, (k_base<T, BaseTiny<T>><<<gtiny, BaseTiny<T>::TPB, BaseTiny<T>::smem_bytes,
                                                          stream>>>(d, ws.init_tasks, ws.init_count, ws.ctr)));
            if (gsmall > 0)
                IPS4O_LAUNCH(6, (k_base<T, BaseSmall<T>><<<gsmall, BaseSmall<T>::TPB, BaseSmall<T>::smem_bytes,
                                                           stream>>>(d, t_small, ws.init_count + 1, ws.ctr)));
            if (glarge > 0)
                IPS4O_LAUNCH(6, (k_base<T, BaseLarge<T>><<<glarge, BaseLarge<T>::TPB, BaseLarge<T>::smem_bytes,
                                                           stream>>>(d, t_large, ws.init_count + 2, ws.ctr)));
            IPS4O_CUDA(cudaMemcpyAsync(h_ctr, ws.ctr, sizeof(ChunkCounters), cudaMemcpyDeviceToHost, stream));
            IPS4O_CUDA(cudaStreamSynchronize(stream));
            IPS4O_CUDA(cudaGetLastError());
            st.stats.base_case_buckets += h_ctr->base_buckets;
            rc = collect_events();
            if (rc != IPS4O_OK) return rc;
            rc = status_from(h_ctr->status);
            if (rc != IPS4O_OK) return rc;
        }
        if (big.empty()) return IPS4O_OK;
        // larger subproblems first: chunks then hold subproblems of similar size
        std::sort(big.begin(), big.end(), [](const Task& a, const Task& b) { return a.n > b.n; });
        return levels(d, std::move(big), nullptr);
    }

    // All segments by the persistent segment scheduler (one CTA per array,
    // largest first).  The host only uploads the queue.
    ips4o_status run_scheduler(E* d, const std::vector<Task>& segs) {
        std::vector<Task> q;
        q.reserve(segs.size());
        u64 total = 0;
        for (const Task& t : segs) {
            total += t.n;
            if (t.n >= 2) q.push_back(t);
        }
        std::sort(q.begin(), q.end(), [](const Task& a, const Task& b) { return a.n > b.n; });
        const Caps<T> c = caps_for_scheduler<T>(st.sms, q.size());
        ips4o_status rc = setup(total, 0, &c);
        if (rc != IPS4O_OK) return rc;
        st.stats.n = total;
        if (q.empty()) return IPS4O_OK;
        const u32 cnt[2] = {(u32)q.size(), 0u};
        IPS4O_CUDA(cudaMemcpyAsync(ws.init_tasks, q.data(), q.size() * sizeof(Task), cudaMemcpyHostToDevice, stream));
        IPS4O_CUDA(cudaMemcpyAsync(ws.init_count, cnt, sizeof cnt, cudaMemcpyHostToDevice, stream));
        IPS4O_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(ChunkCounters), stream));
        const SegQueue sq{ws.init_tasks, ws.init_count, ws.init_count + 1, ws.stacks, (u32)ws.stack_cap};
        IPS4O_LAUNCH(4, (k_segments<T><<<st.sms, SegCfg<T>::TPB, SegCfg<T>::smem_bytes, stream>>>(
                            d, ws, sq, prm.seed, k_max, spin_limit())));
        IPS4O_CUDA(cudaMemcpyAsync(h_ctr, ws.ctr, sizeof(ChunkCounters), cudaMemcpyDeviceToHost, stream));
        IPS4O_CUDA(cudaStreamSynchronize(stream));
        IPS4O_CUDA(cudaGetLastError());
        rc = collect_events();
        if (rc != IPS4O_OK) return rc;
        st.stats.blocks_moved += h_ctr->blocks_moved;
        st.stats.blocks_skipped += h_ctr->blocks_skipped;
        st.stats.base_case_buckets += h_ctr->base_buckets;
        st.stats.subproblems = h_ctr->next_count;      // distribution steps run by the CTAs
        st.stats.levels = h_ctr->next_count ? 1 : 0;  // at least one level (depth is not tracked)
        st.stats.chunks = 1;
        return status_from(h_ctr->status);
    }

    // The same with the offsets in device memory and nothing but enqueued
    // work: no allocation, no host synchronisation (capturable in a CUDA
    // graph).  The workspace must have been reserved.  Errors land in the
    // status word that ips4o_stream_status reads.
    // The enqueue-only segmented sort with the recursion planned on the
    // device, as in enqueue_sort: the segments no larger than the base case
    // are sorted by the base case at once, the larger ones are the first
    // level's queue, and the rounds distribute them level by level (all
    // segments of a level side by side, Section 4's subproblems).  The level
    // queues are sized for the n the workspace was reserved for.  The host
    // does not know the segments' sizes, so it enqueues the rounds of the
    // reserved n plus one round per chunk the first level may need (each
    // segment above the base case takes at least one stripe and its pool
    // area); subproblems the rounds leave go to the segment scheduler.
    ips4o_status enqueue_segments_rounds(E* d, const u64* d_off, u64 num_segments, u64 n_res) {
        const u64 rc_cap = recursion_cap<T>(prm);
        const Caps<T> c = caps_for_segment_rounds<T>(n_res, st.sms, rc_cap, num_segments);
        ips4o_status rc = setup(n_res, 0, &c, kEnqueue);
        if (rc != IPS4O_OK) return rc;
        st.stats.n = 0;                            // the total is known on the device only
        st.d_status = &ws.ls->status;
        const u32 sms = (u32)st.sms;
        IPS4O_LAUNCH(7, (k_seg_rounds_init<T><<<1, 32, 0, stream>>>(ws)));
        const int g = (int)std::min<u64>((num_segments + 255) / 256, (u64)sms * 4);
        IPS4O_LAUNCH(7, (k_seg_big_hist<T><<<g, 256, 0, stream>>>(d_off, num_segments, ws, (u32)rc_cap)));
        IPS4O_LAUNCH(7, (k_seg_scan<<<1, 32, 0, stream>>>(ws.hist, &ws.ls->cur_count, &ws.ls->cur_pos)));
        IPS4O_LAUNCH(7, (k_seg_split<T><<<g, 256, 0, stream>>>(d_off, num_segments, ws, (u32)rc_cap)));
        // the base-case segments: one launch per size class over the whole list
        IPS4O_LAUNCH(6, (k_base<T, BaseTiny<T>><<<4 * sms, BaseTiny<T>::TPB, BaseTiny<T>::smem_bytes, stream>>>(
                            d, ws.init_tasks, ws.init_count, ws.ctr, nullptr, 0, (u64)T::kBaseTiny)));
        IPS4O_LAUNCH(6, (k_base<T, BaseSmall<T>><<<2 * sms, BaseSmall<T>::TPB, BaseSmall<T>::smem_bytes, stream>>>(
                            d, ws.init_tasks, ws.init_count, ws.ctr, nullptr, (u64)T::kBaseTiny, (u64)T::kBaseSmall)));
        IPS4O_LAUNCH(6, (k_base<T, BaseLarge<T>><<<sms, BaseLarge<T>::TPB, BaseLarge<T>::smem_bytes, stream>>>(
                            d, ws.init_tasks, ws.init_count, ws.ctr, nullptr, (u64)T::kBaseSmall, ~0ull)));
        PlanArgs pa{};
        pa.n = n_res;
        pa.k_max = k_max;
        pa.alpha = prm.alpha > 0 ? (u32)prm.alpha : (u32)kDefaultAlpha;
        pa.base_cap = base_cap;
        pa.sms = sms;
        pa.w0 = (u32)std::max(1, prm.stripes_per_sm);
        const u64 per = (u64)kMaxBuckets * (T::kBlock - 1);
        const u64 first_level = std::min<u64>(num_segments, n_res / (rc_cap + 1) + 1);
        const u64 per_chunk = std::max<u64>(1, std::min<u64>(c.max_sub, c.pool_cap / per));
        const u32 R = rounds_for(n_res, rc_cap, base_cap, k_max, c.max_sub) + (u32)((first_level + per_chunk - 1) / per_chunk);
        for (u32 r = 0; r < R; ++r) {
            pa.newlevel = r == 0 ? 1u : 0u;         // the first round plans the first level
            pa.level = 0;
            if ((rc = launch_round(d, d, pa, false)) != IPS4O_OK) return rc;
        }
        IPS4O_LAUNCH(7, (k_rounds_done<T><<<1, 1024, 0, stream>>>(ws)));
        const SegQueue sq{ws.init_tasks, ws.init_count, ws.init_count + 1, ws.stacks, (u32)ws.stack_cap};
        IPS4O_LAUNCH(4, (k_segments<T><<<fallback_grid<T>(c), SegCfg<T>::TPB, SegCfg<T>::smem_bytes, stream>>>(
                            d, ws, sq, prm.seed, k_max, spin_limit())));
        IPS4O_LAUNCH(7, (k_fold<T><<<1, 32, 0, stream>>>(ws)));
        st.pending = true;
        st.pending_ls = ws.ls;
        st.pending_stream = stream;
        return IPS4O_OK;
    }

    ips4o_status enqueue_scheduler(E* d, const u64* d_off, u64 num_segments) {
        const Caps<T> c = caps_for_scheduler<T>(st.sms, num_segments);
        ips4o_status rc = setup(0, 0, &c, kEnqueue);
        if (rc != IPS4O_OK) return rc;
        st.d_status = &ws.ctr->status;
        IPS4O_CUDA(cudaMemsetAsync(ws.ctr, 0, sizeof(ChunkCounters), stream));
        IPS4O_CUDA(cudaMemsetAsync(ws.hist, 0, 65 * sizeof(u32), stream));
        const int g = (int)std::min<u64>((num_segments + 255) / 256, (u64)st.sms * 4);
        IPS4O_LAUNCH(7, (k_seg_hist<<<g, 256, 0, stream>>>(d_off, num_segments, ws.hist)));
        IPS4O_LAUNCH(7, (k_seg_scan<<<1, 32, 0, stream>>>(ws.hist, ws.init_count, ws.init_count + 1)));
        IPS4O_LAUNCH(7, (k_seg_fill<<<g, 256, 0, stream>>>(d_off, num_segments, ws.hist, ws.init_tasks, ws.ctr)));
        const SegQueue sq{ws.init_tasks, ws.init_count, ws.init_count + 1, ws.stacks, (u32)ws.stack_cap};
        IPS4O_LAUNCH(4, (k_segments<T><<<st.sms, SegCfg<T>::TPB, SegCfg<T>::smem_bytes, stream>>>(
                            d, ws, sq, prm.seed, k_max, spin_limit())));
        return IPS4O_OK;
    }

    static constexpr size_t kSortTasksMax = 1 << 16;   // host sort of a level's subproblems up to this many

    ips4o_status levels(E* d, std::vector<Task> level_tasks, PartitionOut* part) {
        ips4o_status rc = IPS4O_OK;
        std::vector<Task> next;
        u32 level = 0;
        while (!level_tasks.empty()) {
            next.clear();
            u64 level_total = 0;
            for (const Task& t : level_tasks) level_total += t.n;
            size_t i = 0;
            while (i < level_tasks.size()) {
                u32 nsub = 0, nstr = 0;
                size_t taken = plan_chunk(level_tasks.data(), level_tasks.size(), i, level_total, level,
                                          part != nullptr, &nsub, &nstr);
                if (taken == 0) return IPS4O_ERR_INTERNAL;
                u32 cnt = 0;
                rc = run_chunk(d, nsub, nstr, part != nullptr, &cnt, level == 0 ? src0 : nullptr);
                if (rc != IPS4O_OK) return rc;
                for (u32 q = 0; q < nsub; ++q) st.stats.elements_distributed += h_subs[q].n;
                if (cnt > 0) {
                    if (cnt > caps.next_cap) return IPS4O_ERR_INTERNAL;
                    IPS4O_CUDA(cudaMemcpyAsync(h_tasks, ws.next_tasks, cnt * sizeof(Task), cudaMemcpyDeviceToHost,
                                               stream));
                    IPS4O_CUDA(cudaStreamSynchronize(stream));
                    next.insert(next.end(), h_tasks, h_tasks + cnt);
                }
                i += taken;
            }
            ++level;
            st.stats.levels = level;
            if (part) {
                // one distribution step only: export its result
                SubDesc sd;
                IPS4O_CUDA(cudaMemcpyAsync(&sd, ws.subs, sizeof(SubDesc), cudaMemcpyDeviceToHost, stream));
                IPS4O_CUDA(cudaStreamSynchronize(stream));
                const u32 nb = sd.nbuckets;
                IPS4O_CUDA(cudaMemcpy(part->bounds, ws.bstart, (nb + 1) * sizeof(u64), cudaMemcpyDeviceToHost));
                const u32 leaves = 1u << sd.log_leaves;
                std::vector<K> spl(kMaxLeaves);
                IPS4O_CUDA(cudaMemcpy(spl.data(), ws.spl, kMaxLeaves * sizeof(K), cudaMemcpyDeviceToHost));
                for (u32 q = 1; q < leaves; ++q) part->splitters[q - 1] = T::key_bits(spl[q]);
                *part->num_splitters = leaves - 1;
                *part->num_buckets = nb;
                *part->eq = (int)sd.eq;
                return IPS4O_OK;
            }
            level_tasks.swap(next);
            // larger subproblems first: their stripes are handed out first,
            // so the dynamic stripe scheduler ends the level with short ones
            if (level_tasks.size() <= kSortTasksMax)
                std::sort(level_tasks.begin(), level_tasks.end(),
                          [](const Task& a, const Task& b) { return a.n > b.n; });
            // guard against a runaway recursion (cannot happen: every level
            // shrinks every non-equality bucket)
            if (level > 64) return IPS4O_ERR_INTERNAL;
        }
        return IPS4O_OK;
    }
};

// ips4o_sort: enqueued work (device-planned levels); ips4o_partition: one
// host-planned distribution step whose result is read back.
template <class T>
ips4o_status sort_t(DeviceState& st, void* d, size_t n, cudaStream_t s, PartitionOut* part) {
    Driver<T> drv(st, s);
    if (part) return drv.run((typename T::elem_t*)d, (u64)n, part);
    return drv.enqueue_sort((typename T::elem_t*)d, (u64)n);
}

// d[0, n) = the sorted elements of src[0, n) (src device-accessible, e.g. the
// device address of pinned host memory; src is only read), enqueued.
template <class T>
ips4o_status sort_from_t(DeviceState& st, void* d, const void* src, size_t n, cudaStream_t s, void* out) {
    Driver<T> drv(st, s);
    return drv.enqueue_sort((typename T::elem_t*)d, (u64)n, (const typename T::elem_t*)src, (typename T::elem_t*)out);
}

// The strictly in-place sort of d[0, n) (Section 4.6); returns when the
// work is enqueued and its last batch found, the caller finalizes.
template <class T>
ips4o_status strict_sort_t(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    Driver<T> drv(st, s);
    return drv.run_strict((typename T::elem_t*)d, (u64)n);
}

// Device workspace of a strict sort of n elements: for n above the base case
// the same for every n.
template <class T>
size_t strict_workspace_bytes_t(size_t n, int sms) {
    const ips4o_params& prm = global_params();
    const u64 cap = recursion_cap<T>(prm);
    const Caps<T> c = n <= cap ? caps_for_rounds<T>(n, sms, cap) : caps_for_strict<T>(n, sms, cap, strict_window<T>(prm));
    return carve<T>(c, nullptr, nullptr);
}

// Grow the stream's workspace and staging to what a call on n elements in
// num_segments segments needs (nothing is freed).
template <class T>
ips4o_status reserve_t(DeviceState& st, u64 n, u64 num_segments) {
    const ips4o_params& prm = global_params();
    Caps<T> c = caps_for<T>(n, st.sms, prm.stripes_per_sm, recursion_cap<T>(prm));
    c.init_cap = num_segments;
    const Caps<T> cs = caps_for_segment_rounds<T>(n, st.sms, recursion_cap<T>(prm), num_segments);
    const size_t need = std::max({carve<T>(c, nullptr, nullptr),
                                  carve<T>(caps_for_scheduler<T>(st.sms, num_segments), nullptr, nullptr),
                                  carve<T>(caps_for_rounds<T>(n, st.sms, recursion_cap<T>(prm)), nullptr, nullptr),
                                  carve<T>(cs, nullptr, nullptr)});
    ips4o_status rc = ensure_device_buffer(&st.d_ws, &st.ws_bytes, need);
    if (rc != IPS4O_OK) return rc;
    st.reserved_n[T::kId] = std::max<u64>(st.reserved_n[T::kId], n);
    st.reserved_segments[T::kId] = std::max<u64>(st.reserved_segments[T::kId], num_segments);
    if (!st.attrs_ready[T::kId] && (rc = set_kernel_attributes<T>(st)) != IPS4O_OK) return rc;
    return ensure_host_pinned(&st.h_stage, &st.h_stage_bytes, host_stage_bytes<T>(c));
}

// Segmented calls that may synchronise take the level-by-level path unless
// the segment scheduler is asked for: measured on GB300 with 2^28 u64 keys
// in arrays of log-uniform lengths up to 2^20, level by level sorts about
// 30 G keys/s and the scheduler about 25 G keys/s.  The enqueue-only entry
// point always uses the scheduler.
template <class T>
ips4o_status sort_segments_t(DeviceState& st, void* d, const std::vector<Task>& segs, cudaStream_t s) {
    Driver<T> drv(st, s);
    if (global_params().segment_scheduler == 2) return drv.run_scheduler((typename T::elem_t*)d, segs);
    return drv.run_segments((typename T::elem_t*)d, segs);
}

template <class T>
ips4o_status upload_class_table_t(const ips4o_class_params* t) {
    unsigned short lv[64], al[64];
    for (int c = 0; c < 64; ++c) { lv[c] = t[c].leaves; al[c] = t[c].alpha; }
    IPS4O_CUDA(cudaMemcpyToSymbol(c_class_leaves, lv, sizeof lv));
    IPS4O_CUDA(cudaMemcpyToSymbol(c_class_alpha, al, sizeof al));
    return IPS4O_OK;
}

template <class T>
ips4o_status enqueue_segments_t(DeviceState& st, void* d, const u64* d_off, u64 num_segments, cudaStream_t s) {
    Driver<T> drv(st, s);
    // the device-planned levels need the total the workspace was reserved
    // for; the segment scheduler (segment_scheduler = 2) needs none
    const u64 n_res = st.reserved_n[T::kId];
    if (global_params().segment_scheduler == 2 || n_res == 0)
        return drv.enqueue_scheduler((typename T::elem_t*)d, d_off, num_segments);
    return drv.enqueue_segments_rounds((typename T::elem_t*)d, d_off, num_segments, n_res);
}

}  // namespace ips4o
