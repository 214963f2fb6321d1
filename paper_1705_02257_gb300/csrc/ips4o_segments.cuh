// ips4o_segments.cuh — the segment scheduler: many independent arrays sorted
// by one persistent launch, one CTA per array at a time.
//
// Section 4 hands the small subproblems of the recursion to single threads,
// each running the sequential algorithm, and assigns them "in a balanced
// way".  On the GPU the unit that sorts one small problem alone is a CTA: it
// runs the whole distribution step of Section 4 on one array -- sampling,
// local classification of the array as a single stripe, the block
// permutation with its own movers, the cleanup -- and sorts the buckets
// that fit the shared-memory base case (Section 4.7) right away; larger
// buckets go to a per-CTA stack and are distributed again by the same CTA.
// The arrays come from a queue ordered by decreasing size (the largest
// first, so that the tail of the launch is made of small arrays), and every
// CTA of the persistent grid takes the next one when it is done.
//
// The launch needs no host decision after it starts, so the whole batched
// sort is one kernel on the stream (plus, for the capturable entry point,
// the kernels that build the queue on the device).
#pragma once

#include "ips4o_kernels.cuh"

namespace ips4o {

// The size-class table (leaves, alpha) on the device; zero = default rule.
static __constant__ unsigned short c_class_leaves[64];
static __constant__ unsigned short c_class_alpha[64];

// Work queue and per-CTA stacks of the scheduler (device memory).
struct SegQueue {
    Task* tasks;        // [count] the arrays, largest first
    u32* count;         // number of tasks in the queue
    u32* next;          // queue cursor
    Task* stacks;       // [gridDim.x][stack_cap] buckets still to distribute
    u32 stack_cap;
};

template <class T>
struct SegCfg {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    static constexpr int TPB = 1024;
    static constexpr int NW = TPB / 32;
    static constexpr int NWP = 128 / PermuteCfg<T>::V;  // mover warps of the block permutation (128 movers)
    static constexpr int B = T::kBlock;
    typedef BaseLarge<T> Base;
    static_assert(Base::TPB == TPB, "the base case runs on the whole CTA");
    // phases reuse one shared-memory area
    static constexpr size_t sample_bytes = (size_t)T::kSampleMax * sizeof(K) + 256 * sizeof(K) + 32 * 4;
    static constexpr size_t prefix_bytes = 32 * 8 + 2 * kMaxStripesPerSub * 4 + (kMaxBuckets + 1) * 4;
    static constexpr size_t perm_buf = (size_t)NWP * 2 * PermuteCfg<T>::V * B * sizeof(E);
    static constexpr size_t perm_bytes = perm_buf + 2 * kMaxLeaves * sizeof(K) + (kMaxBuckets + 1) * 4;
    static constexpr size_t clean_bytes = (size_t)kMaxBuckets * B * sizeof(E);
    static constexpr size_t m1 = ClassifyCfg<T>::smem_bytes > Base::smem_bytes ? ClassifyCfg<T>::smem_bytes
                                                                                  : Base::smem_bytes;
    static constexpr size_t m2 = perm_bytes > clean_bytes ? perm_bytes : clean_bytes;
    static constexpr size_t m3 = sample_bytes > prefix_bytes ? sample_bytes : prefix_bytes;
    static constexpr size_t m12 = m1 > m2 ? m1 : m2;
    static constexpr size_t smem_bytes = m12 > m3 ? m12 : m3;
    static_assert(ClassifyCfg<T>::TPB == TPB, "classification runs on the whole CTA");
};

// Leaves of one distribution step of a subproblem of n elements: the
// adaptive number of buckets (Section 4.7) aimed at buckets of about half
// the base-case class T_small, as in the host driver.
__device__ __forceinline__ u32 seg_leaves(u64 n, u64 base_cap, u32 k_max) {
    const double r = 2.0 * (double)n / (double)base_cap;
    u32 k;
    if (r <= (double)k_max) k = pow2_ceil_u32((u32)ceil(r));
    else if (r <= 2.0 * (double)k_max) k = k_max;
    else if (r <= (double)k_max * (double)k_max) k = pow2_ceil_u32((u32)ceil(sqrt(r)));
    else k = k_max;
    k = k < 4 ? 4 : k;
    return k > k_max ? k_max : k;
}

// Cleanup of subproblem j with a single stripe (Section 4.3), by the whole
// CTA: first every bucket reads the overshoot of its last block into shared
// memory, then every bucket writes its sources (overshoot, partial buffer,
// overflow block) into its empty head and tail.  The barrier between the two
// phases replaces the hand-over flags of the multi-CTA cleanup.
template <class T>
__device__ void cleanup_sub_cta(typename T::elem_t* arr, const Workspace<T>& ws, u32 j, typename T::elem_t* ovbuf) {
    typedef typename T::elem_t E;
    constexpr int B = T::kBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const SubDesc sub = ws.subs[j];
    const u32 nb = sub.nbuckets;
    E* A = arr + sub.begin;
    const u64* bstart = ws.bstart + (u64)j * (kMaxBuckets + 1);
    const u32* dl = ws.delim + (u64)j * (kMaxBuckets + 1);
    const u64 nbc = sub.n / B;
    const bool partial = (sub.n % B) != 0;
    const StripeDesc sd = ws.stripes[sub.stripe_begin];
    auto geometry = [&](u32 b, u64& Bb, u64& Eb, u64& P_lo, u64& P_hi, u32& ov, u32& ovf) {
        Bb = bstart[b];
        Eb = bstart[b + 1];
        const u32 d0 = dl[b];
        const u64 w = (u64)d0 + (u64)pk_w(ws.wr[(u64)j * kMaxBuckets + b]);
        const bool has_blocks = w > d0;
        ovf = (partial && has_blocks && w == nbc + 1) ? (u32)B : 0u;
        P_lo = (u64)d0 * B;
        P_hi = has_blocks ? (ovf ? nbc : w) * B : P_lo;
        ov = (u32)((has_blocks && P_hi > Eb) ? P_hi - Eb : 0);
    };
    for (u32 b = warp; b < nb; b += nw) {
        u64 Bb, Eb, P_lo, P_hi;
        u32 ov, ovf;
        geometry(b, Bb, Eb, P_lo, P_hi, ov, ovf);
        if (ov > (u32)B || Eb < Bb || Eb > sub.n) {
            if (lane == 0) set_status(ws.ctr, kStatusInternal);
            continue;
        }
        for (u32 v = lane; v < ov; v += 32) ovbuf[(u64)b * B + v] = A[Eb + v];
    }
    __syncthreads();
    const E* ovb = ws.overflow + (u64)j * B;
    for (u32 b = warp; b < nb; b += nw) {
        u64 Bb, Eb, P_lo, P_hi;
        u32 ov, ovf;
        geometry(b, Bb, Eb, P_lo, P_hi, ov, ovf);
        if (ov > (u32)B || Eb < Bb || Eb > sub.n) continue;
        const u64 head_hi = P_lo < Eb ? P_lo : Eb;
        const u64 nh = head_hi > Bb ? head_hi - Bb : 0;
        const u64 nt = (P_lo < Eb && P_hi < Eb) ? Eb - P_hi : 0;
        const u64 si = (u64)sub.stripe_begin * kMaxBuckets + b;
        const u32 lc = ws.counts[si] % B;
        const E* lsrc = ws.pool + sd.pool_off + ws.lscan[si];
        const u64 nsrc = (u64)ov + ovf + lc;
        if (nh + nt != nsrc) {
            if (lane == 0) set_status(ws.ctr, kStatusInternal);
            continue;
        }
        for (u64 q = lane; q < nsrc; q += 32) {
            E x;
            if (q < ov) x = ovbuf[(u64)b * B + q];
            else if (q < (u64)ov + ovf) x = ovb[q - ov];
            else x = lsrc[q - ov - ovf];
            A[q < nh ? Bb + q : P_hi + (q - nh)] = x;
        }
    }
    __syncthreads();
}

// The persistent scheduler: grid = one CTA per SM (SegCfg<T>::TPB threads,
// SegCfg<T>::smem_bytes of shared memory).  CTA c uses workspace slot c for
// its subproblem, stripe, pool area and overflow block.
template <class T>
__global__ void __launch_bounds__(SegCfg<T>::TPB, 1)
    k_segments(typename T::elem_t* arr, Workspace<T> ws, SegQueue q, u64 seed, u32 k_max, u32 spin_limit) {
    typedef SegCfg<T> C;
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    constexpr int TPB = C::TPB, B = C::B;
    constexpr u32 CAP = (u32)C::Base::CAP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Task s_task;
    __shared__ u32 s_sp, s_done;
    const int tid = threadIdx.x, warp = tid >> 5;
    const u32 j = blockIdx.x;                       // this CTA's workspace slot
    Task* stack = q.stacks + (u64)j * q.stack_cap;
    u64 moved = 0, skipped = 0, base_buckets = 0;
    bool failed = false;
    if (tid == 0) s_sp = 0;
    __syncthreads();
    for (;;) {
        // next array: this CTA's own stack first, then the shared queue
        if (tid == 0) {
            s_done = 0;
            if (s_sp > 0) {
                s_task = stack[--s_sp];
            } else {
                const u32 i = atomicAdd(q.next, 1u);
                if (i < *q.count) s_task = q.tasks[i];
                else s_done = 1;
            }
        }
        __syncthreads();
        if (s_done) break;
        const Task t = s_task;
        __syncthreads();
        if (t.n < 2) continue;
        if (t.n <= (u64)CAP) {
            cta_sort<T, typename C::Base>(arr + t.begin, (u32)t.n, smem_raw);
            ++base_buckets;
            continue;
        }
        // ---- one distribution step of [t.begin, t.begin + t.n) by this CTA
        if (tid == 0) {
            atomicAdd(&ws.ctr->next_count, 1u);        // the scheduler counts its distribution steps here
            const int cls = 63 - __clzll((long long)t.n);
            u32 K_ = c_class_leaves[cls];
            if (K_ == 0) K_ = seg_leaves(t.n, (u64)T::kBaseSmall, k_max);
            u32 alpha = c_class_alpha[cls] ? c_class_alpha[cls] : 16u;
            if (alpha * K_ > (u32)T::kSampleMax) alpha = (u32)T::kSampleMax / K_;
            SubDesc sd;
            sd.begin = t.begin;
            sd.n = t.n;
            sd.stripe_begin = j;
            sd.num_stripes = 1;
            sd.k_target = K_;
            sd.alpha = alpha;
            sd.level = 0;
            sd.log_leaves = 0;
            sd.eq = 0;
            sd.nbuckets = 0;
            sd.blocks_total = 0;
            ws.subs[j] = sd;
            StripeDesc st;
            st.begin = t.begin;
            st.end = t.begin + t.n;
            st.pool_off = (u64)j * kMaxBuckets * (B - 1);
            st.pool_cap = (u32)(t.n < (u64)kMaxBuckets * (B - 1) ? t.n : (u64)kMaxBuckets * (B - 1));
            st.sub = j;
            ws.stripes[j] = st;
        }
        __syncthreads();
        {
            K* keys = (K*)smem_raw;
            K* cand = keys + T::kSampleMax;
            u32* scan = (u32*)(cand + 256);
            sample_sub<T, TPB>(arr, ws, j, seed, keys, cand, scan);
        }
        classify_stripe<T>(arr, ws, j, smem_raw);
        {
            u64* tmp64 = (u64*)smem_raw;
            u32* s_sbk = (u32*)(tmp64 + 32);
            u32* s_full = s_sbk + kMaxStripesPerSub;
            u32* s_delim = s_full + kMaxStripesPerSub;
            prefix_sub<T, TPB>(ws, j, tmp64, s_sbk, s_full, s_delim);
        }
        // block permutation by the first NWP warps (Section 4.2)
        K* tree = (K*)(smem_raw + C::perm_buf);
        K* spl = tree + kMaxLeaves;
        u32* delim = (u32*)(spl + kMaxLeaves);
        load_sub_tables<T>(ws, j, tree, spl, delim);
        __syncthreads();
        if (warp < C::NWP) {
            constexpr int V = PermuteCfg<T>::V;
            E* wbuf = (E*)smem_raw + (size_t)warp * 2 * V * B;
            if (ws.subs[j].blocks_total > 0)
                permute_group<T>(arr, ws, j, (u32)warp, (u32)(C::NWP * V), wbuf, tree, spl, delim, spin_limit, moved,
                                 skipped, failed);
        }
        __syncthreads();
        cleanup_sub_cta<T>(arr, ws, j, (E*)smem_raw);
        // buckets: the equality buckets are done, the ones that fit the
        // base case are sorted now, the others wait on the stack
        const SubDesc sub = ws.subs[j];
        const u64* bstart = ws.bstart + (u64)j * (kMaxBuckets + 1);
        for (u32 b = 0; b < sub.nbuckets; ++b) {
            const u64 lo = bstart[b], size = bstart[b + 1] - lo;
            if ((sub.eq && (b & 1)) || size < 2) continue;
            if (size <= (u64)CAP) {
                cta_sort<T, typename C::Base>(arr + sub.begin + lo, (u32)size, smem_raw);
                ++base_buckets;
            } else if (tid == 0) {
                if (s_sp < q.stack_cap) stack[s_sp++] = Task{sub.begin + lo, size};
                else set_status(ws.ctr, kStatusCapacity);
            }
        }
        __syncthreads();
    }
    if (moved) atomicAdd(&ws.ctr->blocks_moved, moved);
    if (skipped) atomicAdd(&ws.ctr->blocks_skipped, skipped);
    if (tid == 0 && base_buckets) atomicAdd(&ws.ctr->base_buckets, base_buckets);
}

// Queue of the capturable entry point, built on the device from an offsets
// array: arrays grouped by floor(log2 n), larger groups first (within a
// factor of two of largest-first order).
static __global__ void k_seg_hist(const u64* off, u64 count, u32* hist) {
    __shared__ u32 h[65];
    for (int i = threadIdx.x; i < 65; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (u64)gridDim.x * blockDim.x) {
        const u64 n = off[i + 1] >= off[i] ? off[i + 1] - off[i] : 0;
        atomicAdd(&h[n ? 64 - __clzll((long long)n) : 0], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 65; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// hist[65] counts -> start of each group in the queue (largest group first);
// also checks the offsets and records the queue length.
static __global__ void k_seg_scan(u32* hist, u32* qcount, u32* qnext) {
    if (threadIdx.x == 0) {
        u32 acc = 0;
        for (int g = 64; g >= 0; --g) {
            const u32 c = hist[g];
            hist[g] = acc;
            acc += c;
        }
        *qcount = acc;
        *qnext = 0;
    }
}

static __global__ void k_seg_fill(const u64* off, u64 count, u32* hist, Task* tasks, ChunkCounters* ctr) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (u64)gridDim.x * blockDim.x) {
        if (off[i + 1] < off[i]) {
            set_status(ctr, kStatusInternal);       // decreasing offsets
            continue;
        }
        const u64 n = off[i + 1] - off[i];
        const u32 pos = atomicAdd(&hist[n ? 64 - __clzll((long long)n) : 0], 1u);
        tasks[pos] = Task{off[i], n};
    }
}

}  // namespace ips4o
