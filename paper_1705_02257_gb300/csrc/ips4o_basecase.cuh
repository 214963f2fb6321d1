// ips4o_basecase.cuh — splitter selection (Sections 3, 4.4, 4.7) and the
// shared-memory base case (Section 4.7).
//
// The base case sorts one bucket of at most CAP elements with one CTA, in
// place of the paper's insertion sort of at most n0 = 16 elements.  The
// bucket is read once into registers; its key range is split into about one
// sub-range of equal power-of-two width per element (a bucket left by the
// sampled distribution steps is close to uniform over its range), the
// elements are counted and scattered into their sub-ranges in shared memory,
// and each element is written to global memory at its sub-range's start plus
// its rank among the keys of that sub-range.  Sub-ranges of more than LIMIT
// elements (clustered or repeated keys) are sorted afterwards, one at a time
// by the whole CTA, with a bitonic network in shared memory (or left as they
// are when all their keys are equal).  The bucket is read from and written
// to global memory once.
#pragma once

#include "ips4o_common.cuh"

namespace ips4o {

template <class K>
__device__ __forceinline__ K key_max();
template <>
__device__ __forceinline__ u64 key_max<u64>() { return ~0ull; }
template <>
__device__ __forceinline__ QKey key_max<QKey>() { return QKey{~0ull, ~0ull, ~0ull}; }
template <class K>
__device__ __forceinline__ K key_min();
template <>
__device__ __forceinline__ u64 key_min<u64>() { return 0ull; }
template <>
__device__ __forceinline__ QKey key_min<QKey>() { return QKey{0ull, 0ull, 0ull}; }
template <>
__device__ __forceinline__ RKey key_max<RKey>() { return RKey{~0ull, ~0ull}; }
template <>
__device__ __forceinline__ RKey key_min<RKey>() { return RKey{0ull, 0ull}; }

__device__ __forceinline__ u32 pow2_ceil_u32(u32 x) {
    return x <= 1 ? 1u : (1u << (32 - __clz(x - 1)));
}

// Bitonic sort of keys[0..P) (P a power of two) in shared memory.
template <class K, int TPB>
__device__ void sort_sample(K* keys, u32 P) {
    for (u32 k = 2; k <= P; k <<= 1) {
        for (u32 jj = k >> 1; jj > 0; jj >>= 1) {
            for (u32 i = threadIdx.x; i < P; i += TPB) {
                u32 ixj = i ^ jj;
                if (ixj > i) {
                    K a = keys[i], b = keys[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// The same bitonic network for a full sample of N keys (N a multiple of
// TPB): each thread keeps N / TPB consecutive keys in registers, so the
// stages whose partners lie in the same thread or the same warp need no
// shared memory and no barrier; only the stages across warps go through
// keys[] (about 10 of the 78 stages for 4096 keys and 512 threads).
template <class K, int TPB, int N>
__device__ void sort_sample_reg(K* keys) {
    constexpr int R = N / TPB;
    static_assert(R >= 1 && (R & (R - 1)) == 0 && N % TPB == 0, "whole power-of-two runs per thread");
    const u32 tid = threadIdx.x;
    K v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = keys[tid * R + r];
    __syncthreads();
    for (u32 k = 2; k <= (u32)N; k <<= 1) {
        for (u32 j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32u * R) {
                // partner in another warp: through shared memory
#pragma unroll
                for (int r = 0; r < R; ++r) keys[tid * R + r] = v[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const u32 i = tid * R + r;
                    const K o = keys[i ^ j];
                    const bool up = (i & k) == 0, low = (i & j) == 0;
                    v[r] = (low == up) ? (o < v[r] ? o : v[r]) : (v[r] < o ? o : v[r]);
                }
                __syncthreads();
            } else if (j >= (u32)R) {
                // partner in another lane of this warp
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const u32 i = tid * R + r;
                    const K o = shfl_xor_key(v[r], (int)(j / R));
                    const bool up = (i & k) == 0, low = (i & j) == 0;
                    v[r] = (low == up) ? (o < v[r] ? o : v[r]) : (v[r] < o ? o : v[r]);
                }
            } else {
                // partner in this thread's registers (jr takes the value of j
                // as a constant, so the registers are indexed statically)
#pragma unroll
                for (int jr = R / 2; jr >= 1; jr >>= 1) {
                    if (j != (u32)jr) continue;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (r & jr) continue;
                        const u32 i = tid * R + r;
                        const bool up = (i & k) == 0;
                        const K a = v[r], b = v[r | jr];
                        if ((b < a) == up) {
                            v[r] = b;
                            v[r | jr] = a;
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) keys[tid * R + r] = v[r];
    __syncthreads();
}

// From a sorted sample keys[0..alpha*kk-1), pick kk-1 equally spaced
// splitters s_j = keys[j*alpha - 1] (Section 3), remove duplicates, and turn
// on equality buckets when the sample repeated a splitter (Sections 4.4 and
// 4.7).  With equality buckets the selection is redone with kk/2 leaves so
// that 2*leaves - 1 <= 255 buckets.  The distinct splitters are padded to
// L - 1 (L a power of two) by repeating the largest, and written as the
// sorted array spl[1..L-1] and the implicit tree tree[1..L-1]
// (tree[1] = s_{L/2}, children of node v are 2v and 2v+1).
// Requires blockDim.x >= 256; all threads must call it.
template <class K>
__device__ void select_splitters(const K* keys, u32 kk, u32 alpha, K* cand, u32* scan_tmp, K* tree, K* spl,
                                 u32* log_leaves_out, bool* eq_out) {
    u32 ncand = kk - 1;
    if (threadIdx.x < ncand) cand[threadIdx.x] = keys[(threadIdx.x + 1) * alpha - 1];
    __syncthreads();
    int dup = (threadIdx.x > 0 && threadIdx.x < ncand && cand[threadIdx.x] == cand[threadIdx.x - 1]) ? 1 : 0;
    const bool eq = __syncthreads_or(dup) != 0;
    if (eq && kk >= 4) {
        ncand = kk / 2 - 1;
        if (threadIdx.x < ncand) cand[threadIdx.x] = keys[(threadIdx.x + 1) * 2 * alpha - 1];
        __syncthreads();
    }
    const u32 keep = (threadIdx.x < ncand && (threadIdx.x == 0 || cand[threadIdx.x] != cand[threadIdx.x - 1])) ? 1u : 0u;
    const K mine = threadIdx.x < ncand ? cand[threadIdx.x] : key_min<K>();
    u32 m;
    const u32 pos = block_exclusive_scan<u32>(keep, scan_tmp, &m);
    __syncthreads();
    if (keep) cand[pos] = mine;
    __syncthreads();
    if (m == 0) m = 1;
    const u32 L = pow2_ceil_u32(m + 1);
    for (u32 i = threadIdx.x; i < kMaxLeaves; i += blockDim.x) {
        spl[i] = cand[(i >= 1 ? (i <= m ? i : m) : 1) - 1];
        K val = cand[0];
        if (i >= 1 && i < L) {
            const u32 dd = 31 - __clz(i);
            const u32 idx = (2 * (i - (1u << dd)) + 1) * (L >> (dd + 1));
            val = cand[(idx <= m ? idx : m) - 1];
        }
        tree[i] = val;
    }
    *log_leaves_out = 31 - __clz(L);
    *eq_out = eq;
}

template <class T, int TPB_, int CAP_>
struct BaseCfg {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    static constexpr int TPB = TPB_;
    static constexpr int NW = TPB / 32;
    static constexpr int CAP = CAP_;
    static constexpr int EPT = CAP / TPB;
    static constexpr int N0 = 1;             // target sub-bucket size
    static constexpr int MAXSUB = CAP / N0;  // sub-buckets of the on-chip distribution
    static constexpr int LIMIT = 64;         // larger sub-buckets are sorted one at a time by the CTA
    static constexpr int MAXBIG = CAP / LIMIT;
    // sub-bucket counters/starts: entry s at pad(s) = s + s / 32, so that the
    // SUBS_PER_THREAD consecutive entries each thread scans start in
    // different banks for the 32 lanes of a warp
    static constexpr u32 PADDED = MAXSUB + MAXSUB / 32 + 1;
    static constexpr size_t off_data = 0;
    static constexpr size_t off_off = a16(off_data + (size_t)CAP * sizeof(E));   // u32[PADDED]
    static constexpr size_t off_tmp = a16(off_off + ((size_t)PADDED * 4 + 15) / 16 * 16);
    static constexpr size_t off_big = a16(off_tmp + 64 * sizeof(K));             // u32[MAXBIG + 1]
    static constexpr size_t smem_bytes = a16(off_big + (MAXBIG + 1) * 4);
    static constexpr int SUBS_PER_THREAD = MAXSUB / TPB;
    static_assert(CAP % TPB == 0, "capacity must be a multiple of the CTA size");
    static_assert(CAP <= 65535, "ranks are packed in 16 bits");
    static_assert(MAXSUB % TPB == 0, "whole sub-bucket counters per thread");
    __device__ static __forceinline__ u32 pad(u32 s) { return s + (s >> 5); }
};

// The three size classes: buckets of at most kBaseTiny elements (the typical
// bucket of a last distribution step) are sorted by 256-thread CTAs, four
// per SM; up to kBaseSmall by 512-thread CTAs, two per SM; the rare larger
// ones (up to kBaseCap) by 1024-thread CTAs.
template <class T>
using BaseTiny = BaseCfg<T, 256, T::kBaseTiny>;
template <class T>
using BaseSmall = BaseCfg<T, 512, T::kBaseSmall>;
template <class T>
using BaseLarge = BaseCfg<T, 1024, T::kBaseCap>;

// In-place sort of s[0..n) in shared memory by the whole CTA: a bitonic
// network whose merge stages start by comparing element i with its mirror
// (i ^ (size-1)), so every comparator puts the smaller key at the lower
// index and positions >= n behave as +infinity and are never touched.
template <class T, int TPB>
__device__ void cta_bitonic(typename T::elem_t* s, u32 n) {
    typedef typename T::elem_t E;
    const u32 P = pow2_ceil_u32(n);
    for (u32 k = 2; k <= P; k <<= 1) {
        const u32 half = k >> 1;
        for (u32 t = threadIdx.x; t < P / 2; t += TPB) {
            const u32 i = (t / half) * k + (t % half), j = i ^ (k - 1);
            if (j < n) {
                E a = s[i], b = s[j];
                if (T::key(b) < T::key(a)) { s[i] = b; s[j] = a; }
            }
        }
        __syncthreads();
        for (u32 st = k >> 2; st > 0; st >>= 1) {
            for (u32 t = threadIdx.x; t < P / 2; t += TPB) {
                const u32 i = (t / st) * 2 * st + (t % st), j = i + st;
                if (j < n) {
                    E a = s[i], b = s[j];
                    if (T::key(b) < T::key(a)) { s[i] = b; s[j] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// Sort g[0..m), m <= CAP, with the whole CTA (BaseCfg<T>::TPB threads).
//
// The bucket is read once into registers.  Its key range [lo, hi] is split
// into at most KB (about m / N0) sub-ranges of equal power-of-two width, and
// every element goes to sub-bucket (key - lo) >> shift; a bucket produced by
// the sampled distribution steps is close to uniform over its range, so the
// sub-buckets are small.  After a
// counting-sort scatter into shared memory, each element's final position is
// the start of its sub-bucket plus the number of keys of that sub-bucket
// that are smaller (or equal and earlier), and it is written there directly.
// Sub-buckets of more than LIMIT elements (clustered or repeated keys) are
// handled afterwards, one at a time by the whole CTA: left as they are when
// all their keys are equal, else sorted in shared memory by a bitonic
// network, so the cost stays bounded for any input.  With out, the sorted
// bucket is written to out[0..m) instead of back to g.
template <class T, class C>
__device__ void cta_sort(typename T::elem_t* g, u32 m, unsigned char* smem, typename T::elem_t* out = nullptr) {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    constexpr int TPB = C::TPB, EPT = C::EPT, SPT = C::SUBS_PER_THREAD;
    if (m < 2) {
        if (out && m == 1 && threadIdx.x == 0) out[0] = g[0];
        return;
    }
    E* go = out ? out : g;
    E* data = (E*)(smem + C::off_data);
    u32* off = (u32*)(smem + C::off_off);          // sub-bucket sizes, then (scanned) starts
    K* tmp = (K*)(smem + C::off_tmp);
    u32* big_list = (u32*)(smem + C::off_big);     // [0] count, then the large sub-buckets
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    E e[EPT];
    K lo = key_max<K>(), hi = key_min<K>();
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const u32 idx = tid + q * TPB;
        if (idx < m) {
            e[q] = g[idx];
            const K k = T::key(e[q]);
            lo = k < lo ? k : lo;
            hi = k > hi ? k : hi;
        }
    }
#pragma unroll
    for (int q = 0; q < SPT; ++q) off[C::pad(tid * SPT + q)] = 0;
    if (tid == 0) { off[C::pad(C::MAXSUB)] = 0; big_list[0] = 0; }
    // key range of the bucket
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const K a = shfl_xor_key(lo, o), b = shfl_xor_key(hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    if (lane == 0) { tmp[warp] = lo; tmp[32 + warp] = hi; }
    __syncthreads();
    lo = tmp[0];
    hi = tmp[32];
#pragma unroll
    for (int w = 1; w < C::NW; ++w) {
        lo = tmp[w] < lo ? tmp[w] : lo;
        hi = tmp[32 + w] > hi ? tmp[32 + w] : hi;
    }
    const bool all_equal = lo == hi;
    __syncthreads();                               // every thread has read tmp before it is reused
    if (all_equal) {                               // all keys equal: already sorted (uniform exit)
        if (out) {
#pragma unroll
            for (int q = 0; q < EPT; ++q)
                if (tid + q * TPB < m) out[tid + q * TPB] = e[q];
        }
        return;
    }
    u32 KB = pow2_ceil_u32((m + C::N0 - 1) / C::N0);
    KB = KB < 2 ? 2 : (KB > (u32)C::MAXSUB ? (u32)C::MAXSUB : KB);
    // sub-bucket = (key - lo) >> shift, with shift chosen so that the whole
    // range [lo, hi] maps into [0, KB): a monotone map of the key, so lower
    // sub-buckets hold smaller keys; sub-buckets cover equal key ranges
    // (for a key of several words, the sub-buckets split the range of the
    // leading word; keys equal in it and different in later words share a
    // sub-bucket, which the rank loop or the bitonic network then orders)
    const u64 lo_w = T::sub_key(lo);
    const u64 range = T::sub_key(hi) - lo_w;      // >= 1 for one-word keys
    const int bits = range ? 64 - __clzll((long long)range) : 0;
    const int logkb = 31 - __clz(KB);
    const int shift = bits > logkb ? bits - logkb : 0;
    auto sub_of = [&](const K& k) -> u32 {
        const u64 d = (T::sub_key(k) - lo_w) >> shift;
        return d < (u64)KB ? (u32)d : KB - 1;
    };
    u32 rk2[(EPT + 1) / 2];                          // arrival ranks, two 16-bit ranks per register
#pragma unroll
    for (int q = 0; q < (EPT + 1) / 2; ++q) rk2[q] = 0;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const u32 idx = tid + q * TPB;
        if (idx < m) {
            const u32 r = atomicAdd(&off[C::pad(sub_of(T::key(e[q])))], 1u);
            rk2[q / 2] |= r << (16 * (q & 1));
        }
    }
    __syncthreads();
    // exclusive scan of the sub-bucket sizes in place (SPT consecutive entries
    // per thread, read twice rather than held in registers); entry MAXSUB
    // receives the total
    u32 csum = 0;
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        const u32 cq = off[C::pad(tid * SPT + q)];
        csum += cq;
        if (cq > (u32)C::LIMIT) big_list[1 + atomicAdd(&big_list[0], 1u)] = tid * SPT + q;
    }
    __syncthreads();
    u32 tot;
    u32 pre = block_exclusive_scan<u32>(csum, (u32*)tmp, &tot);
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        const u32 cq = off[C::pad(tid * SPT + q)];
        off[C::pad(tid * SPT + q)] = pre;
        pre += cq;
    }
    if (tid == TPB - 1) off[C::pad(C::MAXSUB)] = pre;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const u32 idx = tid + q * TPB;
        if (idx < m) {
            const u32 r = (rk2[q / 2] >> (16 * (q & 1))) & 0xffffu;
            data[off[C::pad(sub_of(T::key(e[q])))] + r] = e[q];
        }
    }
    __syncthreads();
    // final position = sub-bucket start + rank of the key within it
    // (elements of large sub-buckets are placed below)
    // (not unrolled: the loop body holds the rank loop, and the unrolled
    // copies cost more in instruction fetch than they save)
#pragma unroll 1
    for (int q = 0; q < EPT; ++q) {
        const u32 i = tid + q * TPB;
        if (i < m) {
            const E x = data[i];
            const K k = T::key(x);
            const u32 sb = sub_of(k);
            const u32 o = off[C::pad(sb)], o1 = off[C::pad(sb + 1)];
            if (o1 - o > (u32)C::LIMIT) continue;
            u32 r = 0;
            for (u32 jj = o; jj < o1; ++jj) {
                const K kj = T::key(data[jj]);
                r += (kj < k || (kj == k && jj < i)) ? 1u : 0u;
            }
            go[o + r] = x;
        }
    }
    const u32 nbig = big_list[0];
    for (u32 q = 0; q < nbig; ++q) {
        const u32 sb = big_list[1 + q];
        const u32 o = off[C::pad(sb)], len = off[C::pad(sb + 1)] - o;
        // all keys equal: any order is sorted
        const K k0 = T::key(data[o]);
        int differs = 0;
        for (u32 i = tid; i < len; i += TPB) differs |= T::key(data[o + i]) != k0;
        if (__syncthreads_or(differs)) cta_bitonic<T, TPB>(data + o, len);
        for (u32 i = tid; i < len; i += TPB) go[o + i] = data[o + i];
        __syncthreads();
    }
    __syncthreads();
}

// Base-case tasks (buckets or whole small inputs): a persistent grid whose
// CTAs take the next entry of the list from a counter (ctr->base_next)
// whenever they are free, so that they finish together whatever the sizes;
// the count is read from device memory, so the launch does not depend on the
// host.  The last CTA to take its last entry sets the counter back to zero
// for the next launch (every CTA has then made its last claim: its claim
// returned before it counted itself in ctr->base_done).  With out, each
// sorted bucket goes to the same range of out instead of arr.  With a size
// window (min_excl, max_incl], only the tasks of that size are sorted (a list
// of tasks of all size classes, one launch per class).
template <class T, class C>
__global__ void __launch_bounds__(C::TPB, (C::TPB <= 256 ? 4 : (C::TPB <= 512 ? 2 : 1)))
    k_base(typename T::elem_t* arr, const Task* tasks, const u32* count, ChunkCounters* ctr,
           typename T::elem_t* out = nullptr, u64 min_excl = 0, u64 max_incl = ~0ull) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ u32 s_task;
    const u32 n = *count;
    u32 mine = 0;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(&ctr->base_next, 1u);
        __syncthreads();
        const u32 i = s_task;
        __syncthreads();
        if (i >= n) break;
        const Task t = tasks[i];
        if (t.n <= min_excl || t.n > max_incl) continue;
        if (!IPS4O_GUARD(ctr, t.n <= (u64)C::CAP, t.n, C::CAP)) continue;
        cta_sort<T, C>(arr + t.begin, (u32)t.n, smem_raw, out ? out + t.begin : nullptr);
        ++mine;
    }
    if (threadIdx.x == 0) {
        if (mine) atomicAdd(&ctr->base_buckets, (u64)mine);
        if (atomicAdd(&ctr->base_done, 1u) == gridDim.x - 1) {
            ctr->base_next = 0;
            ctr->base_done = 0;
        }
    }
}

}  // namespace ips4o
