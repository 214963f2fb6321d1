// ips4o_basecase.cuh — splitter selection (Sections 3, 4.4, 4.7) and the
// shared-memory base case.
//
// The base case sorts one bucket of at most T elements with one CTA.  It is
// the method's own recursion carried out on chip: the bucket is loaded once
// into registers and shared memory, a sample gives up to 255 splitters
// (equality buckets when the sample repeats keys), every element is
// classified with the implicit search tree and scattered into its
// sub-bucket in shared memory, and the sub-buckets, about n0 = 16 elements
// each (Section 4.7), are finished by insertion sort.  The bucket is read
// from and written to global memory exactly once.
#pragma once

#include "ips4o_common.cuh"

namespace ips4o {

template <class K>
__device__ __forceinline__ K key_max();
template <>
__device__ __forceinline__ u64 key_max<u64>() { return ~0ull; }

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
    const K mine = threadIdx.x < ncand ? cand[threadIdx.x] : K(0);
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

template <class T>
struct BaseCfg {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    static constexpr int TPB = 512;
    static constexpr int NW = TPB / 32;
    static constexpr int CAP = T::kBaseCap;
    static constexpr int EPT = CAP / TPB;
    static constexpr int MAXSUB = 512;       // sub-buckets of the on-chip distribution
    static constexpr int N0 = 8;             // target sub-bucket size
    static constexpr int LIMIT = 64;         // any larger sub-bucket: whole-bucket bitonic fallback
    static constexpr size_t off_data = 0;
    static constexpr size_t off_cnt = off_data + (size_t)CAP * sizeof(E);
    static constexpr size_t off_off = off_cnt + MAXSUB * 4;
    static constexpr size_t off_tmp = off_off + MAXSUB * 4;
    static constexpr size_t smem_bytes = off_tmp + 64 * 8;
    static_assert(CAP % TPB == 0, "capacity must be a multiple of the CTA size");
    static_assert(CAP < 65536, "ranks are packed in 16 bits");
    static_assert(MAXSUB <= TPB, "one scan entry per thread");
};

template <class T>
__device__ __forceinline__ void insertion_sort(typename T::elem_t* a, u32 n) {
    typedef typename T::elem_t E;
    for (u32 i = 1; i < n; ++i) {
        const E x = a[i];
        const typename T::key_t kx = T::key(x);
        u32 j = i;
        while (j > 0 && kx < T::key(a[j - 1])) {
            a[j] = a[j - 1];
            --j;
        }
        a[j] = x;
    }
}

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
// The bucket is read once into registers (and a shared-memory copy).  Its
// key range [lo, hi] is split into KB equal sub-ranges, KB about m / 8, and
// every element goes to sub-bucket floor((key - lo) * KB / (hi - lo + 1))
// (one 64-bit multiply-high); a bucket produced by the sampled distribution
// steps is close to uniform over its range, so the sub-buckets are small.
// After a counting-sort scatter in shared memory each sub-bucket is
// finished by insertion sort.  If some sub-bucket exceeds LIMIT elements
// (clustered keys), the whole bucket is sorted by a bitonic network
// instead, so the cost stays bounded for any input.
template <class T>
__device__ void cta_sort(typename T::elem_t* g, u32 m, unsigned char* smem, u64 seed) {
    typedef BaseCfg<T> C;
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    constexpr int TPB = C::TPB, EPT = C::EPT;
    (void)seed;
    if (m < 2) return;
    E* data = (E*)(smem + C::off_data);
    u32* cnt = (u32*)(smem + C::off_cnt);
    u32* off = (u32*)(smem + C::off_off);
    u64* tmp = (u64*)(smem + C::off_tmp);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    E e[EPT];
    K lo = ~K(0), hi = K(0);
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const u32 idx = tid + q * TPB;
        if (idx < m) {
            e[q] = g[idx];
            data[idx] = e[q];
            const K k = T::key(e[q]);
            lo = k < lo ? k : lo;
            hi = k > hi ? k : hi;
        }
    }
    if (tid < C::MAXSUB) cnt[tid] = 0;
    // key range of the bucket
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const K a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
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
    if (all_equal) return;                         // all keys equal: already sorted (uniform exit)
    u32 KB = pow2_ceil_u32((m + C::N0 - 1) / C::N0);
    KB = KB < 2 ? 2 : (KB > (u32)C::MAXSUB ? (u32)C::MAXSUB : KB);
    const u64 range = (u64)(hi - lo);             // >= 1
    const bool direct = range < KB;               // few distinct values: one sub-bucket per value
    // floor(2^64 / (range + 1)) * KB, without dividing by zero when the
    // bucket spans the whole 64-bit key range
    const u64 mult = direct ? 0 : (range == ~0ull ? (u64)KB : (~0ull / (range + 1)) * KB);
    u32 br[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const u32 idx = tid + q * TPB;
        if (idx < m) {
            const u64 d = (u64)(T::key(e[q]) - lo);
            u32 b = direct ? (u32)d : (u32)__umul64hi(d, mult);
            b = b < KB ? b : KB - 1;                   // cannot trigger; keeps the index in range
            br[q] = (b << 16) | atomicAdd(&cnt[b], 1u);
        }
    }
    __syncthreads();
    const u32 c = (u32)tid < (u32)C::MAXSUB ? cnt[tid] : 0u;
    const int big = __syncthreads_or(c > (u32)C::LIMIT ? 1 : 0);
    if (big) {
        // clustered keys: the copy in shared memory is sorted as a whole
        cta_bitonic<T, TPB>(data, m);
    } else {
        u32 tot;
        const u32 pre = block_exclusive_scan<u32>(c, (u32*)tmp, &tot);
        if ((u32)tid < (u32)C::MAXSUB) off[tid] = pre;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const u32 idx = tid + q * TPB;
            if (idx < m) data[off[br[q] >> 16] + (br[q] & 0xffffu)] = e[q];
        }
        __syncthreads();
        if ((u32)tid < KB && c > 1) insertion_sort<T>(data + off[tid], c);
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const u32 idx = tid + q * TPB;
        if (idx < m) g[idx] = data[idx];
    }
    __syncthreads();
}

// Whole small inputs or segments: one CTA per segment.
template <class T>
__global__ void __launch_bounds__(BaseCfg<T>::TPB, 2) k_base(typename T::elem_t* arr, const Task* segs, u32 nseg,
                                                          ChunkCounters* ctr, u64 seed) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (u32 i = blockIdx.x; i < nseg; i += gridDim.x) {
        const Task t = segs[i];
        if (t.n > (u64)BaseCfg<T>::CAP) {
            if (threadIdx.x == 0) set_status(ctr, kStatusInternal);
            continue;
        }
        cta_sort<T>(arr + t.begin, (u32)t.n, smem_raw, seed ^ mix64(t.begin));
    }
}

}  // namespace ips4o
