// ips4o_common.cuh — element traits, workspace layout and device primitives
// shared by the distribution-step kernels.
//
// Terminology follows the paper (Sections 3 and 4): k buckets per step,
// blocks of b elements, stripes (one per local-classification work item,
// the GPU counterpart of a thread's stripe), delimiters d_i, write/read
// pointers w_i and r_i, overflow block, equality buckets.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace ips4o {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int kMaxBuckets = 256;      // buckets per step (ids fit one byte)
constexpr int kMaxLeaves = 256;       // leaves of the implicit search tree
constexpr int kMaxStripesPerSub = 1024;
// Per-bucket pointer word of the block permutation (Section 4.2 keeps w_i
// and r_i in one 128-bit word; here one 64-bit word also carries the reader
// count): [w_i - d_i : 25 bits | r_i - d_i + kRBias : 25 bits | readers : 14 bits].
// r_i is biased because failed claims may take it below w_i - 1.
constexpr int kRdBits = 14;
constexpr int kRBits = 25;
constexpr int kWShift = kRdBits + kRBits;                 // 39
constexpr unsigned long long kRBias = 1ull << 16;
constexpr unsigned long long kClaimRead = 1ull - (1ull << kRdBits);   // readers + 1, r - 1
constexpr unsigned long long kClaimWrite = 1ull << kWShift;          // w + 1
constexpr unsigned long long kReadDone = ~0ull;                      // readers - 1
constexpr unsigned long long kMaxRegionBlocks = (1ull << kRBits) - kRBias - 2;
// Reader counts are held per warp (the read claims of a warp's movers on one
// bucket are combined), so a subproblem may have this many mover warps.
constexpr unsigned kMaxReadersPerSub = 16000;             // < 2^kRdBits concurrent readers

// Device status word bits.
constexpr u32 kStatusTimeout = 1u;     // a bounded wait gave up
constexpr u32 kStatusInternal = 2u;    // an invariant check failed
constexpr u32 kStatusCapacity = 4u;    // a fixed-capacity list overflowed

// ---------------------------------------------------------------- traits
// Each element type defines its storage type, its comparable key and the
// block size b in elements.  The paper uses b = max(1, 2^floor(11 - log2 s))
// (about 2 KiB) for CPU caches; here a block is 512 bytes so that the k
// per-bucket buffer blocks of a classification CTA fit in shared memory.

struct TU64 {
    typedef u64 elem_t;
    typedef u64 key_t;
    static constexpr int kId = 0;
    static constexpr int kBlock = 64;                 // 64 x 8 B = 512 B
    static constexpr int kBaseTiny = 4096;             // base case size class sorted by 256-thread CTAs
    static constexpr int kBaseSmall = 8192;            // base case size class sorted by 512-thread CTAs
    static constexpr int kBaseCap = 16384;             // largest bucket sorted in shared memory (128 KiB)
    static constexpr int kSampleMax = 4096;            // largest sample (alpha * leaves) of a step
    __host__ __device__ static inline key_t key(const elem_t& e) { return e; }
    __host__ __device__ static inline elem_t unkey(const key_t& k) { return k; }
    __host__ __device__ static inline u64 key_bits(const key_t& k) { return k; }
    __host__ __device__ static inline u64 sub_key(const key_t& k) { return k; }   // the key's leading word
};

struct TF64 {
    typedef u64 elem_t;     // raw IEEE bits
    typedef u64 key_t;      // order-preserving map of the bits
    static constexpr int kId = 1;
    static constexpr int kBlock = 64;
    static constexpr int kBaseTiny = 4096;
    static constexpr int kBaseSmall = 8192;
    static constexpr int kBaseCap = 16384;
    static constexpr int kSampleMax = 4096;
    __host__ __device__ static inline key_t key(const elem_t& e) {
        return (e >> 63) ? ~e : (e | 0x8000000000000000ull);
    }
    __host__ __device__ static inline elem_t unkey(const key_t& k) {   // inverse of key
        return (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    }
    __host__ __device__ static inline u64 key_bits(const key_t& k) { return k; }
    __host__ __device__ static inline u64 sub_key(const key_t& k) { return k; }
};

struct alignas(16) PairElem {
    u64 k;
    u64 p;
};

struct TPair {
    typedef PairElem elem_t;
    typedef u64 key_t;
    static constexpr int kId = 2;
    static constexpr int kBlock = 32;                 // 32 x 16 B = 512 B
    static constexpr int kBaseTiny = 2048;
    static constexpr int kBaseSmall = 4096;
    static constexpr int kBaseCap = 8192;
    static constexpr int kSampleMax = 4096;
    __host__ __device__ static inline key_t key(const elem_t& e) { return e.k; }
    __host__ __device__ static inline u64 key_bits(const key_t& k) { return k; }
    __host__ __device__ static inline u64 sub_key(const key_t& k) { return k; }
};

// Quartet (Section 5: three key words and one word of associated
// information, compared lexicographically): 32 bytes, key (k0, k1, k2).
struct QKey {
    u64 a, b, c;
};
__host__ __device__ __forceinline__ bool operator<(const QKey& x, const QKey& y) {
    return x.a < y.a || (x.a == y.a && (x.b < y.b || (x.b == y.b && x.c < y.c)));
}
__host__ __device__ __forceinline__ bool operator==(const QKey& x, const QKey& y) {
    return x.a == y.a && x.b == y.b && x.c == y.c;
}
__host__ __device__ __forceinline__ bool operator!=(const QKey& x, const QKey& y) { return !(x == y); }
__host__ __device__ __forceinline__ bool operator>(const QKey& x, const QKey& y) { return y < x; }
__host__ __device__ __forceinline__ bool operator<=(const QKey& x, const QKey& y) { return !(y < x); }
__host__ __device__ __forceinline__ bool operator>=(const QKey& x, const QKey& y) { return !(x < y); }

struct alignas(16) QuartetElem {
    u64 k0, k1, k2;
    u64 p;
};

struct TQuartet {
    typedef QuartetElem elem_t;
    typedef QKey key_t;
    static constexpr int kId = 3;
    static constexpr int kBlock = 16;                 // 16 x 32 B = 512 B
    static constexpr int kBaseTiny = 1024;
    static constexpr int kBaseSmall = 2048;
    static constexpr int kBaseCap = 4096;              // 128 KiB of shared memory
    static constexpr int kSampleMax = 1024;            // 24 KiB of keys
    __host__ __device__ static inline key_t key(const elem_t& e) { return QKey{e.k0, e.k1, e.k2}; }
    __host__ __device__ static inline u64 key_bits(const key_t& k) { return k.a; }
    __host__ __device__ static inline u64 sub_key(const key_t& k) { return k.a; }
};

// 100-byte record (Section 5's 100Bytes), moved in place by the block path:
// key = bytes [0, 10) compared as unsigned bytes, i.e. (big-endian bytes
// 0..7, big-endian bytes 8..9); 4-byte aligned.
struct RKey {
    u64 hi, lo;
};
__host__ __device__ __forceinline__ bool operator<(const RKey& x, const RKey& y) {
    return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
__host__ __device__ __forceinline__ bool operator==(const RKey& x, const RKey& y) { return x.hi == y.hi && x.lo == y.lo; }
__host__ __device__ __forceinline__ bool operator!=(const RKey& x, const RKey& y) { return !(x == y); }
__host__ __device__ __forceinline__ bool operator>(const RKey& x, const RKey& y) { return y < x; }
__host__ __device__ __forceinline__ bool operator<=(const RKey& x, const RKey& y) { return !(y < x); }
__host__ __device__ __forceinline__ bool operator>=(const RKey& x, const RKey& y) { return !(x < y); }

struct alignas(4) RecElem {
    u32 w[25];
};

__host__ __device__ __forceinline__ u32 bswap32(u32 x) {
#ifdef __CUDA_ARCH__
    return __byte_perm(x, 0, 0x0123);
#else
    return (x >> 24) | ((x >> 8) & 0xff00u) | ((x << 8) & 0xff0000u) | (x << 24);
#endif
}

struct TRec {
    typedef RecElem elem_t;
    typedef RKey key_t;
    static constexpr int kId = 4;
    static constexpr int kBlock = 5;                  // 5 x 100 B = 500 B
    static constexpr int kBaseTiny = 256;
    static constexpr int kBaseSmall = 512;
    static constexpr int kBaseCap = 1024;              // 100 KB of shared memory
    static constexpr int kSampleMax = 2048;            // 32 KiB of keys
    __host__ __device__ static inline key_t key(const elem_t& e) {
        return RKey{((u64)bswap32(e.w[0]) << 32) | bswap32(e.w[1]), (u64)(((e.w[2] & 0xffu) << 8) | ((e.w[2] >> 8) & 0xffu))};
    }
    __host__ __device__ static inline u64 key_bits(const key_t& k) { return k.hi; }
    __host__ __device__ static inline u64 sub_key(const key_t& k) { return k.hi; }
};

// Warp shuffle of a key of any of the types above.
__device__ __forceinline__ u64 shfl_xor_key(u64 v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ QKey shfl_xor_key(const QKey& v, int o) {
    return QKey{__shfl_xor_sync(0xffffffffu, v.a, o), __shfl_xor_sync(0xffffffffu, v.b, o),
                __shfl_xor_sync(0xffffffffu, v.c, o)};
}
__device__ __forceinline__ RKey shfl_xor_key(const RKey& v, int o) {
    return RKey{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// ------------------------------------------------------------ descriptors
// One subproblem (a bucket of the previous level, or the whole input) of a
// chunk of work at one recursion level.
struct SubDesc {
    u64 begin;          // absolute element offset
    u64 n;              // elements
    u32 stripe_begin;   // first stripe in the chunk's stripe table
    u32 num_stripes;
    u32 k_target;       // planned number of leaves (power of two)
    u32 alpha;          // oversampling factor
    u32 level;
    // written by the sampling kernel
    u32 log_leaves;
    u32 eq;             // equality buckets on
    u32 nbuckets;       // leaves, or 2*leaves - 1 with equality buckets
    // written by the prefix kernel
    u64 blocks_total;   // full blocks produced by local classification
};

struct StripeDesc {
    u64 begin;          // absolute element index; (begin - sub.begin) % b == 0
    u64 end;
    u64 pool_off;       // element offset of this stripe's leftover area
    u32 sub;            // index of the subproblem in the chunk
    u32 pool_cap;
};

struct Task {           // a subproblem emitted for the next level
    u64 begin;
    u64 n;
};

struct FixItem {        // a bucket region whose empty blocks must be moved (Appendix A)
    u32 sub;
    u32 bucket;
};

// Device-side counters of one chunk.
struct ChunkCounters {
    u32 stripe_next;    // dynamic stripe scheduler for classification
    u32 fix_count;      // entries in the fix list
    u32 ticket;         // cleanup ticket dispenser
    u32 next_count;     // tasks emitted for the next level
    u32 status;         // error bits
    u32 guard_line;     // first failed bounds guard: source line (0 = none)
    u32 guard_hits;     // number of failed bounds guards
    u32 base_next;      // base case: next entry of the task list (zero between launches)
    u32 base_done;      // base case: CTAs of the launch that have taken their last entry
    u32 pad;
    u64 guard_a, guard_b;   // operands of the first failed guard
    u32 base_small;     // base-case tasks of the small size class
    u32 base_large;     // base-case tasks of the large size class
    u32 base_tiny;      // base-case tasks of the tiny size class
    u32 copy_count;     // entries of the copy list (a sort whose result goes to another buffer)
    u64 blocks_moved;
    u64 blocks_skipped;
    u64 fix_blocks;
    u64 base_buckets;
};

// State of a sort whose recursion levels are planned on the device (the
// asynchronous ips4o_sort): the subproblems of the current level are a
// queue in device memory, each round takes the next chunk of it, and the
// cleanup appends the buckets that must recurse to the other queue.
struct LoopState {
    Task* cur_q;            // subproblems of the current level
    Task* next_q;           // subproblems of the next level (appended by the cleanup)
    u32 cur_count;          // entries of cur_q
    u32 cur_pos;            // entries of cur_q already planned
    u32 next_count;         // entries of next_q
    u32 level;
    u32 nsub, nstr;         // the chunk of the current round
    u32 bstride;            // cleanup tickets per subproblem of the chunk
    u32 cta_cleanup;        // 1: one CTA per bucket in the cleanup (subproblems with many stripes)
    u32 status;             // error bits of the whole call
    u32 guard_line, guard_hits, levels;
    u64 guard_a, guard_b;
    u64 stripe_len;         // stripe length of the current level
    u64 blocks_moved, blocks_skipped, fix_blocks, base_buckets, elements_distributed, subproblems, chunks;
    u32 fallback_tasks;     // subproblems left to the segment scheduler after the last round
    u32 strict;             // 1: the strictly in-place recursion (buckets are marked, not queued)
    u32 marks;              // strict: buckets marked by the current batch
    u32 carry_desc;         // strict: the piece that reaches past the scanned window holds a descent
    u64 batch_begin;        // strict: first element of the current batch's subproblems
    u64 scan_pos, scan_end; // strict: the window [scan_pos, scan_end) of the current scan pass
    u64 carry_head;         // strict: head of the piece that reaches past the window (kNoHead: none)
};

constexpr u64 kNoHead = ~0ull;
constexpr u64 kCopyChunk = 1u << 16;   // elements per entry of the result copy list

// Summary of one tile of the strict recursion's bucket-head scan.
struct ScanTile {
    u64 first_head, last_head;   // absolute positions of the tile's first and last head (kNoHead: none)
    u32 desc_first;              // a descent before the first head (the whole tile when it has none)
    u32 desc_last;               // a descent after the last head
    u32 next_head_tile;          // the first tile at or after this one with a head (tile count: none)
    u32 desc_before;             // tiles before this one whose desc_first is set
};

// Pointers into the workspace for one key type.
template <class T>
struct Workspace {
    typedef typename T::elem_t elem_t;
    typedef typename T::key_t key_t;
    SubDesc* subs;            // [max_sub]
    StripeDesc* stripes;      // [max_stripes]
    key_t* tree;              // [max_sub][256]   implicit search tree a[1..L-1]
    key_t* spl;               // [max_sub][256]   sorted splitters s_1..s_{L-1}
    u64* bstart;              // [max_sub][257]   bucket starts relative to sub begin
    u32* delim;               // [max_sub][257]   delimiter block indices d_i
    u64* wr;                  // [max_sub][256]   packed w_i, r_i, reader count (see kWShift)
    u32* flags;               // [max_sub][256]   cleanup hand-over flags
    u32* exhausted;           // [max_sub][8]     bitmap of buckets without unprocessed blocks
    u32* movers;              // [max_sub]        CTAs working on the block permutation of each subproblem
    u32* region_full;         // [max_sub][256]   full blocks inside region [d_i, d_{i+1})
    u32* bucket_full;         // [max_sub][256]   full blocks of bucket i (all stripes)
    u32* counts;              // [max_stripes][256] elements per bucket per stripe
    u32* lscan;               // [max_stripes][256] leftover offset per bucket in the stripe area
    u32* stripe_full;         // [max_stripes]     full blocks flushed by the stripe
    FixItem* fix_list;        // [max_sub * 256]
    elem_t* pool;             // [pool_cap]        partially filled buffer blocks (leftovers)
    elem_t* overflow;         // [max_sub][b]      overflow block per subproblem
    Task* next_tasks;         // [next_cap]
    Task* base_small;         // [max_sub * 256] buckets for the small base case
    Task* base_large;         // [max_sub * 256] buckets for the large base case
    Task* base_tiny;          // [max_sub * 256] buckets for the tiny base case
    Task* init_tasks;         // [init_cap]      segments sorted by the base case alone / scheduler queue
    u32* init_count;          // [4]             tiny / small / large entries of init_tasks; queue length, cursor
    u32* hist;                // [65]            scheduler queue built on the device: size groups
    Task* stacks;             // [max_sub][stack_cap] scheduler: buckets each CTA still has to distribute
    ChunkCounters* ctr;       // [1]
    Task* next_tasks2;        // [next_cap]      the second level queue of the device-planned recursion
    LoopState* ls;            // [1] device-planned recursion; null when the host plans the levels
    u32* stripe_order;        // [max_stripes] device-planned rounds: the order the classification takes stripes
    Task* copy_tasks;         // [copy_cap] ranges final in arr that the result copy moves to out
    elem_t* out;              // where the base case writes its sorted buckets (null: in place)
    key_t* scan_max;          // [scan_cap] strict recursion: largest key per scan tile, then the prefix before it
    ScanTile* scan_tiles;     // [scan_cap] strict recursion: heads and descents per scan tile
    u32 max_sub, max_stripes;
    u64 pool_cap, next_cap, init_cap, stack_cap, scan_cap, copy_cap;
};

// ------------------------------------------------------------ primitives
__device__ __forceinline__ u32 smem_addr(const void* p) {
    return (u32)__cvta_generic_to_shared(p);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem);

template <>
__device__ __forceinline__ void cp_async<8>(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(smem)), "l"(gmem)
                 : "memory");
}
template <>
__device__ __forceinline__ void cp_async<16>(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem)), "l"(gmem)
                 : "memory");
}
template <>
__device__ __forceinline__ void cp_async<4>(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
template <>
__device__ __forceinline__ void cp_async<32>(void* smem, const void* gmem) {
    cp_async<16>(smem, gmem);
    cp_async<16>((char*)smem + 16, (const char*)gmem + 16);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ u64 atom_add_acq_rel(u64* p, u64 v) {
    u64 old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ u64 atom_add_acquire(u64* p, u64 v) {
    u64 old;
    asm volatile("atom.acquire.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ u64 ld_acquire64(const u64* p) {
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_add_release64(u64* p, u64 v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_add_relaxed64(u64* p, u64 v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u32 pk_readers(u64 x) { return (u32)(x & ((1ull << kRdBits) - 1)); }
__device__ __forceinline__ long long pk_r(u64 x) {
    return (long long)((x >> kRdBits) & ((1ull << kRBits) - 1)) - (long long)kRBias;
}
__device__ __forceinline__ long long pk_w(u64 x) { return (long long)(x >> kWShift); }
__device__ __forceinline__ u32 ld_acquire(const u32* p) {
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(u32* p, u32 v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_release(u32* p, u32 v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ u32 ld_relaxed(const u32* p) {
    u32 v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ u64 ld_relaxed64(const u64* p) {
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_add_relaxed(u32* p, u32 v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ u64 ceil_div(u64 a, u64 b) { return (a + b - 1) / b; }

// Shared-memory layouts round every region's start up to 16 bytes, so that
// any key or counter type may follow an element area of any size.
constexpr size_t a16(size_t x) { return (x + 15) / 16 * 16; }

__device__ __forceinline__ void set_status(ChunkCounters* c, u32 bits) { atomicOr(&c->status, bits); }

// A failed bounds guard: the access is skipped, the chunk reports an
// internal error, and the first failure's line and operands are kept.
static __device__ __noinline__ void guard_fail(ChunkCounters* c, u32 line, u64 a, u64 b) {
    if (atomicAdd(&c->guard_hits, 1u) == 0) {
        c->guard_line = line;
        c->guard_a = a;
        c->guard_b = b;
    }
    atomicOr(&c->status, kStatusInternal);
}
// Bounded wait until *flag becomes non-zero (acquire): true when it did,
// false after spin_limit polls (the caller reports IPS4O_ERR_TIMEOUT).
__device__ __forceinline__ bool wait_flag_set(const u32* flag, u32 spin_limit) {
    u32 it = 0;
    while (ld_acquire(flag) == 0) {
        if (++it > spin_limit) return false;
        __nanosleep(32);
    }
    return true;
}

#define IPS4O_GUARD(ctr, cond, a, b) ((cond) ? true : (guard_fail((ctr), __LINE__, (u64)(a), (u64)(b)), false))

// ------------------------------------------------ splitter lookup table
// A shortcut for the tree descent of Section 4.1 with the same result.
// Let i(e) = #{t in [1, L-1] : s_t <= e} be the leaf index the descent
// returns (s_1 <= ... <= s_{L-1}, the largest repeated as padding).  Keys
// from s_1 upwards are mapped monotonically onto at most kLutCells cells
// (linear cells of 2^shift keys over [s_1, s_{L-1}], the last one open
// upwards, or logarithmic cells for keys spread over many orders of
// magnitude); one more entry stands for the keys below s_1.  Entry c holds
// lo_c = i(first key of cell c) and hi_c = i(first key of cell c + 1)
// (L - 1 for the last cell), so that since i is non-decreasing every key e
// of the cell has
//     i(e) = lo_c + #{t in (lo_c, hi_c] : s_t <= e}.
// Where the cells separate the splitters, most keys take one table lookup
// and at most one comparison; cells with more splitters take a binary
// search over (lo_c, hi_c].
constexpr int kLutCells = 4096;
constexpr int kLutBits = 12;                    // log2(kLutCells)
constexpr int kLutMinLevels = 5;                // smaller trees keep the descent

// Index of the lowest set bit of x plus one (0 for x == 0).
__host__ __device__ __forceinline__ int ffs32(u32 x) {
#ifdef __CUDA_ARCH__
    return __ffs((int)x);
#else
    return __builtin_ffs((int)x);
#endif
}

// The first bucket at or after start (cyclically over the 256 bits) that the
// exhausted bitmap exw of the block permutation does not mark; 0xffffffff
// when every bucket is marked.
__host__ __device__ __forceinline__ u32 first_live_bucket(const u32 (&exw)[8], u32 start) {
    for (u32 step = 0; step < 8 * 32;) {
        const u32 c = (start + step) & 255u;
        const u32 free_bits = ~exw[c >> 5] >> (c & 31);
        if (free_bits) return c + (u32)(ffs32(free_bits) - 1);   // stays inside word c >> 5
        step += 32 - (c & 31);
    }
    return 0xffffffffu;
}

// Bit length of x (0 for x == 0).
__host__ __device__ __forceinline__ u32 bitlen64(u64 x) {
#ifdef __CUDA_ARCH__
    return 64u - (u32)__clzll((long long)x);
#else
    u32 b = 0;
    for (; x != 0; x >>= 1) ++b;
    return b;
#endif
}

// shift such that (top - base) >> shift < kLutCells (base <= top).
__host__ __device__ __forceinline__ u32 lut_shift(u64 base, u64 top) {
    const u32 bits = bitlen64(top - base);
    return bits > (u32)kLutBits ? bits - (u32)kLutBits : 0u;
}

// Cell of key e: kLutCells for e < base, else min((e - base) >> shift, kLutCells - 1).
__host__ __device__ __forceinline__ u32 lut_cell(u64 e, u64 base, u32 shift) {
    const u64 d = (e - base) >> shift;
    const u32 c = d < (u64)(kLutCells - 1) ? (u32)d : (u32)(kLutCells - 1);
    return e < base ? (u32)kLutCells : c;
}

// First key of cell c (c < kLutCells); false when it lies above the key
// domain (no key maps to the cell).
__host__ __device__ __forceinline__ bool lut_cell_start(u32 c, u64 base, u32 shift, u64* start) {
    const u64 off = (u64)c << shift;           // c < 2^12 and shift <= 52: no overflow
    if (off > ~base) return false;
    *start = base + off;
    return true;
}

// Logarithmic cells for keys spread over many orders of magnitude: with
// d = e - base, cell d for d < 2^(m+1), otherwise the bit length of d and
// the m bits after its leading one, m = kLutLogMant (64 cells per octave,
// 3776 cells for all of [0, 2^64)).  kLutCells again stands for e < base.
constexpr u32 kLutLogMant = 6;
__host__ __device__ __forceinline__ u32 lut_cell_log(u64 e, u64 base) {
    const u64 d = e - base;
    const u32 bl = bitlen64(d);
    const u32 c = bl <= kLutLogMant + 1
                      ? (u32)d
                      : ((bl - kLutLogMant) << kLutLogMant) |
                            (u32)((d >> (bl - 1 - kLutLogMant)) & ((1u << kLutLogMant) - 1));
    return e < base ? (u32)kLutCells : c;
}

__host__ __device__ __forceinline__ bool lut_cell_start_log(u32 c, u64 base, u64* start) {
    u64 off = c;
    if (c >= (1u << kLutLogMant)) {
        const u32 o = c >> kLutLogMant, mant = c & ((1u << kLutLogMant) - 1);
        if (o + kLutLogMant > 64) return false;       // above every 64-bit d
        off = (u64)((1u << kLutLogMant) | mant) << (o - 1);
    }
    if (off > ~base) return false;
    *start = base + off;
    return true;
}

// Linear cells aligned to multiples of 2^shift of the key domain: cell
// c(e) = (e >> shift) - c0 with c0 = s_1 >> shift, clamped to
// [0, kLutCells - 1], so cell 0 also takes every key below its range and the
// last cell is open upwards.  lut_abs_shift picks shift such that s_1 and
// s_{L-1} are at most kLutCells - 1 cells apart.  For shift >= 32 the cell
// follows from the key's high 32 bits alone (lut_cell_abs_hi).
__host__ __device__ __forceinline__ u32 lut_abs_shift(u64 base, u64 top) {
    u32 sh = lut_shift(base, top);
    if ((top >> sh) - (base >> sh) >= (u64)kLutCells) ++sh;
    return sh;
}
__host__ __device__ __forceinline__ u32 lut_cell_abs(u64 e, u64 c0, u32 shift) {
    const u64 h = e >> shift;
    const u64 d = h - c0;
    return h < c0 ? 0u : (d < (u64)(kLutCells - 1) ? (u32)d : (u32)(kLutCells - 1));
}
__host__ __device__ __forceinline__ u32 lut_cell_abs_hi(u32 ehi, u32 c0, u32 shift_hi) {
    const u32 h = ehi >> shift_hi;
    const u32 d = h - c0;
    return h < c0 ? 0u : (d < (u32)(kLutCells - 1) ? d : (u32)(kLutCells - 1));
}
// First key of cell c (0 for cell 0, which holds every key below cell 1);
// false when it lies above the key domain (no key maps to the cell).
__host__ __device__ __forceinline__ bool lut_cell_start_abs(u32 c, u64 c0, u32 shift, u64* start) {
    if (c == 0) { *start = 0; return true; }
    const u64 h = c0 + c;
    if (h < c0) return false;
    if (shift > 0 && (h >> (64 - shift)) != 0) return false;
    *start = h << shift;
    return true;
}

// i(e) from the table entry (lo | hi << 8) and the sorted splitters spl[1..L-1].
__host__ __device__ __forceinline__ int lut_refine(u64 e, u32 ent, const u64* spl) {
    const int lo = (int)(ent & 0xffu), hi = (int)(ent >> 8);
    const int nx = lo + 1 < kMaxLeaves ? lo + 1 : kMaxLeaves - 1;
    int i = lo + ((hi > lo && spl[nx] <= e) ? 1 : 0);
    if (hi > lo + 1) {
        int a = lo, b = hi;                    // i(e) lies in [a, b]
        while (a < b) {
            const int m = (a + b + 1) >> 1;
            if (spl[m] <= e) a = m;
            else b = m - 1;
        }
        i = a;
    }
    return i;
}

// Bucket of key e (Section 3): descend the implicit tree a[1..L-1]
// (a_1 = s_{L/2}, children of a_j are a_{2j}, a_{2j+1}) with j = 2j + (a_j <= e);
// the leaf index j - L is the number of splitters <= e, so that
// s_i <= e < s_{i+1}.  With equality buckets (Section 4.4) one more
// comparison against s_i separates the keys equal to s_i (bucket 2i-1)
// from those strictly between s_i and s_{i+1} (bucket 2i).
template <class K>
__device__ __forceinline__ int classify_key(const K& e, const K* tree, const K* spl, int log_leaves, bool eq) {
    int j = 1;
#pragma unroll
    for (int l = 0; l < 8; ++l)
        if (l < log_leaves) j = 2 * j + (tree[j] <= e ? 1 : 0);
    int i = j - (1 << log_leaves);
    if (!eq) return i;
    return 2 * i - ((i > 0 && spl[i] == e) ? 1 : 0);
}

// Block-wide exclusive scan of one value per thread for the first
// `count` threads (count <= blockDim.x, blockDim.x multiple of 32).
// Returns the exclusive prefix; *total receives the sum.  Uses `tmp`
// (>= 32 entries) of shared memory and two __syncthreads.
template <typename V>
__device__ __forceinline__ V block_exclusive_scan(V v, V* tmp, V* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    V x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        V t = lane < nwarps ? tmp[lane] : V(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            V y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        tmp[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    V warp_prefix = warp > 0 ? tmp[warp - 1] : V(0);
    *total = tmp[nwarps - 1];
    return warp_prefix + x - v;
}

}  // namespace ips4o
