// ips4o_strict.cuh — the strictly in-place recursion of Section 4.6.
//
// The device-planned sort keeps the subproblems of a level in queues whose
// length grows with n / (base case), the O(log n)-type term of Theorem 2.
// Section 4.6 removes it: a partitioning step stores the largest element of
// each bucket it leaves for later in the bucket's first slot, so that the end
// of that bucket is the first later position holding a larger key (the
// paper's searchNextLargest), and the recursion needs no stack.
//
// Here the array itself describes the work left.  Scanning a window from the
// left, a position is a bucket head exactly when its key is larger than every
// key before it: buckets are ordered (each key of a later bucket is larger
// than each key of an earlier one), and a marked bucket holds no key above its
// head.  The piece from one head to the next is then either a marked bucket
// still to be sorted or a run of equal keys inside a part already sorted; the
// first holds a descent (a key followed by a smaller one) unless all its keys
// are equal, the second never does.  Pieces with a descent become the next
// batch of subproblems, distributed by the rounds of the device-planned sort
// with its queues switched off: buckets small enough for the base case are
// sorted within the round that makes them, and larger ones are marked by
// k_mark.  The host loop follows the paper's: a position behind which all is
// sorted moves over the array window by window, and a window is rescanned
// from the batch's first subproblem when the batch marked new buckets.  The
// window and every list have sizes independent of n.
#pragma once

#include "ips4o_rounds.cuh"

namespace ips4o {

constexpr u32 kScanTPB = 256;
constexpr u32 kScanIPT = 8;
constexpr u32 kScanTile = kScanTPB * kScanIPT;      // elements per tile of the head scan
constexpr u64 kScanWindowBytes = 1ull << 30;        // default window: 1 GiB of elements

// Warp shuffle up of a key of any of the element types' key types.
__device__ __forceinline__ u64 shfl_up_key(u64 v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ QKey shfl_up_key(const QKey& v, int o) {
    return QKey{__shfl_up_sync(0xffffffffu, v.a, o), __shfl_up_sync(0xffffffffu, v.b, o),
                __shfl_up_sync(0xffffffffu, v.c, o)};
}
__device__ __forceinline__ RKey shfl_up_key(const RKey& v, int o) {
    return RKey{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}

// Block-wide exclusive prefix maximum of (v, has) over the threads of a CTA
// of TPB threads; has = false stands for "no key" (below every key).  Warp
// scans by shuffles, then the warps' totals (s_k, s_h: TPB / 32 entries).
template <class K, int TPB>
__device__ __forceinline__ void block_excl_max(K v, bool has, K* s_k, u32* s_h, K* out, bool* out_has) {
    constexpr int NW = TPB / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    K inc = v;
    bool ih = has;
    for (int o = 1; o < 32; o <<= 1) {
        const K a = shfl_up_key(inc, o);
        const bool ah = __shfl_up_sync(0xffffffffu, (u32)ih, o) != 0;
        if (lane >= o && ah && (!ih || inc < a)) {
            inc = a;
            ih = true;
        }
    }
    if (lane == 31) {
        s_k[warp] = inc;
        s_h[warp] = ih;
    }
    // the lane's exclusive value within the warp
    K ex = shfl_up_key(inc, 1);
    bool eh = __shfl_up_sync(0xffffffffu, (u32)ih, 1) != 0 && lane > 0;
    __syncthreads();
    for (int w = 0; w < NW; ++w) {
        if (w >= warp) break;
        if (s_h[w] && (!eh || ex < s_k[w])) {
            ex = s_k[w];
            eh = true;
        }
    }
    *out = ex;
    *out_has = eh;
    __syncthreads();
}

// Block-wide maximum of (v, has), returned to every thread.
template <class K, int TPB>
__device__ __forceinline__ void block_max(K v, bool has, K* s_k, u32* s_h, K* out, bool* out_has) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const K ov = shfl_xor_key(v, o);
        const bool oh = __shfl_xor_sync(0xffffffffu, (u32)has, o) != 0;
        if (oh && (!has || v < ov)) {
            v = ov;
            has = true;
        }
    }
    if (lane == 0) {
        s_k[warp] = v;
        s_h[warp] = has;
    }
    __syncthreads();
    K m = v;
    bool mh = false;
    for (int w = 0; w < TPB / 32; ++w)
        if (s_h[w] && (!mh || m < s_k[w])) {
            m = s_k[w];
            mh = true;
        }
    *out = m;
    *out_has = mh;
    __syncthreads();
}

// A piece with a descent found by the scan: a subproblem of the next batch,
// or a base-case task when it is small enough (a marked bucket never is: the
// round that made it sorted all buckets of at most rec_cap elements).
template <class T>
__device__ __forceinline__ void strict_emit(const Workspace<T>& ws, Task t, u32 rec_cap) {
    if (t.n < 2) return;
    if (t.n <= (u64)rec_cap) {
        emit_bucket<T>(ws, t, rec_cap);
        return;
    }
    LoopState* ls = ws.ls;
    const u32 idx = atomicAdd(&ls->cur_count, 1u);
    if (idx < ws.next_cap) ls->cur_q[idx] = t;
    else atomicOr(&ls->status, kStatusCapacity);
    atomicMin((unsigned long long*)&ls->batch_begin, (unsigned long long)t.begin);
}

// The loop state of a strict sort of n elements: one batch, the whole input.
template <class T>
__global__ void k_strict_init(Workspace<T> ws, u64 n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        LoopState* ls = ws.ls;
        *ls = LoopState{};
        ls->strict = 1;
        ls->cur_q = ws.next_tasks;
        ls->next_q = ws.next_tasks2;
        ls->cur_q[0] = Task{0, n};
        ls->cur_count = 1;
        ls->batch_begin = 0;
        ls->scan_pos = 0;
        ls->carry_head = kNoHead;
        *ws.ctr = ChunkCounters{};
    }
}

// Section 4.6's mark: after a round's cleanup, every bucket of its chunk
// that will be distributed again (more than rec_cap elements, not an
// equality bucket) gets its largest element in its first slot.  One CTA per
// bucket, taken in turn.
template <class T, int TPB>
__global__ void __launch_bounds__(TPB) k_mark(typename T::elem_t* arr, Workspace<T> ws, u32 rec_cap) {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    constexpr int U = sizeof(K) <= 8 ? 8 : 4;       // independent loads in flight per thread
    __shared__ K s_k[TPB / 32];
    __shared__ u32 s_h[TPB / 32];
    __shared__ u64 s_p[TPB / 32];
    const LoopState* ls = ws.ls;
    const u32 nsub = ls->nsub, bstride = ls->bstride;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    u32 marks = 0;
    for (u32 t = blockIdx.x; t < nsub * bstride; t += gridDim.x) {
        const u32 j = t / bstride, b = t % bstride;
        const SubDesc& sub = ws.subs[j];
        if (b >= sub.nbuckets || (sub.eq && (b & 1))) continue;
        const u64* bstart = ws.bstart + (u64)j * (kMaxBuckets + 1);
        const u64 Bb = bstart[b], Eb = bstart[b + 1];
        if (Eb <= Bb || Eb - Bb <= (u64)rec_cap) continue;
        const u64 lo = sub.begin + Bb, hi = sub.begin + Eb;
        K best = T::key(arr[lo]);
        u64 bp = lo;
        for (u64 i0 = lo + tid; i0 < hi; i0 += (u64)TPB * U) {
            K k[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + (u64)u * TPB < hi) k[u] = T::key(arr[i0 + (u64)u * TPB]);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + (u64)u * TPB < hi && best < k[u]) {
                    best = k[u];
                    bp = i0 + (u64)u * TPB;
                }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const K ok = shfl_xor_key(best, o);
            const u64 op = __shfl_xor_sync(0xffffffffu, bp, o);
            if (best < ok) {
                best = ok;
                bp = op;
            }
        }
        if (lane == 0) {
            s_k[warp] = best;
            s_p[warp] = bp;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < TPB / 32; ++w)
                if (best < s_k[w]) {
                    best = s_k[w];
                    bp = s_p[w];
                }
            if (bp != lo) {
                const E x = arr[lo];
                arr[lo] = arr[bp];
                arr[bp] = x;
            }
            ++marks;
        }
        __syncthreads();
    }
    (void)s_h;
    if (tid == 0 && marks) atomicAdd(&ws.ls->marks, marks);
}

// Start of a scan pass (one thread): fold the batch's counters; after a
// batch that marked buckets, go back to its first subproblem; then the
// window [scan_pos, scan_pos + window).
template <class T>
__global__ void k_scan_begin(Workspace<T> ws, u64 n, u64 window) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        LoopState* ls = ws.ls;
        fold_counters(ls, ws.ctr);
        if (ls->marks) {
            ls->scan_pos = ls->batch_begin;
            ls->carry_head = kNoHead;
            ls->carry_desc = 0;
            ls->marks = 0;
        }
        ls->cur_count = 0;
        ls->cur_pos = 0;
        ls->batch_begin = ~0ull;
        ls->scan_end = ls->scan_pos + window < n ? ls->scan_pos + window : n;
        ls->nsub = 0;
    }
}

// Largest key of every tile of the window.
template <class T>
__global__ void __launch_bounds__(kScanTPB) k_scan_max(const typename T::elem_t* arr, Workspace<T> ws) {
    typedef typename T::key_t K;
    __shared__ K s_k[kScanTPB / 32];
    __shared__ u32 s_h[kScanTPB / 32];
    const u64 s = ws.ls->scan_pos, e = ws.ls->scan_end;
    const u64 nt = e > s ? (e - s + kScanTile - 1) / kScanTile : 0;
    for (u64 t = blockIdx.x; t < nt; t += gridDim.x) {
        const u64 base = s + t * kScanTile;
        const u32 len = (u32)(e - base < kScanTile ? e - base : kScanTile);
        K k[kScanIPT];
#pragma unroll
        for (u32 q = 0; q < kScanIPT; ++q)
            if (threadIdx.x + q * kScanTPB < len) k[q] = T::key(arr[base + threadIdx.x + q * kScanTPB]);
        K m = key_min<K>();
        bool has = false;
#pragma unroll
        for (u32 q = 0; q < kScanIPT; ++q)
            if (threadIdx.x + q * kScanTPB < len && (!has || m < k[q])) {
                m = k[q];
                has = true;
            }
        K bm;
        bool bh;
        block_max<K, kScanTPB>(m, has, s_k, s_h, &bm, &bh);
        if (threadIdx.x == 0) ws.scan_max[t] = bm;
    }
}

// Exclusive prefix maximum over the window's tiles, starting from the key of
// the piece carried over from the previous window (one CTA of 1024 threads);
// tile 0 has no prefix when nothing is carried.
template <class T>
__global__ void __launch_bounds__(1024) k_scan_prefix(const typename T::elem_t* arr, Workspace<T> ws) {
    typedef typename T::key_t K;
    __shared__ K s_k[1024];
    __shared__ u32 s_h[1024];
    const u64 s = ws.ls->scan_pos, e = ws.ls->scan_end, carry = ws.ls->carry_head;
    const u64 nt = e > s ? (e - s + kScanTile - 1) / kScanTile : 0;
    const u64 per = (nt + 1023) / 1024;
    const u64 t0 = (u64)threadIdx.x * per, t1 = t0 + per < nt ? t0 + per : nt;
    K agg = key_min<K>();
    bool ah = false;
    for (u64 t = t0; t < t1; ++t) {
        const K k = ws.scan_max[t];
        if (!ah || agg < k) {
            agg = k;
            ah = true;
        }
    }
    K ex;
    bool eh;
    block_excl_max<K, 1024>(agg, ah, s_k, s_h, &ex, &eh);
    if (carry != kNoHead) {
        const K c = T::key(arr[carry]);
        if (!eh || ex < c) {
            ex = c;
            eh = true;
        }
    }
    for (u64 t = t0; t < t1; ++t) {
        const K k = ws.scan_max[t];
        ws.scan_max[t] = eh ? ex : k;          // tile 0 without a prefix: unused
        if (!eh || ex < k) {
            ex = k;
            eh = true;
        }
    }
}

// Heads and descents of every tile: pieces that start and end inside the
// tile and hold a descent are emitted at once; the tile's first and last
// heads and the descents around them go to its summary for k_scan_link.
template <class T>
__global__ void __launch_bounds__(kScanTPB) k_scan_heads(const typename T::elem_t* arr, Workspace<T> ws, u32 rec_cap) {
    typedef typename T::key_t K;
    constexpr u32 IPT = kScanIPT;
    __shared__ K s_k[kScanTPB];
    __shared__ u32 s_h[kScanTPB];
    __shared__ u32 s_cnt[kScanTPB / 32 + 1];
    __shared__ unsigned char s_desc[kScanTile + 1];
    __shared__ unsigned short s_start[kScanTile + 2];
    const LoopState* ls = ws.ls;
    const u64 s = ls->scan_pos, e = ls->scan_end, carry = ls->carry_head;
    const u64 nt = e > s ? (e - s + kScanTile - 1) / kScanTile : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (u64 t = blockIdx.x; t < nt; t += gridDim.x) {
        const u64 base = s + t * kScanTile;
        const u32 len = (u32)(e - base < kScanTile ? e - base : kScanTile);
        for (u32 i = tid; i <= kScanTile; i += kScanTPB) s_desc[i] = 0;
        const u32 i0 = (u32)tid * IPT;
        K k[IPT];
        K agg = key_min<K>();
        bool ah = false;
#pragma unroll
        for (u32 q = 0; q < IPT; ++q)
            if (i0 + q < len) {
                k[q] = T::key(arr[base + i0 + q]);
                if (!ah || agg < k[q]) {
                    agg = k[q];
                    ah = true;
                }
            }
        K m;
        bool mh;
        block_excl_max<K, kScanTPB>(agg, ah, s_k, s_h, &m, &mh);
        const bool tile_has = !(t == 0 && carry == kNoHead);
        if (tile_has) {
            const K ex = ws.scan_max[t];
            if (!mh || m < ex) {
                m = ex;
                mh = true;
            }
        }
        // the element before this thread's first one, when it belongs to a piece of the scan
        K pk = key_min<K>();
        const bool pok = i0 < len && (base + i0 > s || carry != kNoHead);
        if (pok) pk = T::key(arr[base + i0 - 1]);
        u32 hmask = 0, dmask = 0;
#pragma unroll
        for (u32 q = 0; q < IPT; ++q) {
            if (i0 + q >= len) break;
            if (!mh || m < k[q]) {
                m = k[q];
                mh = true;
                hmask |= 1u << q;
            } else {
                const bool ok = q > 0 || pok;
                const K prev = q > 0 ? k[q > 0 ? q - 1 : 0] : pk;
                if (ok && k[q] < prev) dmask |= 1u << q;
            }
        }
        // heads before this thread's: block exclusive sum of the head counts
        const u32 nh = __popc(hmask);
        u32 incl = nh;
        for (int o = 1; o < 32; o <<= 1) {
            const u32 v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_cnt[warp] = incl;
        __syncthreads();
        u32 before = incl - nh, total = 0;
        for (int w = 0; w < (int)(kScanTPB / 32); ++w) {
            if (w < warp) before += s_cnt[w];
            total += s_cnt[w];
        }
        // piece index of each element: heads at or before it (0: the piece
        // that started before the tile)
        u32 seg = before;
#pragma unroll
        for (u32 q = 0; q < IPT; ++q) {
            if ((hmask >> q) & 1u) {
                ++seg;
                s_start[seg] = (unsigned short)(i0 + q);
            }
            if ((dmask >> q) & 1u) s_desc[seg] = 1;
        }
        __syncthreads();
        for (u32 g = 1 + tid; g < total; g += kScanTPB)
            if (s_desc[g]) strict_emit<T>(ws, Task{base + s_start[g], (u64)s_start[g + 1] - s_start[g]}, rec_cap);
        if (tid == 0) {
            ScanTile st;
            st.first_head = total ? base + s_start[1] : kNoHead;
            st.last_head = total ? base + s_start[total] : kNoHead;
            st.desc_first = s_desc[0];
            st.desc_last = total ? s_desc[total] : s_desc[0];
            ws.scan_tiles[t] = st;
        }
        __syncthreads();
    }
}

// Pieces that cross tiles (one CTA of 1024 threads): each starts at the last
// head of a tile (or is the piece carried into the window) and ends at the
// first head of a later tile; the tiles in between have no head.  Two scans
// over the tiles give every tile the next tile with a head and the number of
// earlier tiles with a descent before their first head, so each piece's end
// and descent are found in constant time.  The piece that reaches the end of
// the window is carried into the next one, or ends at n.
template <class T>
__global__ void __launch_bounds__(1024) k_scan_link(Workspace<T> ws, u64 n, u32 rec_cap) {
    constexpr int TPB = 1024;
    __shared__ u32 s_tmp[32];
    __shared__ u32 s_nh[TPB];
    __shared__ u64 s_head;
    __shared__ u32 s_desc, s_set;
    LoopState* ls = ws.ls;
    const u64 s = ls->scan_pos, e = ls->scan_end, carry = ls->carry_head;
    const u32 cdesc = ls->carry_desc;
    const u32 nt = (u32)(e > s ? (e - s + kScanTile - 1) / kScanTile : 0);
    const int tid = threadIdx.x;
    if (tid == 0) s_set = 0;
    // this thread's tiles [t0, t1): descents before a first head, first tile with a head
    const u32 per = (nt + TPB - 1) / TPB;
    const u32 t0 = (u32)tid * per < nt ? (u32)tid * per : nt, t1 = t0 + per < nt ? t0 + per : nt;
    u32 c = 0, fh = nt;
    for (u32 t = t0; t < t1; ++t) {
        const ScanTile tl = ws.scan_tiles[t];
        c += tl.desc_first ? 1u : 0u;
        if (fh == nt && tl.first_head != kNoHead) fh = t;
    }
    u32 tot;
    u32 pd = block_exclusive_scan<u32>(c, s_tmp, &tot);
    // smallest first-head tile of the threads after this one (suffix minimum)
    s_nh[tid] = fh;
    __syncthreads();
    for (int off = 1; off < TPB; off <<= 1) {
        const u32 o = tid + off < TPB ? s_nh[tid + off] : nt;
        __syncthreads();
        if (o < s_nh[tid]) s_nh[tid] = o;
        __syncthreads();
    }
    u32 nh = tid + 1 < TPB ? s_nh[tid + 1] : nt;
    for (u32 t = t1; t > t0; --t) {
        if (ws.scan_tiles[t - 1].first_head != kNoHead) nh = t - 1;
        ws.scan_tiles[t - 1].next_head_tile = nh;
    }
    for (u32 t = t0; t < t1; ++t) {
        ws.scan_tiles[t].desc_before = pd;
        pd += ws.scan_tiles[t].desc_first ? 1u : 0u;
    }
    __syncthreads();                               // the tile fields are visible to the whole CTA
    for (u32 i = tid; i < nt + 1; i += TPB) {
        u64 start;
        u32 desc;
        if (i == 0) {
            if (carry == kNoHead) continue;
            start = carry;
            desc = cdesc;
        } else {
            const ScanTile tl = ws.scan_tiles[i - 1];
            if (tl.last_head == kNoHead) continue;
            start = tl.last_head;
            desc = tl.desc_last;
        }
        // tiles i .. u* (u* the next tile with a head) add their descents before a first head
        const u32 us = i < nt ? ws.scan_tiles[i].next_head_tile : nt;
        const u32 before_i = i < nt ? ws.scan_tiles[i].desc_before : tot;
        u64 end;
        if (us < nt) {
            const ScanTile tu = ws.scan_tiles[us];
            if (tu.desc_before + (tu.desc_first ? 1u : 0u) > before_i) desc = 1;
            end = tu.first_head;
        } else {
            if (tot > before_i) desc = 1;
            if (e < n) {                       // carried into the next window
                s_head = start;
                s_desc = desc;
                s_set = 1;
                continue;
            }
            end = n;
        }
        if (desc) strict_emit<T>(ws, Task{start, end - start}, rec_cap);
    }
    __syncthreads();
    if (tid == 0) {
        ls->scan_pos = e;
        if (e >= n) {
            ls->carry_head = kNoHead;
            ls->carry_desc = 0;
        } else if (s_set) {
            ls->carry_head = s_head;
            ls->carry_desc = s_desc;
        } else {
            ls->status |= kStatusInternal;     // a window always ends inside some piece
        }
    }
}

}  // namespace ips4o
