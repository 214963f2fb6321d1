// ips4o_kernels.cuh — the kernels of one distribution step (Section 4) for a
// chunk of subproblems, plus the shared-memory base case (Section 4.7).
//
//   k_sample     Section 3 / 4 "Sampling": draw alpha*k-1 elements, sort them,
//                pick k-1 equally spaced splitters, remove duplicates and turn
//                on equality buckets when there were any (Sections 4.4, 4.7),
//                build the implicit search tree.
//   k_classify   Section 4.1 "Local Classification": every stripe is streamed
//                through shared memory, each element is classified with the
//                tree and appended to its bucket's buffer block; a full buffer
//                block is written back over the front of the stripe.  Counts
//                per bucket and the partially filled buffers are kept.
//   k_prefix     Section 4.2: prefix sums give the bucket boundaries, the
//                delimiters d_i (rounded up to blocks) and the initial write
//                and read pointers w_i, r_i; buckets crossing a stripe boundary
//                are queued for empty-block movement.
//   k_fix        Appendix A "Empty block movement": within each bucket region,
//                full blocks from the back fill the empty blocks at the front,
//                so every region reads "full blocks, then empty blocks".
//   k_permute    Section 4.2 "Block Permutation": persistent movers (one warp
//                each, the GPU counterpart of a thread with two swap buffers)
//                with primary buckets, atomic (w_i, r_i) updates in one 64-bit
//                word, reader counts, and the skip of blocks already in place.
//   k_cleanup    Section 4.3 "Cleanup": per bucket, the overshoot of its last
//                block, the partial buffers of all stripes and the overflow
//                block are written into the empty head and tail of the bucket;
//                a bucket at most the base-case size is then sorted right away
//                (Section 4.7), larger ones become next-level subproblems.
//   k_base       Section 4.7 base case for whole small inputs / segments.
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

// ------------------------------------------------------------ base case
// In-place sort of s[0..n) in shared memory: a bitonic network whose merge
// stages start by comparing element i with its mirror (i ^ (size-1)), so
// every comparator puts the smaller key at the lower index and the
// positions >= n behave as +infinity and are never touched.
template <class T, int TPB>
__device__ void smem_sort(typename T::elem_t* s, u32 n) {
    typedef typename T::elem_t E;
    if (n < 2) return;
    const u32 P = pow2_ceil_u32(n);
    for (u32 k = 2; k <= P; k <<= 1) {
        const u32 half = k >> 1;
        for (u32 t = threadIdx.x; t < P / 2; t += TPB) {
            u32 i = (t / half) * k + (t % half);
            u32 j = i ^ (k - 1);
            if (j < n) {
                E a = s[i], b = s[j];
                if (T::key(b) < T::key(a)) { s[i] = b; s[j] = a; }
            }
        }
        __syncthreads();
        for (u32 st = k >> 2; st > 0; st >>= 1) {
            for (u32 t = threadIdx.x; t < P / 2; t += TPB) {
                u32 i = (t / st) * 2 * st + (t % st);
                u32 j = i + st;
                if (j < n) {
                    E a = s[i], b = s[j];
                    if (T::key(b) < T::key(a)) { s[i] = b; s[j] = a; }
                }
            }
            __syncthreads();
        }
    }
}

template <class T, int TPB>
__device__ void sort_range_in_smem(typename T::elem_t* A, u64 n, typename T::elem_t* sbuf) {
    for (u32 i = threadIdx.x; i < n; i += TPB) sbuf[i] = A[i];
    __syncthreads();
    smem_sort<T, TPB>(sbuf, (u32)n);
    for (u32 i = threadIdx.x; i < n; i += TPB) A[i] = sbuf[i];
    __syncthreads();
}

// Whole segments of at most `cap` elements: one CTA per segment.
// seg_begin/seg_n describe segment i (absolute offsets).
template <class T, int TPB>
__global__ void __launch_bounds__(TPB) k_base(typename T::elem_t* arr, const Task* segs, u32 nseg, u32 cap,
                                              ChunkCounters* ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::elem_t* sbuf = (typename T::elem_t*)smem_raw;
    for (u32 i = blockIdx.x; i < nseg; i += gridDim.x) {
        Task t = segs[i];
        if (t.n > cap) {
            if (threadIdx.x == 0) set_status(ctr, kStatusInternal);
            continue;
        }
        sort_range_in_smem<T, TPB>(arr + t.begin, t.n, sbuf);
    }
}

// ------------------------------------------------------------- sampling
template <class T, int TPB>
__global__ void __launch_bounds__(TPB) k_sample(const typename T::elem_t* arr, Workspace<T> ws, u32 nsub, u64 seed) {
    typedef typename T::key_t K;
    __shared__ K keys[4096];
    __shared__ K cand[256];
    __shared__ u32 scan_tmp[32];
    const u32 j = blockIdx.x;
    if (j >= nsub) return;
    SubDesc d = ws.subs[j];
    const u32 kk = d.k_target;                 // power of two in [2, 256]
    const u32 alpha = d.alpha;
    const u32 ns = alpha * kk - 1;             // <= 4095 (host guarantees)
    const u32 P = pow2_ceil_u32(ns);
    const u64 st = mix64(seed ^ mix64(d.begin * 0x9E3779B97F4A7C15ull + d.level));
    for (u32 i = threadIdx.x; i < P; i += TPB) {
        if (i < ns) {
            u64 r = mix64(st + (u64)(i + 1) * 0x9E3779B97F4A7C15ull);
            u64 pos = __umul64hi(r, d.n);
            keys[i] = T::key(arr[d.begin + pos]);
        } else {
            keys[i] = key_max<K>();
        }
    }
    __syncthreads();
    // bitonic sort of the (power-of-two padded) sample
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
    // k-1 equally spaced splitters s_j = sample[j*alpha - 1]
    u32 ncand = kk - 1;
    if (threadIdx.x < ncand) cand[threadIdx.x] = keys[(threadIdx.x + 1) * alpha - 1];
    __syncthreads();
    int dup = (threadIdx.x > 0 && threadIdx.x < ncand && cand[threadIdx.x] == cand[threadIdx.x - 1]) ? 1 : 0;
    const bool eq = __syncthreads_or(dup) != 0;
    if (eq && kk >= 4) {
        // Equality buckets double the bucket count; keep it within 256 by
        // reselecting with k/2 splitters (spacing 2*alpha).
        ncand = kk / 2 - 1;
        if (threadIdx.x < ncand) cand[threadIdx.x] = keys[(threadIdx.x + 1) * 2 * alpha - 1];
        __syncthreads();
    }
    // remove duplicates (stable compaction)
    u32 keep = (threadIdx.x < ncand && (threadIdx.x == 0 || cand[threadIdx.x] != cand[threadIdx.x - 1])) ? 1u : 0u;
    K mine = threadIdx.x < ncand ? cand[threadIdx.x] : K(0);
    u32 m;
    u32 pos = block_exclusive_scan<u32>(keep, scan_tmp, &m);
    __syncthreads();
    if (keep) cand[pos] = mine;
    __syncthreads();
    if (m == 0) m = 1;   // cannot happen (ncand >= 1), kept for safety
    const u32 L = pow2_ceil_u32(m + 1);
    u32 logL = 31 - __clz(L);
    K* spl = ws.spl + (u64)j * kMaxLeaves;
    K* tree = ws.tree + (u64)j * kMaxLeaves;
    // padded sorted splitters s_1..s_{L-1} (s_i = s_m for i > m)
    for (u32 i = threadIdx.x; i < kMaxLeaves; i += TPB) {
        K v = cand[(i >= 1 ? (i <= m ? i : m) : 1) - 1];
        spl[i] = v;
    }
    // implicit tree: node v at depth dd holds s_{(2*(v - 2^dd) + 1) * L / 2^(dd+1)}
    for (u32 v = threadIdx.x; v < kMaxLeaves; v += TPB) {
        K val = cand[0];
        if (v >= 1 && v < L) {
            u32 dd = 31 - __clz(v);
            u32 idx = (2 * (v - (1u << dd)) + 1) * (L >> (dd + 1));
            val = cand[(idx <= m ? idx : m) - 1];
        }
        tree[v] = val;
    }
    if (threadIdx.x == 0) {
        ws.subs[j].log_leaves = logL;
        ws.subs[j].eq = eq ? 1u : 0u;
        ws.subs[j].nbuckets = eq ? 2 * L - 1 : L;
    }
}

// ------------------------------------------------- local classification
template <class T>
struct ClassifyCfg {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    static constexpr int TPB = 512;
    static constexpr int NW = TPB / 32;
    static constexpr int STAGES = 3;
    static constexpr int TILE = 16384 / (int)sizeof(E);        // 16 KiB per tile
    static constexpr int IPT = TILE / TPB;
    static constexpr int B = T::kBlock;
    static constexpr int MAXBLK = 320;                        // >= (256*(B-1) + TILE) / B
    static constexpr size_t off_buf = 0;
    static constexpr size_t off_stage = off_buf + (size_t)kMaxBuckets * B * sizeof(E);
    static constexpr size_t off_tree = off_stage + (size_t)STAGES * TILE * sizeof(E);
    static constexpr size_t off_spl = off_tree + kMaxLeaves * sizeof(K);
    static constexpr size_t off_fill = off_spl + kMaxLeaves * sizeof(K);
    static constexpr size_t off_cnt = off_fill + kMaxBuckets * 4;
    static constexpr size_t off_off = off_cnt + kMaxBuckets * 4;
    static constexpr size_t off_bscan = off_off + kMaxBuckets * 4;
    static constexpr size_t off_total = off_bscan + kMaxBuckets * 4;
    static constexpr size_t off_blkb = off_total + kMaxBuckets * 4;
    static constexpr size_t off_misc = off_blkb + MAXBLK * 2;
    static constexpr size_t smem_bytes = off_misc + 64 * 8;
    static_assert((size_t)(256 * (B - 1) + TILE) / B <= (size_t)MAXBLK, "MAXBLK too small");
    static_assert(TILE % TPB == 0, "tile must be a multiple of the CTA size");
};

template <class T>
__global__ void __launch_bounds__(ClassifyCfg<T>::TPB, 1)
    k_classify(typename T::elem_t* arr, Workspace<T> ws, u32 nstripes) {
    typedef ClassifyCfg<T> C;
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    constexpr int TPB = C::TPB, NW = C::NW, STAGES = C::STAGES, TILE = C::TILE, IPT = C::IPT, B = C::B;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = (E*)(smem_raw + C::off_buf);
    E* stage = (E*)(smem_raw + C::off_stage);
    K* s_tree = (K*)(smem_raw + C::off_tree);
    K* s_spl = (K*)(smem_raw + C::off_spl);
    u32* s_fill = (u32*)(smem_raw + C::off_fill);
    u32* s_cnt = (u32*)(smem_raw + C::off_cnt);
    u32* s_off = (u32*)(smem_raw + C::off_off);
    u32* s_bscan = (u32*)(smem_raw + C::off_bscan);
    u32* s_total = (u32*)(smem_raw + C::off_total);
    unsigned short* s_blkb = (unsigned short*)(smem_raw + C::off_blkb);
    u64* s_misc = (u64*)(smem_raw + C::off_misc);   // [0..32) scan tmp, [40] stripe id
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (tid == 0) s_misc[40] = atomicAdd(&ws.ctr->stripe_next, 1u);
        __syncthreads();
        const u32 s = (u32)s_misc[40];
        if (s >= nstripes) break;
        const StripeDesc sd = ws.stripes[s];
        const SubDesc sub = ws.subs[sd.sub];
        const int logL = (int)sub.log_leaves;
        const bool eq = sub.eq != 0;
        for (int i = tid; i < kMaxLeaves; i += TPB) {
            s_tree[i] = ws.tree[(u64)sd.sub * kMaxLeaves + i];
            s_spl[i] = ws.spl[(u64)sd.sub * kMaxLeaves + i];
        }
        for (int b = tid; b < kMaxBuckets; b += TPB) { s_fill[b] = 0; s_cnt[b] = 0; s_total[b] = 0; }
        E* A = arr + sd.begin;
        const u64 len = sd.end - sd.begin;
        const u32 ntiles = (u32)ceil_div(len, TILE);
        u32 front = 0;                       // full blocks written at the stripe front
        __syncthreads();

        auto issue = [&](u32 tn) {
            E* dst = stage + (tn % STAGES) * TILE;
            const u64 tb = (u64)tn * TILE;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                u32 idx = tid + q * TPB;
                if (tb + idx < len) cp_async<sizeof(E)>(dst + idx, A + tb + idx);
            }
        };
#pragma unroll
        for (int p = 0; p < STAGES - 1; ++p) {
            if ((u32)p < ntiles) issue(p);
            cp_async_commit();
        }
        for (u32 t = 0; t < ntiles; ++t) {
            if (t + STAGES - 1 < ntiles) issue(t + STAGES - 1);
            cp_async_commit();
            cp_async_wait<STAGES - 1>();
            __syncthreads();
            E* tile = stage + (t % STAGES) * TILE;
            const u64 tb = (u64)t * TILE;
            const u32 tcount = (u32)((len - tb) < (u64)TILE ? (len - tb) : (u64)TILE);
            E e[IPT];
            int bk[IPT];
            u32 rk[IPT];
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                u32 idx = tid + q * TPB;
                bk[q] = -1;
                if (idx < tcount) {
                    e[q] = tile[idx];
                    bk[q] = classify_key<K>(T::key(e[q]), s_tree, s_spl, logL, eq);
                }
                // rank within the tile's run of the bucket, aggregated per warp
                unsigned peers = __match_any_sync(0xffffffffu, bk[q]);
                int leader = __ffs(peers) - 1;
                u32 base = 0;
                if (lane == leader && bk[q] >= 0) base = atomicAdd(&s_cnt[bk[q]], (u32)__popc(peers));
                base = __shfl_sync(0xffffffffu, base, leader);
                rk[q] = base + __popc(peers & ((1u << lane) - 1u));
            }
            __syncthreads();
            // per-bucket run offsets in the tile and full blocks to emit
            u32 c = 0, f = 0, nfull = 0;
            if (tid < kMaxBuckets) {
                c = s_cnt[tid];
                f = s_fill[tid];
                nfull = (f + c) / B;
            }
            u64 tot;
            u64 pre = block_exclusive_scan<u64>(((u64)c << 32) | nfull, s_misc, &tot);
            const u32 tot_blocks = (u32)(tot & 0xffffffffu);
            if (tid < kMaxBuckets) {
                s_off[tid] = (u32)(pre >> 32);
                s_bscan[tid] = (u32)(pre & 0xffffffffu);
                for (u32 q = 0; q < nfull; ++q) s_blkb[(u32)(pre & 0xffffffffu) + q] = (unsigned short)tid;
            }
            __syncthreads();
            // group the tile by bucket (the staging slot is free now)
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if (bk[q] >= 0) tile[s_off[bk[q]] + rk[q]] = e[q];
            __syncthreads();
            // write full blocks over the front of the stripe
            for (u32 i = warp; i < tot_blocks; i += NW) {
                const u32 b = s_blkb[i];
                const u32 jb = i - s_bscan[b];
                const u32 fb = s_fill[b];
                const u32 ob = s_off[b];
                const u64 dst = (u64)(front + i) * B;
                if (dst + B <= len) {
#pragma unroll
                    for (int v = lane; v < B; v += 32) {
                        const u32 vv = jb * B + v;
                        A[dst + v] = vv < fb ? buf[b * B + vv] : tile[ob + vv - fb];
                    }
                } else if (lane == 0) {
                    set_status(ws.ctr, kStatusInternal);
                }
            }
            __syncthreads();
            // the remainder of each bucket goes (back) into its buffer block
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (bk[q] >= 0) {
                    const int b = bk[q];
                    const u32 fb = s_fill[b], cb = s_cnt[b];
                    const u32 nf = (fb + cb) / B;
                    const u32 p = fb + rk[q];
                    if (p >= nf * B) buf[b * B + (p - nf * B)] = e[q];
                }
            }
            __syncthreads();
            if (tid < kMaxBuckets) {
                s_total[tid] += c;
                s_fill[tid] = (f + c) % B;
                s_cnt[tid] = 0;
            }
            front += tot_blocks;
            __syncthreads();
        }
        cp_async_wait<0>();
        // counts, leftovers (partially filled buffers) to the stripe's pool area
        u32 f = tid < kMaxBuckets ? s_fill[tid] : 0;
        u32 ltot;
        u32 lpre = block_exclusive_scan<u32>(f, (u32*)s_misc, &ltot);
        if (tid < kMaxBuckets) {
            ws.counts[(u64)s * kMaxBuckets + tid] = s_total[tid];
            ws.lscan[(u64)s * kMaxBuckets + tid] = lpre;
            s_off[tid] = lpre;
        }
        __syncthreads();
        if (ltot <= sd.pool_cap) {
            for (int b = warp; b < kMaxBuckets; b += NW) {
                const u32 fb = s_fill[b], ob = s_off[b];
                for (u32 v = lane; v < fb; v += 32) ws.pool[sd.pool_off + ob + v] = buf[b * B + v];
            }
        } else if (tid == 0) {
            set_status(ws.ctr, kStatusInternal);
        }
        if (tid == 0) ws.stripe_full[s] = front;
        __syncthreads();
    }
}

// ----------------------------------------------- prefix sums, pointers
template <class T, int TPB>
__global__ void __launch_bounds__(TPB) k_prefix(Workspace<T> ws, u32 nsub) {
    constexpr int B = T::kBlock;
    static_assert(TPB == kMaxBuckets, "one thread per bucket");
    __shared__ u64 tmp64[32];
    __shared__ u32 s_sbk[kMaxStripesPerSub];
    __shared__ u32 s_full[kMaxStripesPerSub];
    __shared__ u32 s_delim[kMaxBuckets + 1];
    const u32 j = blockIdx.x;
    if (j >= nsub) return;
    const SubDesc sub = ws.subs[j];
    const u32 nb = sub.nbuckets;
    const u32 sb = sub.stripe_begin, ns = sub.num_stripes;
    const int b = threadIdx.x;
    u64 blocks = 0;
    for (u32 i = threadIdx.x; i < ns; i += TPB) {
        const StripeDesc sd = ws.stripes[sb + i];
        s_sbk[i] = (u32)((sd.begin - sub.begin) / B);
        s_full[i] = ws.stripe_full[sb + i];
    }
    __syncthreads();
    u64 c = 0;
    u32 fb = 0;
    if ((u32)b < nb) {
        for (u32 i = 0; i < ns; ++i) {
            u32 x = ws.counts[(u64)(sb + i) * kMaxBuckets + b];
            c += x;
            fb += x / B;
        }
    }
    u64 total;
    u64 start = block_exclusive_scan<u64>(c, tmp64, &total);
    if (total != sub.n && threadIdx.x == 0) set_status(ws.ctr, kStatusInternal);
    u64* bstart = ws.bstart + (u64)j * (kMaxBuckets + 1);
    u32* delim = ws.delim + (u64)j * (kMaxBuckets + 1);
    if ((u32)b < nb) {
        bstart[b] = start;
        s_delim[b] = (u32)ceil_div(start, B);
    }
    if (b == 0) {
        bstart[nb] = sub.n;
        s_delim[nb] = (u32)ceil_div(sub.n, B);
    }
    __syncthreads();
    if ((u32)b < nb) {
        const u32 d0 = s_delim[b], d1 = s_delim[b + 1];
        u32 nfr = 0;
        for (u32 i = 0; i < ns; ++i) {
            u32 lo = max(d0, s_sbk[i]), hi = min(d1, s_sbk[i] + s_full[i]);
            if (hi > lo) nfr += hi - lo;
        }
        u32 in_zone = 0;
        const u32 z1 = d0 + nfr;
        for (u32 i = 0; i < ns; ++i) {
            u32 lo = max(d0, s_sbk[i]), hi = min(z1, s_sbk[i] + s_full[i]);
            if (hi > lo) in_zone += hi - lo;
        }
        const u32 holes = nfr - in_zone;
        delim[b] = d0;
        const u64 r = (u64)d0 + nfr - 1 + kPtrBias;   // r_i = d_i + nfr - 1 (biased)
        ws.wr[(u64)j * kMaxBuckets + b] = ((u64)d0 << 32) | (r & 0xffffffffull);
        ws.readers[(u64)j * kMaxBuckets + b] = 0;
        ws.flags[(u64)j * kMaxBuckets + b] = 0;
        ws.region_full[(u64)j * kMaxBuckets + b] = nfr;
        ws.bucket_full[(u64)j * kMaxBuckets + b] = fb;
        if (holes > 0) {
            u32 idx = atomicAdd(&ws.ctr->fix_count, 1u);
            if (idx < ws.max_sub * kMaxBuckets) ws.fix_list[idx] = FixItem{j, (u32)b};
            else set_status(ws.ctr, kStatusCapacity);
        }
    }
    if (b == 0) delim[nb] = s_delim[nb];
    if (threadIdx.x == 0) {
        for (u32 i = 0; i < ns; ++i) blocks += s_full[i];
        ws.subs[j].blocks_total = blocks;
    }
}

// -------------------------------------------- empty-block movement (App. A)
template <class T, int TPB>
__global__ void __launch_bounds__(TPB) k_fix(typename T::elem_t* arr, Workspace<T> ws) {
    typedef typename T::elem_t E;
    constexpr int B = T::kBlock, NW = TPB / 32;
    __shared__ u32 h_pre[kMaxStripesPerSub + 1], s_pre[kMaxStripesPerSub + 1];
    __shared__ u32 h_at[kMaxStripesPerSub], s_at[kMaxStripesPerSub];
    __shared__ u32 tmp[32];
    const u32 nfix = ws.ctr->fix_count;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 moved = 0;
    for (u32 it = blockIdx.x; it < nfix; it += gridDim.x) {
        const FixItem fi = ws.fix_list[it];
        const SubDesc sub = ws.subs[fi.sub];
        const u32* delim = ws.delim + (u64)fi.sub * (kMaxBuckets + 1);
        const u32 d0 = delim[fi.bucket], d1 = delim[fi.bucket + 1];
        const u32 z1 = d0 + ws.region_full[(u64)fi.sub * kMaxBuckets + fi.bucket];
        const u32 ns = sub.num_stripes, sb = sub.stripe_begin;
        // per stripe: holes = empty slots in [d0, z1); sources = full slots in [z1, d1)
        constexpr int PER = (kMaxStripesPerSub + TPB - 1) / TPB;
        u32 hc[PER], sc[PER], hsum = 0, ssum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const u32 i = threadIdx.x * PER + q;
            hc[q] = sc[q] = 0;
            if (i < ns) {
                const StripeDesc sd = ws.stripes[sb + i];
                const u32 sbk = (u32)((sd.begin - sub.begin) / B);
                const u32 ebk = (u32)ceil_div(sd.end - sub.begin, B);
                const u32 fe = sbk + ws.stripe_full[sb + i];
                u32 lo = max(fe, d0), hi = min(ebk, z1);
                if (hi > lo) hc[q] = hi - lo;
                h_at[i] = lo;
                lo = max(sbk, z1);
                hi = min(fe, d1);
                if (hi > lo) sc[q] = hi - lo;
                s_at[i] = lo;
            }
            hsum += hc[q];
            ssum += sc[q];
        }
        u32 htot, stot;
        u32 hp = block_exclusive_scan<u32>(hsum, tmp, &htot);
        __syncthreads();
        u32 sp = block_exclusive_scan<u32>(ssum, tmp, &stot);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const u32 i = threadIdx.x * PER + q;
            if (i < ns) { h_pre[i] = hp; s_pre[i] = sp; }
            hp += hc[q];
            sp += sc[q];
        }
        if (threadIdx.x == 0) { h_pre[ns] = htot; s_pre[ns] = stot; }
        __syncthreads();
        if (htot != stot) {
            if (threadIdx.x == 0) set_status(ws.ctr, kStatusInternal);
        } else {
            E* A = arr + sub.begin;
            for (u32 q = warp; q < htot; q += NW) {
                // binary search: last stripe with prefix <= q
                u32 lo = 0, hi = ns;
                while (hi - lo > 1) { u32 mid = (lo + hi) >> 1; if (h_pre[mid] <= q) lo = mid; else hi = mid; }
                const u32 hole = h_at[lo] + (q - h_pre[lo]);
                lo = 0; hi = ns;
                while (hi - lo > 1) { u32 mid = (lo + hi) >> 1; if (s_pre[mid] <= q) lo = mid; else hi = mid; }
                const u32 src = s_at[lo] + (q - s_pre[lo]);
                if ((u64)(hole + 1) * B <= sub.n && (u64)(src + 1) * B <= sub.n) {
#pragma unroll
                    for (int v = lane; v < B; v += 32) A[(u64)hole * B + v] = A[(u64)src * B + v];
                } else if (lane == 0) {
                    set_status(ws.ctr, kStatusInternal);
                }
                if (lane == 0) ++moved;
            }
        }
        __syncthreads();
    }
    if (lane == 0 && moved) atomicAdd(&ws.ctr->fix_blocks, moved);
}

// --------------------------------------------------- block permutation
template <class T>
struct PermuteCfg {
    static constexpr int TPB = 256;
    static constexpr int NW = TPB / 32;
    static constexpr int EPL = T::kBlock / 32;   // elements per lane of one block
    static_assert(T::kBlock % 32 == 0, "block must be a multiple of the warp size");
};

template <class T>
__device__ __forceinline__ int classify_block_head(const typename T::elem_t* blk, const typename T::key_t* tree,
                                                   const typename T::key_t* spl, int logL, bool eq,
                                                   typename T::elem_t first) {
    return classify_key<typename T::key_t>(T::key(first), tree, spl, logL, eq);
}

template <class T>
__global__ void __launch_bounds__(PermuteCfg<T>::TPB)
    k_permute(typename T::elem_t* arr, Workspace<T> ws, u32 nsub, u32 spin_limit) {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    typedef PermuteCfg<T> C;
    constexpr int TPB = C::TPB, NW = C::NW, EPL = C::EPL, B = T::kBlock;
    __shared__ u32 s_mpre[1025];
    __shared__ u64 s_tot;
    __shared__ u32 tmp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 M = gridDim.x * NW;
    // movers per subproblem in proportion to its full blocks (at least one)
    u64 mine = 0;
    for (u32 i = threadIdx.x; i < nsub; i += TPB) mine += ws.subs[i].blocks_total;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    atomicAdd(&s_tot, mine);
    __syncthreads();
    const u64 total = s_tot;
    {
        // scan over nsub (<= 1024) entries, PER per thread
        constexpr int PER = 1024 / TPB;
        u32 mv[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const u32 i = threadIdx.x * PER + q;
            mv[q] = 0;
            if (i < nsub && total > 0) {
                const u64 bl = ws.subs[i].blocks_total;
                if (bl > 0) {
                    u64 x = bl * (u64)M / total;
                    mv[q] = (u32)(x < 1 ? 1 : (x > 0x10000000ull ? 0x10000000ull : x));
                }
            }
            sum += mv[q];
        }
        u32 tot;
        u32 p = block_exclusive_scan<u32>(sum, tmp, &tot);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const u32 i = threadIdx.x * PER + q;
            if (i < nsub) s_mpre[i] = p;
            p += mv[q];
        }
        if (threadIdx.x == 0) s_mpre[nsub] = tot;
        __syncthreads();
    }
    const u32 V = s_mpre[nsub];
    u64 moved = 0, skipped = 0;
    bool failed = false;
    for (u32 v = blockIdx.x * NW + warp; v < V && !failed; v += M) {
        u32 lo = 0, hi = nsub;
        while (hi - lo > 1) { u32 mid = (lo + hi) >> 1; if (s_mpre[mid] <= v) lo = mid; else hi = mid; }
        const u32 j = lo;
        const u32 local = v - s_mpre[j];
        const u32 nmov = s_mpre[j + 1] - s_mpre[j];
        const SubDesc sub = ws.subs[j];
        const u32 nb = sub.nbuckets;
        const int logL = (int)sub.log_leaves;
        const bool eq = sub.eq != 0;
        const K* tree = ws.tree + (u64)j * kMaxLeaves;
        const K* spl = ws.spl + (u64)j * kMaxLeaves;
        u64* wr = ws.wr + (u64)j * kMaxBuckets;
        u32* readers = ws.readers + (u64)j * kMaxBuckets;
        const u32* delim = ws.delim + (u64)j * (kMaxBuckets + 1);
        E* A = arr + sub.begin;
        E* ovf = ws.overflow + (u64)j * B;
        const u64 nbc = sub.n / B;                   // complete block slots
        const bool partial = (sub.n % B) != 0;
        const u32 p0 = (u32)(((u64)local * nb) / (nmov ? nmov : 1));
        E buf[EPL], tmpb[EPL];
        for (u32 step = 0; step < nb && !failed; ++step) {
            const u32 p = (p0 + step) % nb;
            for (;;) {
                // take an unprocessed block from the primary bucket: r_p--
                u64 old = 0;
                if (lane == 0) {
                    red_add_relaxed(&readers[p], 1u);
                    old = atom_add_acq_rel(&wr[p], ~0ull);
                }
                old = __shfl_sync(0xffffffffu, old, 0);
                const long long w = (long long)(old >> 32);
                const long long r = (long long)(u32)(old & 0xffffffffull) - (long long)kPtrBias;
                if (r < w) {
                    if (lane == 0) red_add_relaxed(&readers[p], ~0u);
                    break;                                   // bucket p has no unprocessed blocks left
                }
                if (r < 0 || (u64)(r + 1) * B > sub.n) {
                    if (lane == 0) { set_status(ws.ctr, kStatusInternal); red_add_relaxed(&readers[p], ~0u); }
                    failed = true;
                    break;
                }
#pragma unroll
                for (int q = 0; q < EPL; ++q) buf[q] = A[(u64)r * B + lane + 32 * q];
                __threadfence();
                __syncwarp();
                if (lane == 0) red_add_relaxed(&readers[p], ~0u);
                // move the block until it lands in an empty slot
                int t = classify_key<K>(__shfl_sync(0xffffffffu, T::key(buf[0]), 0), tree, spl, logL, eq);
                for (;;) {
                    if (lane == 0) old = atom_add_acq_rel(&wr[t], 1ull << 32);
                    old = __shfl_sync(0xffffffffu, old, 0);
                    const long long wt = (long long)(old >> 32);
                    const long long rt = (long long)(u32)(old & 0xffffffffull) - (long long)kPtrBias;
                    if ((u64)wt >= delim[t + 1]) {
                        if (lane == 0) set_status(ws.ctr, kStatusInternal);
                        failed = true;
                        break;
                    }
                    if (wt <= rt) {
                        // slot wt is unprocessed: swap unless its block already belongs to t
#pragma unroll
                        for (int q = 0; q < EPL; ++q) tmpb[q] = A[(u64)wt * B + lane + 32 * q];
                        const int t2 = classify_key<K>(__shfl_sync(0xffffffffu, T::key(tmpb[0]), 0), tree, spl, logL, eq);
                        if (t2 == t) {
                            ++skipped;
                            continue;
                        }
#pragma unroll
                        for (int q = 0; q < EPL; ++q) {
                            A[(u64)wt * B + lane + 32 * q] = buf[q];
                            buf[q] = tmpb[q];
                        }
                        ++moved;
                        t = t2;
                        continue;
                    }
                    // slot wt is empty: wait until nobody reads from bucket t
                    u32 ok = 1;
                    if (lane == 0) {
                        u32 it = 0;
                        while (ld_acquire(&readers[t]) != 0) {
                            if (++it > spin_limit) { ok = 0; break; }
                            __nanosleep(64);
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) {
                        if (lane == 0) set_status(ws.ctr, kStatusTimeout);
                        failed = true;
                        break;
                    }
                    if ((u64)wt < nbc) {
#pragma unroll
                        for (int q = 0; q < EPL; ++q) A[(u64)wt * B + lane + 32 * q] = buf[q];
                    } else if (partial && (u64)wt == nbc) {
#pragma unroll
                        for (int q = 0; q < EPL; ++q) ovf[lane + 32 * q] = buf[q];
                    } else {
                        if (lane == 0) set_status(ws.ctr, kStatusInternal);
                        failed = true;
                    }
                    ++moved;
                    break;
                }
                if (failed) break;
            }
        }
    }
    if (lane == 0) {
        if (moved) atomicAdd(&ws.ctr->blocks_moved, moved);
        if (skipped) atomicAdd(&ws.ctr->blocks_skipped, skipped);
    }
}

// --------------------------------------------------------------- cleanup
template <class T>
struct CleanupCfg {
    typedef typename T::elem_t E;
    static constexpr int TPB = 512;
    static constexpr int B = T::kBlock;
    static constexpr size_t off_sort = 0;
    static constexpr size_t off_ov = off_sort + (size_t)T::kBaseCap * sizeof(E);
    static constexpr size_t off_lpre = off_ov + (size_t)B * sizeof(E);
    static constexpr size_t off_src = off_lpre + (size_t)(kMaxStripesPerSub + 1) * 4 + 4;
    static constexpr size_t smem_bytes = off_src + (size_t)kMaxStripesPerSub * 8;
};

template <class T>
__global__ void __launch_bounds__(CleanupCfg<T>::TPB)
    k_cleanup(typename T::elem_t* arr, Workspace<T> ws, u32 nsub, u32 base_cap, u32 spin_limit, u32 partition_only) {
    typedef typename T::elem_t E;
    typedef CleanupCfg<T> C;
    constexpr int TPB = C::TPB, B = C::B;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* s_sort = (E*)(smem_raw + C::off_sort);
    E* s_ov = (E*)(smem_raw + C::off_ov);
    u32* s_lpre = (u32*)(smem_raw + C::off_lpre);
    u64* s_src = (u64*)(smem_raw + C::off_src);
    __shared__ u32 s_ticket, s_ok;
    __shared__ u32 tmp[32];
    if (threadIdx.x == 0) s_ticket = atomicAdd(&ws.ctr->ticket, 1u);
    __syncthreads();
    const u32 ticket = s_ticket;
    const u32 j = ticket / kMaxBuckets, b = ticket % kMaxBuckets;
    if (j >= nsub) return;
    const SubDesc sub = ws.subs[j];
    const u32 nb = sub.nbuckets;
    if (b >= nb) return;
    E* A = arr + sub.begin;
    const u64* bstart = ws.bstart + (u64)j * (kMaxBuckets + 1);
    const u64 Bb = bstart[b], Eb = bstart[b + 1];
    const u32 d0 = ws.delim[(u64)j * (kMaxBuckets + 1) + b];
    const u64 w = ws.wr[(u64)j * kMaxBuckets + b] >> 32;
    const u64 nbc = sub.n / B;
    const bool partial = (sub.n % B) != 0;
    const bool has_blocks = w > d0;
    // the bucket's last full block went to the overflow block
    const u32 ovf = (partial && has_blocks && w == nbc + 1) ? (u32)B : 0u;
    const u64 P_lo = (u64)d0 * B;
    const u64 P_hi = has_blocks ? (ovf ? nbc : w) * B : P_lo;    // end of its blocks in the array
    const u32 ov = (u32)((has_blocks && P_hi > Eb) ? P_hi - Eb : 0);  // overshoot into the next head
    bool bad = ov > (u32)B || Eb < Bb || Eb > sub.n;
    // read the overshoot before the next bucket may overwrite its head
    if (!bad)
        for (u32 v = threadIdx.x; v < ov; v += TPB) s_ov[v] = A[Eb + v];
    __threadfence();
    __syncthreads();
    u32* flags = ws.flags + (u64)j * kMaxBuckets;
    if (threadIdx.x == 0) {
        st_release(&flags[b], 1u);
        u32 ok = 1;
        if (b > 0) {
            u32 it = 0;
            while (ld_acquire(&flags[b - 1]) == 0) {
                if (++it > spin_limit) { ok = 0; break; }
                __nanosleep(32);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) {
        if (threadIdx.x == 0) set_status(ws.ctr, kStatusTimeout);
        return;
    }
    // empty slots: head [Bb, min(P_lo, Eb)) and tail [P_hi, Eb)
    const u64 head_hi = P_lo < Eb ? P_lo : Eb;
    const u64 nh = head_hi > Bb ? head_hi - Bb : 0;
    const u64 nt = (P_lo < Eb && P_hi < Eb) ? Eb - P_hi : 0;
    // sources: overshoot, overflow block, partial buffers of all stripes
    const u32 ns = sub.num_stripes, sb = sub.stripe_begin;
    constexpr int PER = (kMaxStripesPerSub + TPB - 1) / TPB;
    u32 lc[PER], lsum = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const u32 i = threadIdx.x * PER + q;
        lc[q] = 0;
        if (i < ns) {
            const u64 si = (u64)(sb + i) * kMaxBuckets + b;
            lc[q] = ws.counts[si] % B;
            s_src[i] = ws.stripes[sb + i].pool_off + ws.lscan[si];
        }
        lsum += lc[q];
    }
    u32 ltot;
    u32 lp = block_exclusive_scan<u32>(lsum, tmp, &ltot);
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const u32 i = threadIdx.x * PER + q;
        if (i < ns) s_lpre[i] = lp;
        lp += lc[q];
    }
    if (threadIdx.x == 0) s_lpre[ns] = ltot;
    __syncthreads();
    const u64 nsrc = (u64)ov + ovf + ltot;
    if (bad || nh + nt != nsrc) {
        if (threadIdx.x == 0) set_status(ws.ctr, kStatusInternal);
        return;
    }
    const E* ovb = ws.overflow + (u64)j * B;
    for (u64 q = threadIdx.x; q < nsrc; q += TPB) {
        E x;
        if (q < ov) {
            x = s_ov[q];
        } else if (q < (u64)ov + ovf) {
            x = ovb[q - ov];
        } else {
            const u32 rr = (u32)(q - ov - ovf);
            u32 lo = 0, hi = ns;
            while (hi - lo > 1) { u32 mid = (lo + hi) >> 1; if (s_lpre[mid] <= rr) lo = mid; else hi = mid; }
            x = ws.pool[s_src[lo] + (rr - s_lpre[lo])];
        }
        const u64 dst = q < nh ? Bb + q : P_hi + (q - nh);
        A[dst] = x;
    }
    __syncthreads();
    if (partition_only) return;
    const u64 size = Eb - Bb;
    const bool is_eq = sub.eq && (b & 1);
    if (is_eq || size < 2) return;
    if (size <= base_cap) {
        sort_range_in_smem<T, TPB>(A + Bb, size, s_sort);
        if (threadIdx.x == 0) atomicAdd(&ws.ctr->base_buckets, 1ull);
    } else if (threadIdx.x == 0) {
        u32 idx = atomicAdd(&ws.ctr->next_count, 1u);
        if (idx < ws.next_cap) ws.next_tasks[idx] = Task{sub.begin + Bb, size};
        else set_status(ws.ctr, kStatusCapacity);
    }
}

}  // namespace ips4o
