// ips4o_kernels.cuh — the kernels of one distribution step (Section 4) for a
// chunk of subproblems, plus the shared-memory base case (Section 4.7).
//
//   k_sample     Section 3 / 4 "Sampling": draw alpha*k-1 elements, sort them,
//                pick k-1 equally spaced splitters, remove duplicates and turn
//                on equality buckets when there were any (Sections 4.4, 4.7),
//                build the implicit search tree.
//   k_classify   Section 4.1 "Local Classification": every stripe is streamed
//                through registers in 64 KiB tiles, each element is classified
//                (through the splitter lookup table, or the tree descent) and
//                appended to its bucket's buffer block in shared memory; a full
//                buffer block is written back over the front of the stripe.
//                Counts per bucket and the partially filled buffers are kept.
//   k_prefix     Section 4.2: prefix sums give the bucket boundaries, the
//                delimiters d_i (rounded up to blocks) and the initial write
//                and read pointers w_i, r_i; buckets crossing a stripe boundary
//                are queued for empty-block movement.
//   k_fix        Appendix A "Empty block movement": within each bucket region,
//                full blocks from the back fill the empty blocks at the front,
//                so every region reads "full blocks, then empty blocks".
//   k_permute    Section 4.2 "Block Permutation": persistent movers (lanes of
//                a warp, each the GPU counterpart of a thread with two swap
//                buffers) with primary buckets, atomic (w_i, r_i) updates in one
//                64-bit word, reader counts, and the skip of blocks already in
//                place.
//   k_cleanup    Section 4.3 "Cleanup": per bucket, the overshoot of its last
//                block, the partial buffers of all stripes and the overflow
//                block are written into the empty head and tail of the bucket;
//                a bucket at most the base-case size is then sorted right away
//                (Section 4.7), larger ones become next-level subproblems.
//   k_base       Section 4.7 base case for whole small inputs / segments.
#pragma once

#include "ips4o_basecase.cuh"
#include "ips4o_common.cuh"

namespace ips4o {

// ------------------------------------------------------------- sampling
// Sample and splitters of subproblem j by the whole CTA (TPB threads, at
// least 256): keys[4096], cand[256] and scan_tmp[32] are shared memory.
template <class T, int TPB>
__device__ void sample_sub(const typename T::elem_t* arr, const Workspace<T>& ws, u32 j, u64 seed,
                           typename T::key_t* keys, typename T::key_t* cand, u32* scan_tmp) {
    typedef typename T::key_t K;
    SubDesc d = ws.subs[j];
    const u32 kk = d.k_target;                 // power of two in [2, 256]
    const u32 alpha = d.alpha;
    const u32 ns = alpha * kk - 1;             // < T::kSampleMax (the planners guarantee)
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
    if constexpr (T::kSampleMax % TPB == 0 && T::kSampleMax >= TPB) {
        if (P == (u32)T::kSampleMax) sort_sample_reg<K, TPB, T::kSampleMax>(keys);   // the usual full sample
        else sort_sample<K, TPB>(keys, P);
    } else {
        sort_sample<K, TPB>(keys, P);
    }
    u32 logL;
    bool eq;
    select_splitters<K>(keys, kk, alpha, cand, scan_tmp, ws.tree + (u64)j * kMaxLeaves, ws.spl + (u64)j * kMaxLeaves,
                        &logL, &eq);
    const u32 L = 1u << logL;
    if (threadIdx.x == 0) {
        ws.subs[j].log_leaves = logL;
        ws.subs[j].eq = eq ? 1u : 0u;
        ws.subs[j].nbuckets = eq ? 2 * L - 1 : L;
    }
    __syncthreads();
}

template <class T, int TPB>
__global__ void __launch_bounds__(TPB) k_sample(const typename T::elem_t* arr, Workspace<T> ws, u32 nsub, u64 seed) {
    typedef typename T::key_t K;
    __shared__ K keys[T::kSampleMax];
    __shared__ K cand[256];
    __shared__ u32 scan_tmp[32];
    if (ws.ls) nsub = ws.ls->nsub;                  // device-planned round
    for (u32 j = blockIdx.x; j < nsub; j += gridDim.x) sample_sub<T, TPB>(arr, ws, j, seed, keys, cand, scan_tmp);
}

// ------------------------------------------------- local classification
template <class T>
struct ClassifyCfg {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    static constexpr int TPB = 1024;
    static constexpr int NW = TPB / 32;
    static constexpr int STAGES = 2;
    static constexpr int TILE = 32768 / (int)sizeof(E);        // 32 KiB per tile
    static constexpr int IPT = TILE / TPB;
    static constexpr int B = T::kBlock;
    static constexpr int MAXBLK = 352;                        // >= (256*(B-1) + TILE) / B
    static constexpr size_t off_buf = 0;
    static constexpr size_t off_stage = a16(off_buf + (size_t)kMaxBuckets * B * sizeof(E));
    static constexpr size_t off_tree = a16(off_stage + (size_t)STAGES * TILE * sizeof(E));
    static constexpr size_t off_spl = a16(off_tree + kMaxLeaves * sizeof(K));
    static constexpr size_t off_fill = a16(off_spl + kMaxLeaves * sizeof(K));
    static constexpr size_t off_cnt = a16(off_fill + kMaxBuckets * 4);
    static constexpr size_t off_off = a16(off_cnt + kMaxBuckets * 4);
    static constexpr size_t off_bscan = a16(off_off + kMaxBuckets * 4);
    static constexpr size_t off_total = a16(off_bscan + kMaxBuckets * 4);
    static constexpr size_t off_blkb = a16(off_total + kMaxBuckets * 4);
    static constexpr size_t off_emit = a16(off_blkb + MAXBLK * 2);
    static constexpr size_t off_misc = a16(off_emit + kMaxBuckets * 2);
    static constexpr size_t smem_bytes = a16(off_misc + 64 * 8);
    static_assert((size_t)(256 * (B - 1) + TILE) / B <= (size_t)MAXBLK, "MAXBLK too small");
    static_assert(MAXBLK < 65536 && TILE < (1 << 30), "packed scan fields");
    static_assert(TILE % TPB == 0, "tile must be a multiple of the CTA size");
};

template <class T>
struct ClassifyRegCfg {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    static constexpr int TPB = 512;
    static constexpr int NW = TPB / 32;
    static constexpr int TILE = 65536 / (int)sizeof(E) / TPB * TPB;   // about 64 KiB per tile
    static constexpr int IPT = TILE / TPB;
    static constexpr int B = T::kBlock;
    // a block is 512 bytes, one 16-byte chunk per lane (100-byte records:
    // 500 bytes in 4-byte words); 8-byte elements
    // share a chunk, so a grouping run then starts at the parity that makes
    // its blocks 16-byte aligned (PAD: at most one element of padding per
    // bucket and at the end); larger elements are aligned by themselves
    static constexpr bool PAD = sizeof(E) < 16;
    // grouping area: the new elements of the buckets that emit blocks in a tile
    static constexpr int GRP = TILE + (PAD ? 2 * kMaxBuckets : 0);
    static constexpr int MAXBLK = 384;                         // >= (256*(B-1) + TILE) / B
    static constexpr size_t off_buf = 0;
    static constexpr size_t off_grp = a16(off_buf + (size_t)kMaxBuckets * B * sizeof(E));
    static constexpr size_t off_tree = a16(off_grp + (size_t)GRP * sizeof(E));
    static constexpr size_t off_spl = a16(off_tree + kMaxLeaves * sizeof(K));
    static constexpr size_t off_fill = a16(off_spl + (kMaxLeaves + 8) * sizeof(K));
    static constexpr size_t off_cnt = a16(off_fill + kMaxBuckets * 4);          // u32[2][kMaxBuckets]
    static constexpr size_t off_total = a16(off_cnt + 2 * kMaxBuckets * 4);
    static constexpr size_t off_dst = a16(off_total + kMaxBuckets * 4);
    static constexpr size_t off_binfo = a16(off_dst + kMaxBuckets * 4);         // uint2[2][kMaxBuckets]
    static constexpr size_t off_desc = a16(off_binfo + 2 * kMaxBuckets * 8);    // u32[2][MAXBLK]
    static constexpr size_t off_misc = a16(off_desc + 2 * MAXBLK * 4);         // u32[16]
    static constexpr size_t off_lut = a16(off_misc + 64);                       // u16[kLutCells + 8]
    static constexpr size_t smem_bytes = a16(off_lut + (kLutCells + 8) * 2);
    static_assert(off_grp % 16 == 0 && off_grp % sizeof(E) == 0 && off_buf == 0,
                  "destinations count elements from the base");
    static_assert((size_t)(256 * (B - 1) + TILE) / B <= (size_t)MAXBLK, "MAXBLK too small");
    static_assert(TILE % TPB == 0 && TPB >= kMaxBuckets, "tile must be a multiple of the CTA size");
    static_assert(kLutCells % TPB == 0 && (size_t)GRP * sizeof(E) >= kLutCells, "table build layout");
    static_assert(TILE <= 65536 && GRP + 64 < 65536, "ranks and grouping offsets are packed in 16 bits");
    static_assert((B * (int)sizeof(E) == 32 * 16 && (sizeof(E) == 8 || sizeof(E) % 16 == 0)) ||
                      (sizeof(E) % 4 == 0 && B * (int)sizeof(E) <= 512),
                  "a block is one 16-byte chunk per lane, or at most 512 bytes of 4-byte words");
    static_assert(IPT >= 1, "at least one element per thread and tile");
    static_assert(smem_bytes <= 232448, "shared memory of one CTA");
};

// Bucket ids of IPT keys, descending the tree level by level for all keys at
// once so that the IPT independent shared-memory lookups overlap.  LOGL is
// the tree depth (log2 of the number of leaves), fixed at compile time.
template <class K, int IPT, int LOGL>
__device__ __forceinline__ void classify_fixed(const K (&k)[IPT], const K* tree, const K* spl, bool eq,
                                               int (&bk)[IPT]) {
    int j[IPT];
#pragma unroll
    for (int q = 0; q < IPT; ++q) j[q] = 1;
#pragma unroll
    for (int l = 0; l < LOGL; ++l) {
#pragma unroll
        for (int q = 0; q < IPT; ++q) j[q] = 2 * j[q] + (tree[j[q]] <= k[q] ? 1 : 0);
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        int i = j[q] - (1 << LOGL);
        if (eq) i = 2 * i - ((i > 0 && spl[i] == k[q]) ? 1 : 0);
        bk[q] = i;
    }
}

// The same descent over a tree of 64-bit keys kept as two 32-bit halves:
// a_j <= e is decided on the high halves, and the low half of a_j is read
// only when the high halves are equal, so most steps move 4 bytes per lane
// through shared memory instead of 8.
template <int IPT, int LOGL>
__device__ __forceinline__ void classify_fixed_split(const u64 (&k)[IPT], const u32* thi, const u32* tlo,
                                                     const u64* spl, bool eq, int (&bk)[IPT]) {
    int j[IPT];
    u32 khi[IPT], klo[IPT];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        j[q] = 1;
        khi[q] = (u32)(k[q] >> 32);
        klo[q] = (u32)k[q];
    }
#pragma unroll
    for (int l = 0; l < LOGL; ++l) {
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const u32 ah = thi[j[q]];
            bool le = ah < khi[q];
            if (ah == khi[q]) le = tlo[j[q]] <= klo[q];
            j[q] = 2 * j[q] + (le ? 1 : 0);
        }
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        int i = j[q] - (1 << LOGL);
        if (eq) i = 2 * i - ((i > 0 && spl[i] == k[q]) ? 1 : 0);
        bk[q] = i;
    }
}

// The same for keys of several words (the tree kept as whole keys).
template <class K, int IPT>
__device__ __forceinline__ void classify_many_k(const K (&k)[IPT], const K* tree, const K* spl, int logL, bool eq,
                                                int (&bk)[IPT]) {
    switch (logL) {
    case 8: classify_fixed<K, IPT, 8>(k, tree, spl, eq, bk); break;
    case 7: classify_fixed<K, IPT, 7>(k, tree, spl, eq, bk); break;
    case 6: classify_fixed<K, IPT, 6>(k, tree, spl, eq, bk); break;
    case 5: classify_fixed<K, IPT, 5>(k, tree, spl, eq, bk); break;
    case 4: classify_fixed<K, IPT, 4>(k, tree, spl, eq, bk); break;
    case 3: classify_fixed<K, IPT, 3>(k, tree, spl, eq, bk); break;
    case 2: classify_fixed<K, IPT, 2>(k, tree, spl, eq, bk); break;
    default: classify_fixed<K, IPT, 1>(k, tree, spl, eq, bk); break;
    }
}

template <int IPT>
__device__ __forceinline__ void classify_many(const u64 (&k)[IPT], const u32* thi, const u32* tlo, const u64* spl,
                                              int logL, bool eq, int (&bk)[IPT]) {
    switch (logL) {
    case 8: classify_fixed_split<IPT, 8>(k, thi, tlo, spl, eq, bk); break;
    case 7: classify_fixed_split<IPT, 7>(k, thi, tlo, spl, eq, bk); break;
    case 6: classify_fixed_split<IPT, 6>(k, thi, tlo, spl, eq, bk); break;
    case 5: classify_fixed_split<IPT, 5>(k, thi, tlo, spl, eq, bk); break;
    case 4: classify_fixed_split<IPT, 4>(k, thi, tlo, spl, eq, bk); break;
    case 3: classify_fixed_split<IPT, 3>(k, thi, tlo, spl, eq, bk); break;
    case 2: classify_fixed_split<IPT, 2>(k, thi, tlo, spl, eq, bk); break;
    default: classify_fixed_split<IPT, 1>(k, thi, tlo, spl, eq, bk); break;
    }
}

// Loads subproblem j's search tree and splitters into shared memory for the
// classification: 64-bit keys as the tree's 32-bit halves (thi, tlo), other
// keys as whole keys in `tree`.
template <class T>
__device__ __forceinline__ void load_class_tree(const Workspace<T>& ws, u32 j, typename T::key_t* tree,
                                                typename T::key_t* spl, int tid, int nthreads) {
    typedef typename T::key_t K;
    for (int i = tid; i < kMaxLeaves; i += nthreads) {
        const K a = ws.tree[(u64)j * kMaxLeaves + i];
        if constexpr (std::is_same<K, u64>::value) {
            ((u32*)tree)[i] = (u32)(a >> 32);
            ((u32*)tree)[kMaxLeaves + i] = (u32)a;
        } else {
            tree[i] = a;
        }
        spl[i] = ws.spl[(u64)j * kMaxLeaves + i];
    }
}

// Buckets of IPT keys by the tree descent (after load_class_tree).
template <class K, int IPT>
__device__ __forceinline__ void classify_keys(const K (&k)[IPT], const K* tree, const K* spl, int logL, bool eq,
                                              int (&bk)[IPT]) {
    if constexpr (std::is_same<K, u64>::value) {
        const u32* thi = (const u32*)tree;
        classify_many<IPT>(k, thi, thi + kMaxLeaves, spl, logL, eq, bk);
    } else {
        classify_many_k<K, IPT>(k, tree, spl, logL, eq, bk);
    }
}


// Local classification of stripe s (Section 4.1) by the whole CTA
// (ClassifyCfg<T>::TPB threads, ClassifyCfg<T>::smem_bytes of shared memory).
template <class T>
__device__ void classify_stripe(typename T::elem_t* arr, const Workspace<T>& ws, u32 s, unsigned char* smem_raw) {
    typedef ClassifyCfg<T> C;
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    constexpr int TPB = C::TPB, NW = C::NW, STAGES = C::STAGES, TILE = C::TILE, IPT = C::IPT, B = C::B;
    E* buf = (E*)(smem_raw + C::off_buf);
    E* stage = (E*)(smem_raw + C::off_stage);
    K* s_tree = (K*)(smem_raw + C::off_tree);
    K* s_spl = (K*)(smem_raw + C::off_spl);
    u32* s_fill = (u32*)(smem_raw + C::off_fill);
    u32* s_cnt = (u32*)(smem_raw + C::off_cnt);
    u32* s_off = (u32*)(smem_raw + C::off_off);     // grouped-tile offset of a bucket that fills a block
    u32* s_bscan = (u32*)(smem_raw + C::off_bscan);
    u32* s_total = (u32*)(smem_raw + C::off_total);
    unsigned short* s_blkb = (unsigned short*)(smem_raw + C::off_blkb);
    unsigned short* s_emit = (unsigned short*)(smem_raw + C::off_emit);   // buckets emitting in this tile
    u64* s_misc = (u64*)(smem_raw + C::off_misc);   // [0..32) scan tmp
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const StripeDesc sd = ws.stripes[s];
        const SubDesc sub = ws.subs[sd.sub];
        const int logL = (int)sub.log_leaves;
        const bool eq = sub.eq != 0;
        load_class_tree<T>(ws, sd.sub, s_tree, s_spl, tid, TPB);
        for (int b = tid; b < kMaxBuckets; b += TPB) { s_fill[b] = 0; s_cnt[b] = 0; s_total[b] = 0; }
        E* A = arr + sd.begin;
        const u32 len = (u32)(sd.end - sd.begin);   // a stripe holds < 2^32 elements
        const u32 ntiles = (len + TILE - 1) / TILE;
        u32 front = 0;                       // full blocks written at the stripe front
        __syncthreads();

        auto issue = [&](u32 tn) {
            E* dst = stage + (tn % STAGES) * TILE;
            const u32 tb = tn * TILE;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const u32 idx = tid + q * TPB;
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
            const u32 tb = t * TILE;
            const u32 tcount = len - tb < (u32)TILE ? len - tb : (u32)TILE;
            E e[IPT];
            K k[IPT];
            int bk[IPT];
            u32 rk[IPT];
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const u32 idx = tid + q * TPB;
                e[q] = tile[idx < tcount ? idx : 0];
                k[q] = T::key(e[q]);
            }
            classify_keys<K, IPT>(k, s_tree, s_spl, logL, eq, bk);
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (tid + q * TPB >= tcount) bk[q] = -1;
                // rank within the tile's run of the bucket; a warp whose lanes
                // all hit one bucket (long runs, repeated keys) takes one atomic
                const int b0 = __shfl_sync(0xffffffffu, bk[q], 0);
                if (__all_sync(0xffffffffu, bk[q] == b0)) {
                    u32 base = 0;
                    if (lane == 0 && b0 >= 0) base = atomicAdd(&s_cnt[b0], 32u);
                    rk[q] = __shfl_sync(0xffffffffu, base, 0) + lane;
                } else {
                    rk[q] = bk[q] >= 0 ? atomicAdd(&s_cnt[bk[q]], 1u) : 0u;
                }
            }
            __syncthreads();
            // Buckets whose buffer block fills in this tile emit full blocks;
            // their new elements are grouped in the (now free) staging slot.
            // The new elements of every other bucket go straight into its
            // buffer block.
            u32 c = 0, f = 0, nfull = 0;
            if (tid < kMaxBuckets) {
                c = s_cnt[tid];
                f = s_fill[tid];
                nfull = (f + c) / B;
            }
            // one scan of three packed counts: [tile offset 32 | blocks 16 | emitting buckets 16]
            u64 tot;
            const u64 pre = block_exclusive_scan<u64>(((u64)(nfull ? c : 0u) << 32) | ((u64)nfull << 16) |
                                                          (nfull ? 1u : 0u),
                                                      s_misc, &tot);
            const u32 tot_blocks = (u32)((tot >> 16) & 0xffffu);
            const u32 n_emit = (u32)(tot & 0xffffu);
            if (tid < kMaxBuckets) {
                const u32 bpre = (u32)((pre >> 16) & 0xffffu);
                s_off[tid] = nfull ? (u32)(pre >> 32) : 0xffffffffu;
                s_bscan[tid] = bpre;
                for (u32 q = 0; q < nfull; ++q) s_blkb[bpre + q] = (unsigned short)tid;
                if (nfull) s_emit[(u32)(pre & 0xffffu)] = (unsigned short)tid;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (bk[q] >= 0) {
                    const u32 ob = s_off[bk[q]];
                    if (ob == 0xffffffffu) buf[bk[q] * B + s_fill[bk[q]] + rk[q]] = e[q];
                    else tile[ob + rk[q]] = e[q];
                }
            }
            __syncthreads();
            // write full blocks over the front of the stripe
            for (u32 i = warp; i < tot_blocks; i += NW) {
                const u32 b = s_blkb[i];
                const u32 jb = i - s_bscan[b];
                const u32 fb = s_fill[b];
                const u32 ob = s_off[b];
                const u32 dst = (front + i) * B;
                if (dst + B <= len) {
                    E* g = A + dst;
#pragma unroll
                    for (int v = lane; v < B; v += 32) {
                        const u32 vv = jb * B + v;
                        g[v] = vv < fb ? buf[b * B + vv] : tile[ob + vv - fb];
                    }
                } else if (lane == 0) {
                    set_status(ws.ctr, kStatusInternal);
                }
            }
            __syncthreads();
            // the remainder of a bucket that emitted blocks goes back into its
            // buffer block (one warp per such bucket)
            for (u32 i = warp; i < n_emit; i += NW) {
                const u32 b = s_emit[i];
                const u32 fb = s_fill[b], cb = s_cnt[b];
                const u32 nf = (fb + cb) / B, rem = (fb + cb) % B;
                const u32 from = s_off[b] + nf * B - fb;
                for (u32 v = lane; v < rem; v += 32) buf[b * B + v] = tile[from + v];
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

// Local classification of stripe s (Section 4.1) with tiles held in
// registers (ClassifyRegCfg<T>::TPB threads).  Each thread keeps IPT
// elements of the current tile and loads its elements of the next tile while
// the current one is processed, so shared memory holds no input staging.
// Keys are classified through the splitter lookup table (lut_refine) where
// its cells separate the splitters, else by the tree descent; the table is
// built once per stripe from the subproblem's tree and gives the buckets of
// the descent.
//
// A tile goes through three phases separated by barriers:
//   A  warp 0 turns the tile's bucket counts into destinations (the bucket's
//      buffer block, or for a bucket whose buffer fills, a run in the
//      grouping area that starts at the parity which makes its blocks 16-byte
//      aligned), block descriptors and new fill levels; meanwhile the other
//      warps write the full blocks of the previous tile over the front of the
//      stripe, one 16-byte chunk per lane, and copy each emitting bucket's
//      remainder back into its buffer block;
//   B  every thread scatters its elements to their destinations;
//   C  every thread classifies its elements of the next tile and takes their
//      ranks within their buckets (shared-memory counters, double-buffered
//      so that phase A of this tile may still read the other set).
template <class T>
__device__ void classify_stripe_reg(typename T::elem_t* arr, const typename T::elem_t* src, const Workspace<T>& ws,
                                    u32 s, unsigned char* smem_raw) {
    typedef ClassifyRegCfg<T> C;
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    constexpr int TPB = C::TPB, NW = C::NW, TILE = C::TILE, IPT = C::IPT, B = C::B;
    constexpr u32 GRP0 = (u32)(C::off_grp / sizeof(E));   // grouping area, in elements from the base
    E* buf = (E*)(smem_raw + C::off_buf);
    E* grp = (E*)(smem_raw + C::off_grp);
    K* s_tree = (K*)(smem_raw + C::off_tree);
    K* s_spl = (K*)(smem_raw + C::off_spl);
    u32* s_fill = (u32*)(smem_raw + C::off_fill);
    u32* s_cnt = (u32*)(smem_raw + C::off_cnt);
    u32* s_total = (u32*)(smem_raw + C::off_total);
    // where the tile's next element of a bucket goes, in elements from the
    // start of shared memory: its buffer block, or its grouping-area run
    u32* s_dst = (u32*)(smem_raw + C::off_dst);
    uint2* s_binfo = (uint2*)(smem_raw + C::off_binfo);
    u32* s_desc = (u32*)(smem_raw + C::off_desc);
    u32* s_misc = (u32*)(smem_raw + C::off_misc);   // [0..1] blocks of a tile, [2..3] stripe front before it
    unsigned short* s_lut = (unsigned short*)(smem_raw + C::off_lut);
    E* s_elem = (E*)smem_raw;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const StripeDesc sd = ws.stripes[s];
    const SubDesc sub = ws.subs[sd.sub];
    const int logL = (int)sub.log_leaves;
    const bool eq = sub.eq != 0;
    load_class_tree<T>(ws, sd.sub, s_tree, s_spl, tid, TPB);
    for (int b = tid; b < kMaxBuckets; b += TPB) {
        s_fill[b] = 0;
        s_cnt[b] = 0;
        s_cnt[kMaxBuckets + b] = 0;
        s_total[b] = 0;
    }
    E* A = arr + sd.begin;
    const E* S = src + sd.begin;                 // the stripe's input: A itself, or a copy elsewhere
    const u32 len = (u32)(sd.end - sd.begin);    // a stripe holds < 2^32 elements
    const u32 ntiles = (len + TILE - 1) / TILE;
    const bool g16 = ((uintptr_t)A & 15) == 0;   // block stores as 16-byte chunks
    __syncthreads();
    // The splitter lookup table (keys of one 64-bit word).  Its cells are
    // linear (aligned to multiples of 2^shift of the key domain) or
    // logarithmic, whichever puts fewer pairs of adjacent distinct splitters
    // into one cell (each such pair is a bucket whose keys all need the binary
    // search); with more than L/16 such pairs either way, or a tree of fewer
    // than kLutMinLevels levels (a few comparisons), the stripe keeps the tree
    // descent.  lut_mode: 0 descent, 1 linear, 2 logarithmic, 3 linear with
    // the cell taken from the key's high 32 bits (shift >= 32).
    const int L = 1 << logL;
    u64 lbase = 0, lc0 = 0;
    u32 lsh = 0;
    int lut_mode = 0;
    if constexpr (std::is_same<K, u64>::value) {
        const u32* s_thi = (const u32*)s_tree;
        const u32* s_tlo = s_thi + kMaxLeaves;
        lbase = s_spl[1];
        const u64 ltop = s_spl[L - 1];
        lsh = lut_abs_shift(lbase, ltop);
        lc0 = lbase >> lsh;
        {
            int crowd_lin = 0, crowd_log = 0;
            if (tid >= 1 && tid + 1 < L) {
                const u64 a = s_spl[tid], b = s_spl[tid + 1];
                if (a != b) {
                    crowd_lin = lut_cell_abs(a, lc0, lsh) == lut_cell_abs(b, lc0, lsh) ? 1 : 0;
                    crowd_log = lut_cell_log(a, lbase) == lut_cell_log(b, lbase) ? 1 : 0;
                }
            }
            const int n_lin = __syncthreads_count(crowd_lin);
            const int n_log = __syncthreads_count(crowd_log);
            if (logL >= kLutMinLevels && (n_lin * 16 <= L || n_log * 16 <= L)) lut_mode = n_lin <= n_log ? 1 : 2;
            if (lut_mode == 1 && lsh >= 32) lut_mode = 3;
        }
        if (lut_mode != 0) {
            // i(first key of every cell) by the tree descent into the (still
            // free) grouping area, then the (lo, hi) entries
            constexpr int CPT = kLutCells / TPB;
            unsigned char* s_lo = (unsigned char*)grp;
            u64 ck[CPT];
            int ci[CPT];
            bool ok[CPT];
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const u32 c = (u32)(tid + q * TPB);
                ok[q] = lut_mode == 2 ? lut_cell_start_log(c, lbase, &ck[q]) : lut_cell_start_abs(c, lc0, lsh, &ck[q]);
                if (!ok[q]) ck[q] = ltop;
            }
            classify_many<CPT>(ck, s_thi, s_tlo, s_spl, logL, false, ci);
#pragma unroll
            for (int q = 0; q < CPT; ++q) s_lo[tid + q * TPB] = (unsigned char)(ok[q] ? ci[q] : L - 1);
            __syncthreads();
            for (int c = tid; c <= kLutCells; c += TPB) {
                u32 ent = 0;                      // cell kLutCells (logarithmic map): keys below s_1
                if (c < kLutCells) ent = (u32)s_lo[c] | ((c + 1 < kLutCells ? (u32)s_lo[c + 1] : (u32)(L - 1)) << 8);
                s_lut[c] = (unsigned short)ent;
            }
            __syncthreads();
        }
    }

    E e[IPT], nx[IPT];
    u32 rk[IPT];
    auto load_tile = [&](u32 tn) {
        const u32 tb = tn * TILE;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const u32 idx = tid + q * TPB;
            if (tb + idx < len) nx[q] = S[tb + idx];
        }
    };
    // buckets of the tile's elements and their ranks (bucket << 16 | rank)
    auto classify_rank = [&](u32 tn, u32* cnt) {
        const u32 tcount = len - tn * TILE < (u32)TILE ? len - tn * TILE : (u32)TILE;
        int (&bk)[IPT] = *reinterpret_cast<int(*)[IPT]>(&rk);   // the buckets, then bucket << 16 | rank
        if constexpr (std::is_same<K, u64>::value) {
            if (lut_mode == 3) {
                const u32 c0 = (u32)lc0, shh = lsh - 32;
#pragma unroll
                for (int q = 0; q < IPT; ++q) {
                    const K kq = T::key(e[q]);
                    const int i = lut_refine(kq, s_lut[lut_cell_abs_hi((u32)(kq >> 32), c0, shh)], s_spl);
                    bk[q] = eq ? 2 * i - ((i > 0 && s_spl[i] == kq) ? 1 : 0) : i;
                }
            } else if (lut_mode == 1) {
#pragma unroll
                for (int q = 0; q < IPT; ++q) {
                    const K kq = T::key(e[q]);
                    const int i = lut_refine(kq, s_lut[lut_cell_abs(kq, lc0, lsh)], s_spl);
                    bk[q] = eq ? 2 * i - ((i > 0 && s_spl[i] == kq) ? 1 : 0) : i;
                }
            } else if (lut_mode == 2) {
#pragma unroll
                for (int q = 0; q < IPT; ++q) {
                    const K kq = T::key(e[q]);
                    const int i = lut_refine(kq, s_lut[lut_cell_log(kq, lbase)], s_spl);
                    bk[q] = eq ? 2 * i - ((i > 0 && s_spl[i] == kq) ? 1 : 0) : i;
                }
            } else if constexpr (std::is_same<E, K>::value) {
                // the keys replace the elements for the descent (one fewer
                // register array), which the inverse map then restores
#pragma unroll
                for (int q = 0; q < IPT; ++q) e[q] = T::key(e[q]);
                classify_keys<K, IPT>(e, s_tree, s_spl, logL, eq, bk);
#pragma unroll
                for (int q = 0; q < IPT; ++q) e[q] = T::unkey(e[q]);
            } else {
                K k[IPT];
#pragma unroll
                for (int q = 0; q < IPT; ++q) k[q] = T::key(e[q]);
                classify_keys<K, IPT>(k, s_tree, s_spl, logL, eq, bk);
            }
        } else {
            K k[IPT];
#pragma unroll
            for (int q = 0; q < IPT; ++q) k[q] = T::key(e[q]);
            classify_keys<K, IPT>(k, s_tree, s_spl, logL, eq, bk);
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (tid + q * TPB >= tcount) bk[q] = -1;
            // rank within the tile's run of the bucket; a warp whose lanes
            // all hit one bucket (long runs, repeated keys) takes one atomic
            const int b0 = __shfl_sync(0xffffffffu, bk[q], 0);
            u32 r;
            if (__all_sync(0xffffffffu, bk[q] == b0)) {
                u32 base = 0;
                if (lane == 0 && b0 >= 0) base = atomicAdd(&cnt[b0], 32u);
                r = __shfl_sync(0xffffffffu, base, 0) + lane;
            } else {
                r = bk[q] >= 0 ? atomicAdd(&cnt[bk[q]], 1u) : 0u;
            }
            rk[q] = bk[q] >= 0 ? ((u32)bk[q] << 16) | r : 0xffffffffu;
        }
    };
    // Phase A, warp 0: destinations, block descriptors and fill levels of
    // the tile whose counts are cnt (set par); lane l handles 8 buckets.
    u32 front = 0;                               // full blocks written at the stripe front (warp 0's count)
    auto scan_tile = [&](u32 par) {
        constexpr int BPL = kMaxBuckets / 32;
        u32* cnt = s_cnt + par * kMaxBuckets;
        uint2* binfo = s_binfo + par * kMaxBuckets;
        u32* desc = s_desc + par * C::MAXBLK;
        const int b0 = lane * BPL;
        // run sizes in the grouping area (even, room for the parity pad) and blocks
        u32 mine = 0;
#pragma unroll
        for (int j = 0; j < BPL; j += 4) {
            const uint4 cv = *(const uint4*)(cnt + b0 + j), fv = *(const uint4*)(s_fill + b0 + j);
            const u32 cc[4] = {cv.x, cv.y, cv.z, cv.w}, ff[4] = {fv.x, fv.y, fv.z, fv.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const u32 nf = (ff[h] + cc[h]) / B;
                const u32 run = C::PAD ? ((cc[h] + (ff[h] & 1u) + 1u) & ~1u) : cc[h];
                mine += (nf ? run : 0u) | (nf << 16);
            }
        }
        u32 x = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const u32 tot = __shfl_sync(0xffffffffu, x, 31);
        u32 off = (x - mine) & 0xffffu, blk = (x - mine) >> 16;
        for (int j = 0; j < BPL; ++j) {
            const u32 b = (u32)(b0 + j), cj = cnt[b], fj = s_fill[b], t = fj + cj, nf = t / B, rem = t - nf * B;
            if (nf) {
                // with PAD, p - f is even: the run's blocks are 16-byte aligned
                const u32 p = off + (C::PAD ? (fj & 1u) : 0u);
                s_dst[b] = GRP0 + p;
                binfo[b] = make_uint2((p - fj + 64u) | (fj << 16) | (rem << 24), nf);
                for (u32 q = 0; q < nf; ++q) desc[blk + q] = b | (q << 8);
                blk += nf;
                off += C::PAD ? ((cj + (fj & 1u) + 1u) & ~1u) : cj;
            } else {
                s_dst[b] = b * B + fj;
            }
            s_fill[b] = rem;
            s_total[b] += cj;
            cnt[b] = 0;
        }
        if (lane == 0) {
            s_misc[par] = tot >> 16;
            s_misc[2 + par] = front;
        }
        front += tot >> 16;
    };
    // Full blocks of the tile of set par, block i by warp w0 + i (step nw):
    // a block is 512 bytes, one 16-byte chunk per lane.  The first block of a
    // bucket starts with the f elements its buffer block held; the warp that
    // writes it then copies the bucket's remainder back into the buffer.
    auto write_blocks = [&](u32 par, u32 w0, u32 nw) {
        const uint2* binfo = s_binfo + par * kMaxBuckets;
        const u32* desc = s_desc + par * C::MAXBLK;
        const u32 nblk = s_misc[par], fr = s_misc[2 + par];
        for (u32 i = w0; i < nblk; i += nw) {
            const u32 d = desc[i], b = d & 0xffu, q = d >> 8;
            const uint2 bi = binfo[b];
            const int vs = (int)(bi.x & 0xffffu) - 64;           // grouping index of block 0's element 0
            const u32 f = q == 0 ? (bi.x >> 16) & 0xffu : 0u;
            const u32 slot = fr + i;
            if ((u64)(slot + 1) * B > len) {
                if (lane == 0) set_status(ws.ctr, kStatusInternal);
                continue;
            }
            if constexpr (sizeof(E) == 8) {
                // lane's chunk: elements v0, v0 + 1
                const u32 v0 = (u32)lane * 2;
                const E* from = v0 < f ? buf + b * B + v0 : grp + (vs + (int)(q * B) + (int)v0);
                E* to = A + (size_t)slot * B + v0;
                u64 x0, x1;
                if (v0 + 1 == f) {                                 // the chunk straddles buffer and run
                    x0 = buf[b * B + v0];
                    x1 = grp[vs + (int)v0 + 1];
                } else {
                    const ulonglong2 v = *(const ulonglong2*)from;
                    x0 = v.x;
                    x1 = v.y;
                }
                if (g16) {
                    *(ulonglong2*)to = make_ulonglong2(x0, x1);
                } else {
                    to[0] = x0;
                    to[1] = x1;
                }
                const u32 rem = bi.x >> 24;
                if (q == 0 && rem > 0) {
                    __syncwarp();                                  // block 0 has read the buffer
                    const E* rs = grp + (vs + (int)(bi.y * B) + (int)v0);
                    if (v0 < rem) *(uint4*)(buf + b * B + v0) = *(const uint4*)rs;
                }
            } else if constexpr (sizeof(E) % 16 != 0) {
                // 4-byte words (100-byte records): word wi of the block lies
                // in element wi / WPE
                constexpr u32 WPE = (u32)sizeof(E) / 4, WPB = (u32)B * WPE;
                u32* to = (u32*)(A + (size_t)slot * B);
                for (u32 wi = (u32)lane; wi < WPB; wi += 32) {
                    const u32 v = wi / WPE;
                    const E* from = v < f ? buf + b * B + v : grp + (vs + (int)(q * B) + (int)v);
                    to[wi] = ((const u32*)from)[wi - v * WPE];
                }
                const u32 rem = bi.x >> 24;
                if (q == 0 && rem > 0) {
                    __syncwarp();                                  // block 0 has read the buffer
                    const E* rs = grp + (vs + (int)(bi.y * B));
                    for (u32 wi = (u32)lane; wi < rem * WPE; wi += 32)
                        ((u32*)(buf + b * B))[wi] = ((const u32*)rs)[wi];
                }
            } else {
                // lane's chunk: bytes [16 lane, 16 lane + 16) of the block,
                // inside element v0 (elements of 16 bytes or more)
                const u32 cb = (u32)lane * 16, v0 = cb / (u32)sizeof(E), co = cb % (u32)sizeof(E);
                const E* from = v0 < f ? buf + b * B + v0 : grp + (vs + (int)(q * B) + (int)v0);
                *(uint4*)((char*)(A + (size_t)slot * B) + cb) = *(const uint4*)((const char*)from + co);
                const u32 rem = bi.x >> 24;
                if (q == 0 && rem > 0) {
                    __syncwarp();                                  // block 0 has read the buffer
                    if (v0 < rem) {
                        const E* rs = grp + (vs + (int)(bi.y * B) + (int)v0);
                        *(uint4*)((char*)(buf + b * B + v0) + co) = *(const uint4*)((const char*)rs + co);
                    }
                }
            }
        }
    };

    if (ntiles > 0) load_tile(0);
    for (u32 t = 0; t < ntiles; ++t) {
        const u32 par = t & 1u;
        // C: this tile's buckets and ranks (its loads were issued a tile ago)
#pragma unroll
        for (int q = 0; q < IPT; ++q) e[q] = nx[q];
        if (t + 1 < ntiles) load_tile(t + 1);
        classify_rank(t, s_cnt + par * kMaxBuckets);
        __syncthreads();
        // A: scan of this tile by warp 0; blocks of the previous tile by the others
        if (warp == 0) scan_tile(par);
        else if (t > 0) write_blocks(par ^ 1u, (u32)warp - 1u, NW - 1u);
        __syncthreads();
        // B: scatter into buffer blocks and grouping runs
#pragma unroll
        for (int q = 0; q < IPT; ++q)
            if (rk[q] != 0xffffffffu) s_elem[s_dst[rk[q] >> 16] + (rk[q] & 0xffffu)] = e[q];
        __syncthreads();
    }
    if (ntiles > 0) {
        write_blocks((ntiles - 1) & 1u, (u32)warp, NW);
        __syncthreads();
    }
    // counts, leftovers (partially filled buffers) to the stripe's pool area
    u32 f = tid < kMaxBuckets ? s_fill[tid] : 0;
    u32 ltot;
    u32* s_off = s_dst;                          // free now: leftover offsets
    u32 lpre = block_exclusive_scan<u32>(f, s_desc, &ltot);
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
    if (tid == 0) {
        u32 fr = 0;
        if (ntiles > 0) fr = s_misc[2 + ((ntiles - 1) & 1u)] + s_misc[(ntiles - 1) & 1u];
        ws.stripe_full[s] = fr;
    }
    __syncthreads();
}

// src: where the elements of the stripes are read (arr itself for the usual
// in-place step; the first step of a sort from host memory reads the host
// buffer through its device address and writes the blocks into arr).
template <class T>
__global__ void __launch_bounds__(ClassifyRegCfg<T>::TPB, 1)
    k_classify(typename T::elem_t* arr, const typename T::elem_t* src, Workspace<T> ws, u32 nstripes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ u32 s_stripe;
    if (ws.ls) nstripes = ws.ls->nstr;              // device-planned round
    for (;;) {
        if (threadIdx.x == 0) s_stripe = atomicAdd(&ws.ctr->stripe_next, 1u);
        __syncthreads();
        const u32 s = s_stripe;
        __syncthreads();
        if (s >= nstripes) break;
        classify_stripe_reg<T>(arr, src, ws, ws.stripe_order ? ws.stripe_order[s] : s, smem_raw);
    }
}

// ----------------------------------------------- prefix sums, pointers
// Bucket starts, delimiters, (w, r) words, empty-block fix list and the
// exhausted bitmap of subproblem j, by a CTA of TPB >= 256 threads (thread b
// handles bucket b).  Shared memory: tmp64[32], s_sbk and s_full
// [kMaxStripesPerSub], s_delim[kMaxBuckets + 1].
template <class T, int TPB>
__device__ void prefix_sub(const Workspace<T>& ws, u32 j, u64* tmp64, u32* s_sbk, u32* s_full, u32* s_delim) {
    constexpr int B = T::kBlock;
    static_assert(TPB >= kMaxBuckets && TPB % 32 == 0, "one thread per bucket");
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
    // a subproblem whose elements all fall into one bucket (e.g. all keys
    // equal): every full block already lies in that bucket's region, so the
    // block permutation has nothing to move
    const bool single = __syncthreads_or((u32)b < nb && c == sub.n) != 0;
    bool no_blocks = true;
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
        // w_i = d_i, r_i = d_i + nfr - 1 (the last full block of the region), no
        // readers; with a single non-empty bucket, w_i = d_i + nfr: its blocks
        // count as already written in place
        if ((u64)(d1 - d0) > kMaxRegionBlocks) set_status(ws.ctr, kStatusCapacity);
        const u64 w0 = single ? (u64)nfr << kWShift : 0ull;
        ws.wr[(u64)j * kMaxBuckets + b] = w0 | ((u64)((long long)nfr - 1 + (long long)kRBias) << kRdBits);
        no_blocks = single || nfr == 0;
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
    // buckets without unprocessed blocks (beyond nb, no full block in the
    // region, or all in place) start out exhausted: no mover probes them
    const u32 word = __ballot_sync(0xffffffffu, no_blocks);
    if ((b & 31) == 0 && b < kMaxBuckets) ws.exhausted[(u64)j * 8 + (b >> 5)] = word;
    if (threadIdx.x == 0) {
        ws.movers[j] = 0;
        for (u32 i = 0; i < ns; ++i) blocks += s_full[i];
        ws.subs[j].blocks_total = blocks;
    }
    __syncthreads();
}

template <class T, int TPB>
__global__ void __launch_bounds__(TPB) k_prefix(Workspace<T> ws, u32 nsub) {
    __shared__ u64 tmp64[32];
    __shared__ u32 s_sbk[kMaxStripesPerSub];
    __shared__ u32 s_full[kMaxStripesPerSub];
    __shared__ u32 s_delim[kMaxBuckets + 1];
    if (ws.ls) nsub = ws.ls->nsub;                  // device-planned round
    for (u32 j = blockIdx.x; j < nsub; j += gridDim.x) {
        prefix_sub<T, TPB>(ws, j, tmp64, s_sbk, s_full, s_delim);
        __syncthreads();
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
//
// A mover is the GPU counterpart of one thread of Section 4.2: it owns a
// primary bucket, takes unprocessed blocks from it by decrementing r_p, and
// carries each block to its destination bucket t by incrementing w_t: a swap
// with the unprocessed block found there (or a skip when that block already
// belongs to t, which leaves it in place), or a write into an empty slot,
// after which it reads again.  When its primary bucket has no unprocessed
// block left it moves to the next one; it stops when no bucket has any.
//
// w_i, r_i and the number of movers currently reading from bucket i share
// one 64-bit word, so a claim is a single atomic add and every mover sees
// the three consistently.  A block claimed for reading stays protected until
// its reader drops the count with a release; a write into an empty slot
// waits (boundedly) until the count it observed has drained.  Buckets found
// empty are recorded in a bitmap so that movers stop probing them.
//
// Lane v < V of a warp is mover v: its pointer claims, decisions, the
// classification of block heads and the search for a new primary bucket run
// in parallel across the lanes.  Blocks are moved by the whole warp, one
// coalesced 512-byte copy per block (cp.async into the mover's two
// shared-memory block buffers; stores from shared memory), so one warp keeps
// up to V blocks in flight.
template <class T>
struct PermuteCfg {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    static constexpr int TPB = 128;
    static constexpr int NW = TPB / 32;
    static constexpr int V = 16;                 // movers per warp (lanes 0..V-1)
    static constexpr int MIN_CTAS = 3;           // shared memory admits 3 per SM (192 movers)
    // one block (512 bytes; 500 for 100-byte records) is copied by the warp
    // in chunks of CHB bytes, at most NCH per lane
    static constexpr int BB = T::kBlock * (int)sizeof(E);
    static constexpr int CHB = sizeof(E) % 16 == 0 ? 16 : (sizeof(E) % 8 == 0 ? 8 : 4);
    static constexpr int NCHT = BB / CHB;
    static constexpr int NCH = (NCHT + 31) / 32;
    static constexpr int MAX_MOVERS_PER_BUCKET = 128;
    static constexpr int MAX_JOINS = 32;         // subproblems a CTA joins after its own groups
    // block buffers of the warps, then one copy of the subproblem's tables
    // shared by the CTA (all its warps move blocks of the same subproblem)
    static constexpr size_t off_buf = 0;                                          // E[NW][2][V][B]
    static constexpr size_t off_tree = a16(off_buf + (size_t)NW * 2 * V * T::kBlock * sizeof(E));
    static constexpr size_t off_spl = a16(off_tree + (size_t)kMaxLeaves * sizeof(K));
    static constexpr size_t off_delim = a16(off_spl + (size_t)kMaxLeaves * sizeof(K));
    static constexpr size_t off_gpre = a16(off_delim + (size_t)(kMaxBuckets + 4) * 4);   // u16[1025]
    static constexpr size_t off_misc = a16(off_gpre + 1032 * 2);
    static constexpr size_t smem_bytes = a16(off_misc + 40 * 8);
    static_assert(BB <= 512 && BB % CHB == 0, "a block is at most 512 bytes of whole chunks");
};

// Copy subproblem j's search tree, splitters and delimiters into shared
// memory (all threads of the CTA take part).
template <class T>
__device__ __forceinline__ void load_sub_tables(const Workspace<T>& ws, u32 j, typename T::key_t* tree,
                                                typename T::key_t* spl, u32* delim) {
    for (int i = threadIdx.x; i < kMaxLeaves; i += blockDim.x) {
        tree[i] = ws.tree[(u64)j * kMaxLeaves + i];
        spl[i] = ws.spl[(u64)j * kMaxLeaves + i];
    }
    for (int i = threadIdx.x; i <= kMaxBuckets; i += blockDim.x) delim[i] = ws.delim[(u64)j * (kMaxBuckets + 1) + i];
}

// One mover group (a warp of V movers) of subproblem j: group gl of the
// subproblem's groups, nmov movers in all (Section 4.2).  wbuf is the warp's
// [2][V][b] block buffer; tree, spl, delim the subproblem's search tree,
// splitters and delimiters in shared memory (load_sub_tables).  A group that
// joins a subproblem already being permuted (join) starts each mover on the
// first bucket at or after its share that the exhausted bitmap does not
// mark, so no mover starts with a claim on a bucket known to be used up.
template <class T>
__device__ __forceinline__ void permute_group(typename T::elem_t* arr, const Workspace<T>& ws, u32 j, u32 gl,
                                              u32 nmov, typename T::elem_t* wbuf, const typename T::key_t* tree,
                                              const typename T::key_t* spl, const u32* delim, u32 spin_limit,
                                              u64& moved, u64& skipped, bool& failed, bool join = false) {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    typedef PermuteCfg<T> C;
    constexpr int V = C::V, CHB = C::CHB, NCH = C::NCH, NCHT = C::NCHT, B = T::kBlock;
    const int lane = threadIdx.x & 31;
    const bool is_mover = lane < V;
    const SubDesc sub = ws.subs[j];
    const u32 nb = sub.nbuckets;
    const int logL = (int)sub.log_leaves;
    const bool eq = sub.eq != 0;
    u64* wr = ws.wr + (u64)j * kMaxBuckets;
    u32* exh = ws.exhausted + (u64)j * 8;
    E* A = arr + sub.begin;
    E* ovf = ws.overflow + (u64)j * B;
    const u64 nbc = sub.n / B;                   // complete block slots
    const bool partial = (sub.n % B) != 0;

    // per-lane mover state (lanes >= V never become active)
    u32 prim = is_mover ? (u32)(((u64)(gl * V + lane) * nb) / nmov) : 0u;
    u32 tgt = 0, hand = 0;                     // hand: which of the two buffers holds the carried block
    bool have = false, done = !is_mover;
    u32 exw[8];
#pragma unroll
    for (int w8 = 0; w8 < 8; ++w8) exw[w8] = 0;
    if (join && is_mover) {
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) exw[w8] = ld_relaxed(&exh[w8]);
        const u32 np = first_live_bucket(exw, prim);
        if (np == 0xffffffffu || np >= nb) done = true;
        else prim = np;
    }
    for (;;) {
        if (!__any_sync(0xffffffffu, !done) || failed) break;
        // ---- one claim per active mover.  The read claims of the lanes that
        // share a primary bucket are one atomic (r - count, readers + 1): the
        // lane of rank q in the group reads block r - q, and the group holds
        // one reader count until the warp has loaded its blocks, so the count
        // is bounded by the warps of a subproblem, not by its movers.
        u64 old = 0;
        const bool rclaim = !done && !have;
        const unsigned rmask = __ballot_sync(0xffffffffu, rclaim);
        u32 rrank = 0;
        bool holds_reader = false;
        if (rclaim) {
            const unsigned grp = __match_any_sync(rmask, prim);
            const int lead = __ffs(grp) - 1;
            rrank = (u32)__popc(grp & ((1u << lane) - 1u));
            u64 o = 0;
            if (lane == lead) o = atomicAdd(&wr[prim], 1ull - ((u64)__popc(grp) << kRdBits));
            old = __shfl_sync(grp, o, lead);
            if (lane == lead) {
                if (pk_r(old) < pk_w(old)) red_add_relaxed64(&wr[prim], kReadDone);   // no lane got a block: undo
                else holds_reader = true;
            }
        } else if (!done) {
            old = atom_add_acquire(&wr[tgt], kClaimWrite);
        }
        const long long w = pk_w(old), r = pk_r(old) - (long long)rrank;
        const u32 rd = pk_readers(old);
        bool ldn = false, ldt = false, emp = false, exd = false;
        u64 slot = 0;
        if (!done) {
            if (!have) {
                if (r < w) {
                    // no unprocessed block left in the primary bucket
                    atomicOr(&exh[prim >> 5], 1u << (prim & 31));
                    exd = true;
                } else {
                    slot = (u64)delim[prim] + (u64)r;
                    if (IPS4O_GUARD(ws.ctr, r >= 0 && slot < nbc, slot, nbc)) ldn = true;
                    else failed = true;
                }
            } else {
                slot = (u64)delim[tgt] + (u64)w;
                if (!IPS4O_GUARD(ws.ctr, slot < delim[tgt + 1], slot, delim[tgt + 1])) {
                    failed = true;
                } else if (w <= r) {
                    if (IPS4O_GUARD(ws.ctr, slot < nbc, slot, nbc)) ldt = true;
                    else failed = true;
                } else {
                    emp = true;
                }
            }
        }
        if (__any_sync(0xffffffffu, failed)) { failed = true; break; }
        // ---- block loads of all movers, one coalesced copy per block
        {
            unsigned m = __ballot_sync(0xffffffffu, ldn || ldt);
            while (m) {
                const int v = __ffs(m) - 1;
                m &= m - 1;
                const u64 sv = __shfl_sync(0xffffffffu, slot, v);
                const u32 hb = __shfl_sync(0xffffffffu, hand, v) ^ 1u;      // the free buffer
                char* dst = (char*)(wbuf + ((size_t)hb * V + v) * B);
                const char* src = (const char*)(A + sv * B);
#pragma unroll
                for (int q = 0; q < NCH; ++q)
                    if (NCHT % 32 == 0 || lane + 32 * q < NCHT)
                        cp_async<CHB>(dst + CHB * (lane + 32 * q), src + CHB * (lane + 32 * q));
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp();
        }
        // The warp barrier orders every lane's copies of the claimed blocks
        // before the release that drops the reader count (release is
        // cumulative): a writer that sees the count drained cannot overwrite
        // a slot that is still being read.  Counts are dropped before this
        // warp waits on any count, so movers of one warp never wait on each
        // other.
        if (holds_reader) red_add_release64(&wr[prim], kReadDone);
        // ---- writes into empty slots (after the reader counts drained)
        bool ok = true;
        if (emp && rd != 0) {
            u32 it = 0;
            while (pk_readers(ld_acquire64(&wr[tgt])) != 0) {
                if (++it > spin_limit) { ok = false; break; }
                __nanosleep(32);
            }
        }
        if (!ok) set_status(ws.ctr, kStatusTimeout);
        if (__any_sync(0xffffffffu, !ok)) { failed = true; break; }
        bool bad_slot = emp && !(slot < nbc || (partial && slot == nbc));
        if (bad_slot) IPS4O_GUARD(ws.ctr, false, slot, nbc);
        if (__any_sync(0xffffffffu, bad_slot)) { failed = true; break; }
        // ---- classify the head of every block just loaded
        int t = 0;
        if (ldn || ldt) {
            const E* blk = wbuf + ((size_t)(hand ^ 1u) * V + lane) * B;
            t = classify_key<K>(T::key(blk[0]), tree, spl, logL, eq);
            if (!IPS4O_GUARD(ws.ctr, t >= 0 && (u32)t < nb, t, nb)) failed = true;
        }
        if (__any_sync(0xffffffffu, failed)) { failed = true; break; }
        const bool swp = ldt && (u32)t != tgt;           // the slot's block must move on
        if (ldt && !swp) ++skipped;                       // already in its bucket: leave it
        // ---- stores: carried blocks into empty slots and swap slots
        {
            unsigned m = __ballot_sync(0xffffffffu, emp || swp);
            while (m) {
                const int v = __ffs(m) - 1;
                m &= m - 1;
                const u64 sv = __shfl_sync(0xffffffffu, slot, v);
                const u32 hb = __shfl_sync(0xffffffffu, hand, v);
                const char* src = (const char*)(wbuf + ((size_t)hb * V + v) * B);
                char* dst = (char*)(sv < nbc ? A + sv * B : ovf);
#pragma unroll
                for (int q = 0; q < NCH; ++q) {
                    if (NCHT % 32 != 0 && lane + 32 * q >= NCHT) continue;
                    const int off = CHB * (lane + 32 * q);
                    if constexpr (CHB == 16) *(uint4*)(dst + off) = *(const uint4*)(src + off);
                    else if constexpr (CHB == 8) *(u64*)(dst + off) = *(const u64*)(src + off);
                    else *(u32*)(dst + off) = *(const u32*)(src + off);
                }
            }
            __syncwarp();
        }
        if (emp) { have = false; ++moved; }
        if (swp) { hand ^= 1u; tgt = (u32)t; ++moved; }
        if (ldn) { hand ^= 1u; tgt = (u32)t; have = true; }
        // ---- movers whose primary bucket ran dry pick the next live one
        if (__any_sync(0xffffffffu, exd)) {
            if (exd) {
#pragma unroll
                for (int w8 = 0; w8 < 8; ++w8) exw[w8] = ld_relaxed(&exh[w8]);
                // first non-exhausted bucket after prim, cyclically
                const u32 np = first_live_bucket(exw, prim + 1u);
                if (np == 0xffffffffu) done = true;
                else if (IPS4O_GUARD(ws.ctr, np < nb, np, nb)) prim = np;
                else { failed = true; done = true; }
            }
        }
    }
}

constexpr u32 kJoinNone = 0xffffffffu;
constexpr u32 kJoinRetry = 0xfffffffeu;

// For a CTA of k_permute whose own groups are done: the subproblem of the
// round with the most estimated unprocessed blocks per CTA working on it
// (r_i - w_i + 1 summed over 8 sampled buckets, scaled to all buckets),
// kJoinNone when none has 4 blocks per mover left, kJoinRetry when the
// chosen one filled up meanwhile.  Thread 0 counts the CTA in ws.movers; all
// threads receive the index.  s_red: NW + 1 words of shared memory.
//
// The cap on CTAs per subproblem also bounds how far r_i may fall below
// w_i - 1: every mover fails a read claim on a bucket at most once per
// group, and a group that joins starts its movers only on buckets the
// exhausted bitmap does not mark; a subproblem is joined only while all movers
// of the grid together with its own cap stay below the bias kRBias.
template <class T>
__device__ u32 pick_join(const Workspace<T>& ws, u32 nsub, u32 G, u32 salt, u64* s_red) {
    typedef PermuteCfg<T> C;
    constexpr int TPB = C::TPB, NW = C::NW;
    constexpr u32 MOV = (u32)NW * C::V;
    u64 best = 0;                                // score << 32 | tie-break << 16 | subproblem
    for (u32 i = threadIdx.x; i < nsub; i += TPB) {
        const u32 nb = ws.subs[i].nbuckets;
        if (nb == 0 || nb > (u32)kMaxBuckets || ws.subs[i].blocks_total == 0) continue;
        const u64 cap_b = ((u64)nb * C::MAX_MOVERS_PER_BUCKET + MOV - 1) / MOV;
        if (((u64)G + cap_b) * MOV >= kRBias) continue;
        const u32 act = ld_relaxed(&ws.movers[i]);
        if (act >= cap_b) continue;
        const u64* wr = ws.wr + (u64)i * kMaxBuckets;
        u64 rem = 0;
#pragma unroll
        for (u32 q = 0; q < 8; ++q) {
            const u64 x = ld_relaxed64(&wr[(q * nb) >> 3]);
            const long long d = pk_r(x) - pk_w(x) + 1;
            rem += d > 0 ? (u64)d : 0ull;
        }
        rem = rem * nb / 8;
        if (rem < 4ull * MOV) continue;
        u64 score = rem * 256 / (act + 1);
        score = score < 0xffffffffull ? score : 0xffffffffull;
        const u64 tie = mix64(((u64)salt << 32) | i) >> 48;
        const u64 key = (score << 32) | (tie << 16) | i;
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y > best ? y : best;
    }
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 b = s_red[0];
        for (int w = 1; w < NW; ++w) b = s_red[w] > b ? s_red[w] : b;
        u32 j = kJoinNone;
        if (b != 0) {
            j = (u32)(b & 0xffffu);
            const u32 cap_b = (ws.subs[j].nbuckets * (u32)C::MAX_MOVERS_PER_BUCKET + MOV - 1) / MOV;
            if (atomicAdd(&ws.movers[j], 1u) >= cap_b) {
                atomicSub(&ws.movers[j], 1u);
                j = kJoinRetry;
            }
        }
        s_red[NW] = j;
    }
    __syncthreads();
    const u32 j = (u32)s_red[NW];
    __syncthreads();                             // s_red is read before the next pick writes it
    return j;
}

template <class T>
__global__ void __launch_bounds__(PermuteCfg<T>::TPB, PermuteCfg<T>::MIN_CTAS)
    k_permute(typename T::elem_t* arr, Workspace<T> ws, u32 nsub, u32 spin_limit) {
    typedef typename T::elem_t E;
    typedef typename T::key_t K;
    typedef PermuteCfg<T> C;
    constexpr int TPB = C::TPB, NW = C::NW, V = C::V, B = T::kBlock;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned short* s_gpre = (unsigned short*)(smem_raw + C::off_gpre);
    u64* s_misc = (u64*)(smem_raw + C::off_misc);   // [0] total, [1..33] scan tmp
    const int warp = threadIdx.x >> 5;
    if (ws.ls) nsub = ws.ls->nsub;                  // device-planned round
    const u32 G = gridDim.x;                      // CTAs in the grid
    constexpr u32 MOV = (u32)NW * V;              // movers of one CTA
    // CTAs per subproblem, in proportion to its full blocks (rounded down,
    // then one more for each of the first subproblems, the largest, until the
    // grid is used up), so that one wave of groups covers the round when it
    // has no more subproblems than CTAs; the warps of a CTA all work on one
    // subproblem and share its tables
    u64 mine = 0;
    for (u32 i = threadIdx.x; i < nsub; i += TPB) mine += ws.subs[i].blocks_total;
    if (threadIdx.x == 0) s_misc[0] = 0;
    __syncthreads();
    atomicAdd(&s_misc[0], mine);
    __syncthreads();
    const u64 total = s_misc[0];
    {
        constexpr int PER = 1024 / TPB;
        u32 gv[PER], cap[PER], sum = 0, below = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const u32 i = threadIdx.x * PER + q;
            gv[q] = 0;
            cap[q] = 0;
            if (i < nsub && total > 0) {
                const SubDesc& sd = ws.subs[i];
                const u64 bl = sd.blocks_total;
                if (bl > 0) {
                    u64 x = bl * (u64)G / total;
                    const u64 cap_b = ((u64)sd.nbuckets * C::MAX_MOVERS_PER_BUCKET + MOV - 1) / MOV;
                    const u64 cap_k = (bl + MOV - 1) / MOV;
                    const u64 cap_r = kMaxReadersPerSub / NW;
                    u64 c = cap_b < cap_k ? cap_b : cap_k;
                    c = c < cap_r ? c : cap_r;
                    c = c < 1 ? 1 : c;
                    x = x < c ? x : c;
                    gv[q] = (u32)(x < 1 ? 1 : x);
                    cap[q] = (u32)c;
                }
            }
            sum += gv[q];
            below += gv[q] < cap[q] ? 1u : 0u;
        }
        u32 tot, nbelow;
        block_exclusive_scan<u32>(sum, (u32*)(s_misc + 1), &tot);
        __syncthreads();                          // the scan's scratch is read before it is reused
        u32 rank = block_exclusive_scan<u32>(below, (u32*)(s_misc + 1), &nbelow);
        const u32 spare = tot < G ? G - tot : 0u;
        sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            if (gv[q] < cap[q]) {
                if (rank < spare) ++gv[q];
                ++rank;
            }
            sum += gv[q];
        }
        __syncthreads();
        u32 p = block_exclusive_scan<u32>(sum, (u32*)(s_misc + 1), &tot);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const u32 i = threadIdx.x * PER + q;
            if (i < nsub) s_gpre[i] = (unsigned short)p;
            p += gv[q];
        }
        if (threadIdx.x == 0) s_gpre[nsub] = (unsigned short)tot;
        __syncthreads();
    }
    const u32 GT = s_gpre[nsub];
    E* wbuf = (E*)(smem_raw + C::off_buf) + (size_t)warp * 2 * V * B;   // [2][V][B]
    K* tree = (K*)(smem_raw + C::off_tree);
    K* spl = (K*)(smem_raw + C::off_spl);
    u32* delim = (u32*)(smem_raw + C::off_delim);
    u64 moved = 0, skipped = 0;
    bool failed = false, cta_failed = false;
    for (u32 g = blockIdx.x; g < GT; g += G) {
        u32 lo = 0, hi = nsub;
        while (hi - lo > 1) { u32 mid = (lo + hi) >> 1; if (s_gpre[mid] <= g) lo = mid; else hi = mid; }
        const u32 j = lo;
        const u32 cl = g - s_gpre[j];
        const u32 nmov = (s_gpre[j + 1] - s_gpre[j]) * MOV;
        __syncthreads();                          // the previous group is done with the tables
        load_sub_tables<T>(ws, j, tree, spl, delim);
        if (threadIdx.x == 0) atomicAdd(&ws.movers[j], 1u);
        __syncthreads();
        permute_group<T>(arr, ws, j, cl * NW + warp, nmov, wbuf, tree, spl, delim, spin_limit, moved, skipped,
                         failed);
        cta_failed = __syncthreads_or(failed) != 0;
        if (threadIdx.x == 0) atomicSub(&ws.movers[j], 1u);
        if (cta_failed) break;
    }
    // A CTA whose groups are done joins a subproblem whose permutation still
    // has unprocessed blocks (the movers of a subproblem need not start
    // together), so that the round does not wait on the subproblems whose
    // CTAs had the most blocks each.
    for (u32 round = 0; round < C::MAX_JOINS && !cta_failed; ++round) {
        const u32 j = pick_join<T>(ws, nsub, G, blockIdx.x * C::MAX_JOINS + round, s_misc + 1);
        if (j == kJoinNone) break;
        if (j == kJoinRetry) continue;
        load_sub_tables<T>(ws, j, tree, spl, delim);
        __syncthreads();
        permute_group<T>(arr, ws, j, (u32)warp, MOV, wbuf, tree, spl, delim, spin_limit, moved, skipped, failed,
                         true);
        cta_failed = __syncthreads_or(failed) != 0;
        if (threadIdx.x == 0) atomicSub(&ws.movers[j], 1u);
    }
    if (moved) atomicAdd(&ws.ctr->blocks_moved, moved);
    if (skipped) atomicAdd(&ws.ctr->blocks_skipped, skipped);
}

// --------------------------------------------------------------- cleanup
// A bucket whose cleanup is done: buckets up to the base-case capacity go to
// the list of their base-case size class, sorted in shared memory by the
// kernels that follow; larger ones recurse (Section 4) as subproblems of the
// next level, appended to the next-level queue of a device-planned sort or
// to the chunk's task list of a host-planned one.
template <class T>
__device__ __forceinline__ void emit_bucket(const Workspace<T>& ws, Task task, u32 rec_cap) {
    const u64 size = task.n;
    if (size > (u64)rec_cap) {
        if (ws.ls && ws.ls->strict) return;       // marked by k_mark and found again by the scan
        if (ws.ls) {
            const u32 idx = atomicAdd(&ws.ls->next_count, 1u);
            if (idx < ws.next_cap) ws.ls->next_q[idx] = task;
            else set_status(ws.ctr, kStatusCapacity);
        } else {
            const u32 idx = atomicAdd(&ws.ctr->next_count, 1u);
            if (idx < ws.next_cap) ws.next_tasks[idx] = task;
            else set_status(ws.ctr, kStatusCapacity);
        }
    } else if (size <= (u64)T::kBaseTiny) {
        const u32 idx = atomicAdd(&ws.ctr->base_tiny, 1u);
        if (IPS4O_GUARD(ws.ctr, idx < ws.max_sub * kMaxBuckets, idx, ws.max_sub)) ws.base_tiny[idx] = task;
    } else if (size <= (u64)T::kBaseSmall) {
        const u32 idx = atomicAdd(&ws.ctr->base_small, 1u);
        if (IPS4O_GUARD(ws.ctr, idx < ws.max_sub * kMaxBuckets, idx, ws.max_sub)) ws.base_small[idx] = task;
    } else {
        const u32 idx = atomicAdd(&ws.ctr->base_large, 1u);
        if (IPS4O_GUARD(ws.ctr, idx < ws.max_sub * kMaxBuckets, idx, ws.max_sub)) ws.base_large[idx] = task;
    }
}

// A final range [begin, begin + size) of the array that the base case will
// not write to ws.out (an equality bucket, a single element, a subproblem
// the segment scheduler sorts in place): queued for the result copy in
// pieces of at most kCopyChunk elements.  One thread.
template <class T>
__device__ __forceinline__ void emit_copy(const Workspace<T>& ws, u64 begin, u64 size) {
    const u64 nch = (size + kCopyChunk - 1) / kCopyChunk;
    const u32 first = atomicAdd(&ws.ctr->copy_count, (u32)nch);
    for (u64 c = 0; c < nch; ++c) {
        const u64 b = begin + c * kCopyChunk, e = b + kCopyChunk < begin + size ? b + kCopyChunk : begin + size;
        if ((u64)first + c < ws.copy_cap) ws.copy_tasks[first + c] = Task{b, e - b};
        else set_status(ws.ctr, kStatusCapacity);
    }
}

// The result copy: src[t.begin, t.begin + t.n) to dst for every entry t of
// the copy list, one warp per entry.
template <class T>
__global__ void __launch_bounds__(256) k_copy_tasks(const typename T::elem_t* src, typename T::elem_t* dst,
                                                    const Task* tasks, const u32* count, u64 cap) {
    const u32 n = (u64)*count < cap ? *count : (u32)cap;
    const int lane = threadIdx.x & 31;
    const u32 warps = gridDim.x * (blockDim.x / 32);
    for (u32 i = (blockIdx.x * blockDim.x + threadIdx.x) / 32; i < n; i += warps) {
        const Task t = tasks[i];
#pragma unroll 4
        for (u64 k = lane; k < t.n; k += 32) dst[t.begin + k] = src[t.begin + k];
    }
}

// One warp per (subproblem, bucket), taken in ticket order; WPC warps per CTA
// (subproblems with few stripes: the lower levels).
template <class T>
struct CleanupCfg {
    typedef typename T::elem_t E;
    static constexpr int TPB = 256;
    static constexpr int WPC = TPB / 32;
    static constexpr int B = T::kBlock;
    static constexpr size_t off_ov = 0;                                 // E[WPC][B] overshoot per warp
    static constexpr size_t smem_bytes = a16(off_ov + (size_t)WPC * B * sizeof(E));
};

// Cleanup of bucket b of subproblem j by one warp (Section 4.3): its
// overshoot is read first and published with a flag; its head is written
// only after the owner of block slot d_b - 1 has published; then the
// sources (overshoot, overflow block, partial buffers of every stripe in
// stripe order) fill the head and tail slots, and the bucket is queued for
// the base case or the next level.
template <class T>
__device__ __forceinline__ void cleanup_bucket_warp(typename T::elem_t* arr, const Workspace<T>& ws, u32 j, u32 b,
                                                    typename T::elem_t* s_ov, u32 spin_limit, u32 partition_only,
                                                    u32 rec_cap) {
    typedef typename T::elem_t E;
    constexpr int B = T::kBlock;
    const int lane = threadIdx.x & 31;
    const SubDesc sub = ws.subs[j];
    const u32 nb = sub.nbuckets;
    if (b >= nb) return;
    E* A = arr + sub.begin;
    const u64* bstart = ws.bstart + (u64)j * (kMaxBuckets + 1);
    const u32* dl = ws.delim + (u64)j * (kMaxBuckets + 1);
    const u64 Bb = bstart[b], Eb = bstart[b + 1];
    const u32 d0 = dl[b];
    const u64 w = (u64)d0 + (u64)pk_w(ws.wr[(u64)j * kMaxBuckets + b]);
    const u64 nbc = sub.n / B;
    const bool partial = (sub.n % B) != 0;
    const bool has_blocks = w > d0;
    // the bucket's last full block went to the overflow block
    const u32 ovf = (partial && has_blocks && w == nbc + 1) ? (u32)B : 0u;
    const u64 P_lo = (u64)d0 * B;
    const u64 P_hi = has_blocks ? (ovf ? nbc : w) * B : P_lo;    // end of its blocks in the array
    const u32 ov = (u32)((has_blocks && P_hi > Eb) ? P_hi - Eb : 0);  // overshoot into the next head
    const bool bad = ov > (u32)B || Eb < Bb || Eb > sub.n;
    // read the overshoot before a later bucket may overwrite that head
    if (!bad)
        for (u32 v = lane; v < ov; v += 32) s_ov[v] = A[Eb + v];
    __syncwarp();
    u32* flags = ws.flags + (u64)j * kMaxBuckets;
    u32 ok = 1;
    if (lane == 0) {
        st_release(&flags[b], 1u);
        // this bucket's head [Bb, d0 * b) lies in block slot d0 - 1, the last
        // slot of the region of bucket x, the last bucket before this one
        // whose region starts below d0 (buckets in between are smaller than
        // a block and share d0): only x's blocks can overshoot into it
        int x = (int)b - 1;
        while (x >= 0 && dl[x] >= d0) --x;
        if (x >= 0 && !wait_flag_set(&flags[x], spin_limit)) ok = 0;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
        if (lane == 0) set_status(ws.ctr, kStatusTimeout);
        return;
    }
    // empty slots: head [Bb, min(P_lo, Eb)) and tail [P_hi, Eb)
    const u64 head_hi = P_lo < Eb ? P_lo : Eb;
    const u64 nh = head_hi > Bb ? head_hi - Bb : 0;
    const u64 nt = (P_lo < Eb && P_hi < Eb) ? Eb - P_hi : 0;
    const u32 ns = sub.num_stripes, sb = sub.stripe_begin;
    u64 ltot = 0;
    for (u32 i0 = 0; i0 < ns; i0 += 32) {
        const u32 i = i0 + lane;
        const u32 c = i < ns ? ws.counts[(u64)(sb + i) * kMaxBuckets + b] % B : 0u;
        ltot += __reduce_add_sync(0xffffffffu, c);
    }
    const u64 nsrc = (u64)ov + ovf + ltot;
    if (bad || nh + nt != nsrc) {
        if (lane == 0) set_status(ws.ctr, kStatusInternal);
        return;
    }
    auto dst_of = [&](u64 q) -> u64 { return q < nh ? Bb + q : P_hi + (q - nh); };
    for (u32 q = lane; q < ov; q += 32) A[dst_of(q)] = s_ov[q];
    const E* ovb = ws.overflow + (u64)j * B;
    for (u32 q = lane; q < ovf; q += 32) A[dst_of(ov + q)] = ovb[q];
    // partial buffers, stripe by stripe
    u64 at = (u64)ov + ovf;
    for (u32 i = 0; i < ns; ++i) {
        const u64 si = (u64)(sb + i) * kMaxBuckets + b;
        const u32 c = ws.counts[si] % B;
        if (c == 0) continue;
        const E* src = ws.pool + ws.stripes[sb + i].pool_off + ws.lscan[si];
        for (u32 v = lane; v < c; v += 32) A[dst_of(at + v)] = src[v];
        at += c;
    }
    if (partition_only) return;
    const u64 size = Eb - Bb;
    const bool is_eq = sub.eq && (b & 1);
    if (lane != 0) return;
    if (is_eq || size < 2) {                        // final: all keys equal, or one element
        if (ws.out && size > 0) emit_copy<T>(ws, sub.begin + Bb, size);
        return;
    }
    emit_bucket<T>(ws, Task{sub.begin + Bb, size}, rec_cap);
}

template <class T>
__global__ void __launch_bounds__(CleanupCfg<T>::TPB)
    k_cleanup(typename T::elem_t* arr, Workspace<T> ws, u32 nsub, u32 bstride, u32 spin_limit, u32 partition_only,
              u32 rec_cap) {
    typedef typename T::elem_t E;
    typedef CleanupCfg<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (ws.ls) {                                    // device-planned round: this variant or the CTA one
        if (ws.ls->cta_cleanup) return;
        nsub = ws.ls->nsub;
        bstride = ws.ls->bstride;
    }
    E* s_ov = (E*)(smem_raw + C::off_ov) + (size_t)warp * C::B;
    // tickets enumerate (subproblem, bucket) with bstride >= the chunk's
    // largest bucket count, in increasing bucket order within a subproblem;
    // a warp takes its next ticket only after finishing the last, so every
    // bucket a cleanup waits for is held by a running warp or done
    for (;;) {
        u32 ticket = 0;
        if (lane == 0) ticket = atomicAdd(&ws.ctr->ticket, 1u);
        ticket = __shfl_sync(0xffffffffu, ticket, 0);
        const u32 j = ticket / bstride, b = ticket % bstride;
        if (j >= nsub) return;
        if (b == 0 && lane == 0) IPS4O_GUARD(ws.ctr, ws.subs[j].nbuckets <= bstride, ws.subs[j].nbuckets, bstride);
        cleanup_bucket_warp<T>(arr, ws, j, b, s_ov, spin_limit, partition_only, rec_cap);
        __syncwarp();
    }
}

// ------------------------------------------------- cleanup, CTA per bucket
// For subproblems with many stripes (the top level), where a bucket gathers
// partial buffers from hundreds of stripes: one CTA per bucket.
template <class T>
struct CleanupCtaCfg {
    typedef typename T::elem_t E;
    static constexpr int TPB = 256;
    static constexpr int B = T::kBlock;
    static constexpr size_t off_ov = 0;
    static constexpr size_t off_lpre = a16(off_ov + (size_t)B * sizeof(E));
    static constexpr size_t off_src = a16(off_lpre + (size_t)(kMaxStripesPerSub + 1) * 4 + 4);
    static constexpr size_t smem_bytes = a16(off_src + (size_t)kMaxStripesPerSub * 8);
    // 100-byte records leave B * sizeof(E) a multiple of 4 only: the tables
    // after the block start on their own 16-byte boundary
    static_assert(off_lpre % 16 == 0 && off_src % 16 == 0, "aligned tables");
};

// Cleanup of bucket b of subproblem j by the whole CTA (CleanupCtaCfg<T>::TPB
// threads): the same steps as cleanup_bucket_warp, with the partial buffers
// of many stripes gathered in parallel.
template <class T>
__device__ void cleanup_bucket_cta(typename T::elem_t* arr, const Workspace<T>& ws, u32 j, u32 b, u32 bstride,
                                   u32 spin_limit, u32 partition_only, u32 rec_cap, unsigned char* smem_raw,
                                   u32* s_ok_p, u32* tmp) {
    typedef typename T::elem_t E;
    typedef CleanupCtaCfg<T> C;
    constexpr int TPB = C::TPB, B = C::B;
    E* s_ov = (E*)(smem_raw + C::off_ov);
    u32* s_lpre = (u32*)(smem_raw + C::off_lpre);
    u64* s_src = (u64*)(smem_raw + C::off_src);
    u32& s_ok = *s_ok_p;
    const SubDesc sub = ws.subs[j];
    const u32 nb = sub.nbuckets;
    if (b == 0 && threadIdx.x == 0) IPS4O_GUARD(ws.ctr, nb <= bstride, nb, bstride);
    if (b >= nb) return;
    E* A = arr + sub.begin;
    const u64* bstart = ws.bstart + (u64)j * (kMaxBuckets + 1);
    const u64 Bb = bstart[b], Eb = bstart[b + 1];
    const u32 d0 = ws.delim[(u64)j * (kMaxBuckets + 1) + b];
    const u64 w = (u64)d0 + (u64)pk_w(ws.wr[(u64)j * kMaxBuckets + b]);
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
        // This bucket's head [Bb, d0 * b) lies in block slot d0 - 1, the last
        // slot of the region of bucket x, the last bucket before this one
        // whose region starts below d0 (buckets in between are smaller than a
        // block and share d0).  Only x's blocks can overshoot into that slot,
        // so the head may be written once x has read its overshoot.
        const u32* dl = ws.delim + (u64)j * (kMaxBuckets + 1);
        int x = (int)b - 1;
        while (x >= 0 && dl[x] >= d0) --x;
        u32 ok = 1;
        if (x >= 0 && !wait_flag_set(&flags[x], spin_limit)) ok = 0;
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
    if (is_eq || size < 2) {                        // final: all keys equal, or one element
        if (ws.out && size > 0 && threadIdx.x == 0) emit_copy<T>(ws, sub.begin + Bb, size);
        return;
    }
    if (threadIdx.x == 0) emit_bucket<T>(ws, Task{sub.begin + Bb, size}, rec_cap);
}

template <class T>
__global__ void __launch_bounds__(CleanupCtaCfg<T>::TPB)
    k_cleanup_cta(typename T::elem_t* arr, Workspace<T> ws, u32 nsub, u32 bstride, u32 spin_limit, u32 partition_only,
              u32 rec_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ u32 s_ticket, s_ok;
    __shared__ u32 tmp[32];
    if (ws.ls) {                                    // device-planned round: this variant or the warp one
        if (!ws.ls->cta_cleanup) return;
        nsub = ws.ls->nsub;
        bstride = ws.ls->bstride;
    }
    // tickets enumerate (subproblem, bucket) with bstride >= the chunk's
    // largest bucket count, in increasing bucket order within a subproblem;
    // a CTA takes its next ticket only after finishing the last
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_ticket = atomicAdd(&ws.ctr->ticket, 1u);
        __syncthreads();
        const u32 ticket = s_ticket;
        const u32 j = ticket / bstride, b = ticket % bstride;
        if (j >= nsub) return;
        cleanup_bucket_cta<T>(arr, ws, j, b, bstride, spin_limit, partition_only, rec_cap, smem_raw, &s_ok, tmp);
    }
}

}  // namespace ips4o
