// ips4o_rounds.cuh — the recursion of Section 4 planned on the device, so
// that a sort is enqueued work only (no host synchronisation between
// levels; the call can be captured in a CUDA graph).
//
// The subproblems of a level are a queue in device memory.  A round takes
// the next chunk of that queue: k_plan (one CTA) picks as many subproblems as
// the workspace holds, lays out their stripes and writes the chunk's
// descriptors; the distribution-step kernels then run the chunk, reading its
// size from the loop state, and the cleanup appends the buckets that must
// recurse to the other queue (the next level).  When the current queue is
// used up, k_plan swaps the queues.  The host enqueues a fixed number of
// rounds computed from n (the nominal depth log_k(n / base case) and the
// chunks per level, plus one); subproblems still left after the last round
// are sorted by the segment scheduler (one CTA per subproblem), which
// handles any size.
#pragma once

#include "ips4o_segments.cuh"

namespace ips4o {

constexpr u64 kMinStripe = 1u << 16;     // elements; keeps leftovers small relative to a stripe

// Arguments of k_plan (by value).
struct PlanArgs {
    u64 n;              // elements of the whole sort
    u32 first;          // 1 for the first round: the queue starts as the whole input
    u32 k_max;          // largest number of leaves of a step
    u32 alpha;          // oversampling factor (0: the default, 16)
    u32 base_cap;       // base-case class the adaptive number of leaves aims at (half of it per bucket)
    u32 sms;            // SMs: stripes should fill whole waves of them
    u32 w0;             // fewest stripes per SM tried for a level
    u32 newlevel;       // strict recursion: this round starts a batch (planned like a new level)
    u32 level;          // strict recursion: the batch's number (the sampling seed depends on it)
};

// Stripes of a subproblem of n elements for the level's stripe length len:
// ns stripes of slen elements (a multiple of the block), the last shorter;
// need = partial-buffer elements they may leave in the pool.
__device__ __forceinline__ void plan_task(u64 n, u64 len, u64 B, u32 max_ns, u32* ns_out, u64* slen_out,
                                          u64* need_out) {
    const u64 per = (u64)kMaxBuckets * (B - 1);
    u64 ns = (n + len - 1) / len;
    ns = ns < 1 ? 1 : (ns > max_ns ? max_ns : ns);
    const u64 slen = ((n + ns - 1) / ns + B - 1) / B * B;
    ns = (n + slen - 1) / slen;
    const u64 last = n - (ns - 1) * slen;
    *ns_out = (u32)ns;
    *slen_out = slen;
    *need_out = (ns - 1) * (slen < per ? slen : per) + (last < per ? last : per);
}

template <typename V>
__device__ __forceinline__ V block_sum(V v, V* tmp) {
    V t;
    block_exclusive_scan<V>(v, tmp, &t);
    __syncthreads();
    return t;
}

// Fold the counters of the chunk that just ran into the loop state and clear
// them for the next one (one thread).
__device__ __forceinline__ void fold_counters(LoopState* ls, ChunkCounters* c) {
    ls->blocks_moved += c->blocks_moved;
    ls->blocks_skipped += c->blocks_skipped;
    ls->fix_blocks += c->fix_blocks;
    ls->base_buckets += c->base_buckets;
    ls->status |= c->status;
    if (c->guard_hits && !ls->guard_hits) {
        ls->guard_line = c->guard_line;
        ls->guard_a = c->guard_a;
        ls->guard_b = c->guard_b;
    }
    ls->guard_hits += c->guard_hits;
    *c = ChunkCounters{};
}

// One round's plan (one CTA of 1024 threads).
template <class T>
__global__ void __launch_bounds__(1024) k_plan(Workspace<T> ws, PlanArgs pa) {
    constexpr u64 B = T::kBlock;
    constexpr int TPB = 1024;
    LoopState* ls = ws.ls;
    __shared__ u64 s_n[TPB];
    __shared__ u64 s_beg[TPB];
    __shared__ u64 s_key[TPB];
    __shared__ u32 s_ns[TPB], s_sb[TPB];
    __shared__ u64 s_tmp64[32];
    __shared__ u32 s_tmp32[32];
    __shared__ u32 s_work, s_newlevel, s_m, s_ns0;
    const int tid = threadIdx.x;
    if (tid == 0) {
        if (pa.first) {
            *ls = LoopState{};
            ls->cur_q = ws.next_tasks;
            ls->next_q = ws.next_tasks2;
            ls->cur_q[0] = Task{0, pa.n};
            ls->cur_count = 1;
            *ws.ctr = ChunkCounters{};
        } else {
            fold_counters(ls, ws.ctr);
        }
        s_newlevel = pa.first | pa.newlevel;
        if (pa.newlevel) ls->level = pa.level;
        if (ls->next_count > ws.next_cap) ls->status |= kStatusCapacity;   // (cannot happen: buckets are disjoint)
        if (!pa.first && ls->status == 0 && ls->cur_pos >= ls->cur_count && ls->next_count > 0) {
            Task* t = ls->cur_q;
            ls->cur_q = ls->next_q;
            ls->next_q = t;
            ls->cur_count = ls->next_count;
            ls->next_count = 0;
            ls->cur_pos = 0;
            ls->level += 1;
            s_newlevel = 1;
        }
        s_work = ls->status == 0 && ls->cur_pos < ls->cur_count;
        if (!s_work) {
            ls->nsub = 0;
            ls->nstr = 0;
            ls->bstride = 1;
            ls->cta_cleanup = 0;
        }
    }
    __syncthreads();
    if (!s_work) return;
    const Task* q = ls->cur_q;
    const u32 cnt = ls->cur_count, pos = ls->cur_pos;
    if (s_newlevel) {
        // Stripe length of the level: classification CTAs (one per SM) take
        // stripes dynamically, so the stripe count should fill whole waves.
        // Stripes never cross a subproblem, so the count is a sum of per-
        // subproblem roundings: try w0, w0 + 1, ... stripes per SM and keep
        // the count whose last wave is fullest, with a small charge for
        // extra stripes (more partial buffers to clean up).
        u64 part = 0, pmax = 0;
        for (u32 i = tid; i < cnt; i += TPB) {
            part += q[i].n;
            pmax = q[i].n > pmax ? q[i].n : pmax;
        }
        const u64 total = block_sum<u64>(part, s_tmp64);
        for (int o = 16; o > 0; o >>= 1) {
            const u64 v = __shfl_xor_sync(0xffffffffu, pmax, o);
            pmax = v > pmax ? v : pmax;
        }
        if ((tid & 31) == 0) s_n[tid >> 5] = pmax;
        __syncthreads();
        u64 nmax = 0;
        for (int w = 0; w < TPB / 32; ++w) nmax = s_n[w] > nmax ? s_n[w] : nmax;
        __syncthreads();
        const u32 w1 = cnt <= ws.max_sub ? pa.w0 + 6 : pa.w0;
        u64 best_len = 0;
        double best_score = -1e30;
        for (u32 wv = pa.w0; wv <= w1; ++wv) {
            const u64 K = (u64)wv * pa.sms;
            u64 len = (total + K - 1) / K;
            len = len < kMinStripe ? kMinStripe : len;
            len = (len + B - 1) / B * B;
            if (K >= cnt && nmax > len) {
                // With subproblems of unequal sizes the length total / K
                // rounds each of them up to whole stripes and gives fewer,
                // uneven waves (256 subproblems of about 2^20 keys, one
                // stripe each, are 1.68 waves of 152 SMs).  The smallest
                // length (in blocks) whose stripes number at most K splits
                // only the largest subproblems and fills the waves.
                u64 lo = len / B, hi = (nmax + B - 1) / B;   // count(hi * B) = cnt <= K
                for (int it = 0; it < 24 && lo < hi; ++it) {
                    const u64 mid = (lo + hi) / 2;
                    u64 c = 0;
                    for (u32 i = tid; i < cnt; i += TPB) c += (q[i].n + mid * B - 1) / (mid * B);
                    c = block_sum<u64>(c, s_tmp64);
                    if (c <= K) hi = mid;
                    else lo = mid + 1;
                }
                len = hi * B;
            }
            u64 ns_part = 0, pool_part = 0;
            for (u32 i = tid; i < cnt; i += TPB) {
                u32 ns;
                u64 slen, need;
                plan_task(q[i].n, len, B, kMaxStripesPerSub, &ns, &slen, &need);
                ns_part += ns;
                pool_part += need;
            }
            const u64 tot_ns = block_sum<u64>(ns_part, s_tmp64);
            const u64 tot_pool = block_sum<u64>(pool_part, s_tmp64);
            // more stripes than a chunk holds would split the level into
            // more chunks: only the first candidate may do that
            if (wv > pa.w0 && (tot_ns > ws.max_stripes || tot_pool > ws.pool_cap)) break;
            const u64 waves = (tot_ns + pa.sms - 1) / pa.sms;
            const double score = (double)tot_ns / (double)(waves * pa.sms) - 0.02 * (double)(wv - pa.w0);
            if (score > best_score + 1e-9) {
                best_score = score;
                best_len = len;
            }
            if (len == kMinStripe) break;               // shorter stripes are not allowed
            if (tot_ns == waves * pa.sms) break;       // full waves: later candidates cannot score higher
        }
        if (tid == 0) {
            ls->stripe_len = best_len;
            ls->levels = ls->level + 1;
        }
        __syncthreads();
    }
    const u64 len = ls->stripe_len;
    // the chunk: the longest prefix of the remaining queue whose stripes and
    // partial buffers fit the workspace (prefix sums in queue order)
    const u32 m_max = cnt - pos < ws.max_sub ? cnt - pos : ws.max_sub;
    u32 ns_i = 0;
    u64 need_i = 0, slen_i = 0;
    if ((u32)tid < m_max) plan_task(q[pos + tid].n, len, B, kMaxStripesPerSub, &ns_i, &slen_i, &need_i);
    u32 tot_ns32;
    const u32 ex_ns = block_exclusive_scan<u32>(ns_i, s_tmp32, &tot_ns32);
    __syncthreads();
    u64 tot_need;
    const u64 ex_need = block_exclusive_scan<u64>(need_i, s_tmp64, &tot_need);
    __syncthreads();
    const bool fits = (u32)tid < m_max && ex_ns + ns_i <= ws.max_stripes && ex_need + need_i <= ws.pool_cap;
    const u32 m_fit = (u32)__syncthreads_count(fits);
    if (tid == 0) {
        s_m = m_fit;
        s_ns0 = 0;
        if (m_fit == 0) {
            // the first subproblem alone: fewer, longer stripes until it fits
            u64 n0 = q[pos].n;
            u32 ns = ns_i;
            for (;;) {
                const u64 sl = ((n0 + ns - 1) / ns + B - 1) / B * B;
                const u64 nsr = (n0 + sl - 1) / sl;
                const u64 per = (u64)kMaxBuckets * (B - 1);
                const u64 need = (nsr - 1) * (sl < per ? sl : per) + ((n0 - (nsr - 1) * sl) < per ? n0 - (nsr - 1) * sl : per);
                if ((nsr <= ws.max_stripes && need <= ws.pool_cap) || ns == 1) {
                    s_ns0 = (u32)nsr;
                    break;
                }
                ns = ns / 2 ? ns / 2 : 1;
            }
            s_m = 1;
        }
    }
    __syncthreads();
    const u32 m = s_m;
    // largest subproblems first (the block permutation hands out its movers
    // in this order too)
    u32 P = 1;
    while (P < m) P <<= 1;
    s_n[tid] = (u32)tid < m ? q[pos + tid].n : 0;
    s_beg[tid] = (u32)tid < m ? q[pos + tid].begin : 0;
    __syncthreads();
    for (u32 k = 2; k <= P; k <<= 1) {
        for (u32 jj = k >> 1; jj > 0; jj >>= 1) {
            const u32 i = (u32)tid, ixj = i ^ jj;
            if (i < P && ixj > i) {
                const bool desc = (i & k) == 0;
                const u64 a = s_n[i], b = s_n[ixj];
                if (desc ? a < b : a > b) {
                    s_n[i] = b;
                    s_n[ixj] = a;
                    const u64 t = s_beg[i];
                    s_beg[i] = s_beg[ixj];
                    s_beg[ixj] = t;
                }
            }
            __syncthreads();
        }
    }
    // stripes and pool areas of the sorted chunk, then its descriptors
    ns_i = 0;
    need_i = 0;
    slen_i = 0;
    u64 n_i = 0;
    u32 k_i = 0;
    if ((u32)tid < m) {
        n_i = s_n[tid];
        plan_task(n_i, len, B, kMaxStripesPerSub, &ns_i, &slen_i, &need_i);
        if (s_ns0) {                                    // the one oversized subproblem
            const u64 sl = ((n_i + s_ns0 - 1) / s_ns0 + B - 1) / B * B;
            ns_i = (u32)((n_i + sl - 1) / sl);
            slen_i = sl;
        }
    }
    const u32 sbeg = block_exclusive_scan<u32>(ns_i, s_tmp32, &tot_ns32);
    __syncthreads();
    u64 pool_base = 0;
    {
        // pool offsets: each stripe takes min(k (b - 1), its length)
        const u64 per = (u64)kMaxBuckets * (B - 1);
        u64 mine = 0;
        if ((u32)tid < m) {
            const u64 last = n_i - (u64)(ns_i - 1) * slen_i;
            mine = (u64)(ns_i - 1) * (slen_i < per ? slen_i : per) + (last < per ? last : per);
        }
        u64 tot;
        pool_base = block_exclusive_scan<u64>(mine, s_tmp64, &tot);
        __syncthreads();
    }
    if ((u32)tid < m) {
        const int cls = 63 - __clzll((long long)n_i);
        u32 K = c_class_leaves[cls];
        if (K == 0) K = seg_leaves(n_i, (u64)pa.base_cap, pa.k_max);
        u32 alpha = pa.alpha > 0 ? pa.alpha : 16u;
        if (c_class_alpha[cls]) alpha = c_class_alpha[cls];
        if (alpha * K > (u32)T::kSampleMax) alpha = (u32)T::kSampleMax / K;
        if (alpha < 1) alpha = 1;
        k_i = K;
        SubDesc sd;
        sd.begin = s_beg[tid];
        sd.n = n_i;
        sd.stripe_begin = sbeg;
        sd.num_stripes = ns_i;
        sd.k_target = K;
        sd.alpha = alpha;
        sd.level = ls->level;
        sd.log_leaves = 0;
        sd.eq = 0;
        sd.nbuckets = 0;
        sd.blocks_total = 0;
        ws.subs[tid] = sd;
        const u64 per = (u64)kMaxBuckets * (B - 1);
        u64 po = pool_base;
        for (u32 s = 0; s < ns_i; ++s) {
            StripeDesc x;
            x.begin = sd.begin + (u64)s * slen_i;
            x.end = sd.begin + ((u64)(s + 1) * slen_i < n_i ? (u64)(s + 1) * slen_i : n_i);
            x.pool_off = po;
            const u64 l = x.end - x.begin;
            x.pool_cap = (u32)(l < per ? l : per);
            x.sub = (u32)tid;
            po += x.pool_cap;
            ws.stripes[sbeg + s] = x;
        }
    }
    // chunk-wide values: largest leaves, most stripes, elements
    u32 kmax_part = k_i, nsmax_part = ns_i;
    for (int o = 16; o > 0; o >>= 1) {
        kmax_part = max(kmax_part, __shfl_xor_sync(0xffffffffu, kmax_part, o));
        nsmax_part = max(nsmax_part, __shfl_xor_sync(0xffffffffu, nsmax_part, o));
    }
    if ((tid & 31) == 0) {
        s_tmp32[tid >> 5] = kmax_part;
        s_n[tid >> 5] = nsmax_part;                       // s_n is free again
    }
    const u64 elems = block_sum<u64>(n_i, s_tmp64);
    if (tid == 0) {
        u32 kk = 1, nsm = 1;
        for (int w = 0; w < TPB / 32; ++w) {
            kk = max(kk, s_tmp32[w]);
            nsm = max(nsm, (u32)s_n[w]);
        }
        ls->nsub = m;
        ls->nstr = tot_ns32;
        ls->bstride = kk >= 4 ? (kk < (u32)kMaxBuckets ? kk : (u32)kMaxBuckets) : 2 * kk;
        ls->cta_cleanup = nsm > 16 ? 1u : 0u;
        ls->cur_pos = pos + m;
        ls->subproblems += m;
        ls->elements_distributed += elems;
        ls->chunks += 1;
    }
    // the order in which the classification takes the chunk's stripes:
    // longest first, so that the dynamic stripe scheduler approximates
    // largest-first scheduling and ends the level with short stripes (the
    // subproblems themselves stay largest first: the block permutation hands
    // out its movers in their order)
    if (ws.stripe_order) {
        s_ns[tid] = (u32)tid < m ? ns_i : 0u;
        s_sb[tid] = sbeg;
        s_key[tid] = (u32)tid < m ? slen_i : 0;
        s_beg[tid] = (u64)tid;
        __syncthreads();
        for (u32 k = 2; k <= P; k <<= 1) {
            for (u32 jj = k >> 1; jj > 0; jj >>= 1) {
                const u32 i = (u32)tid, ixj = i ^ jj;
                if (i < P && ixj > i) {
                    const bool desc = (i & k) == 0;
                    const u64 a = s_key[i], b = s_key[ixj];
                    if (desc ? a < b : a > b) {
                        s_key[i] = b;
                        s_key[ixj] = a;
                        const u64 t = s_beg[i];
                        s_beg[i] = s_beg[ixj];
                        s_beg[ixj] = t;
                    }
                }
                __syncthreads();
            }
        }
        const u32 j = (u32)s_beg[tid];
        const u32 nsj = (u32)tid < m ? s_ns[j] : 0u;
        u32 tot;
        const u32 o = block_exclusive_scan<u32>(nsj, s_tmp32, &tot);
        for (u32 q2 = 0; q2 < nsj; ++q2) ws.stripe_order[o + q2] = s_sb[j] + q2;
    }
}

// After the last round: fold its counters, and hand the subproblems still
// queued (a deeper recursion than the rounds covered) to the segment
// scheduler's queue.  One CTA.
template <class T>
__global__ void __launch_bounds__(1024) k_rounds_done(Workspace<T> ws) {
    LoopState* ls = ws.ls;
    __shared__ u32 s_rem, s_next, s_ok;
    if (threadIdx.x == 0) {
        fold_counters(ls, ws.ctr);
        s_ok = ls->status == 0;
        s_rem = ls->cur_count > ls->cur_pos ? ls->cur_count - ls->cur_pos : 0;
        s_next = ls->next_count;
    }
    __syncthreads();
    const u32 rem = s_ok ? s_rem : 0, nxt = s_ok ? s_next : 0;
    const u64 cap = ws.init_cap;
    for (u32 i = threadIdx.x; i < rem + nxt; i += blockDim.x) {
        const Task t = i < rem ? ls->cur_q[ls->cur_pos + i] : ls->next_q[i - rem];
        if (i < cap) ws.init_tasks[i] = t;
        // a result written elsewhere: the scheduler sorts these in place, the copy moves them
        if (ws.out) emit_copy<T>(ws, t.begin, t.n);
    }
    if (threadIdx.x == 0) {
        const u32 total = (u64)(rem + nxt) <= cap ? rem + nxt : (u32)cap;
        if ((u64)(rem + nxt) > cap) ls->status |= kStatusCapacity;
        ws.init_count[0] = total;
        ws.init_count[1] = 0;
        ls->fallback_tasks = total;
        ls->nsub = 0;
    }
}

// After the segment scheduler: fold its counters.  One thread.
template <class T>
__global__ void k_fold(Workspace<T> ws) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ws.ls->subproblems += ws.ctr->next_count;        // the scheduler's distribution steps
        fold_counters(ws.ls, ws.ctr);
    }
}

// The loop state of an enqueue-only segmented sort: no subproblem yet.
template <class T>
__global__ void k_seg_rounds_init(Workspace<T> ws) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *ws.ls = LoopState{};
        ws.ls->cur_q = ws.next_tasks;
        ws.ls->next_q = ws.next_tasks2;
        *ws.ctr = ChunkCounters{};
        ws.init_count[0] = 0;
    }
    for (int g = threadIdx.x; g < 65; g += blockDim.x) ws.hist[g] = 0;
}

// Size groups (2^(g-1) <= n < 2^g) of the segments above the base case, so
// that the first level's queue can hold them largest group first: chunks of
// the level then take subproblems of similar size, as the host driver's
// sorted levels do.
template <class T>
__global__ void k_seg_big_hist(const u64* off, u64 num, Workspace<T> ws, u32 rec_cap) {
    __shared__ u32 h[65];
    for (int i = threadIdx.x; i < 65; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < num; i += (u64)gridDim.x * blockDim.x) {
        const u64 n = off[i + 1] >= off[i] ? off[i + 1] - off[i] : 0;
        if (n > (u64)rec_cap) atomicAdd(&h[64 - __clzll((long long)n)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 65; i += blockDim.x)
        if (h[i]) atomicAdd(&ws.hist[i], h[i]);
}

// The segments [off[i], off[i + 1]) of an enqueue-only segmented sort: those
// no larger than the base case go to init_tasks (sorted by the base case
// straight away), the larger ones form the first level's queue, largest
// size group first.  Offsets that decrease are an error of the call.
template <class T>
__global__ void k_seg_split(const u64* off, u64 num, Workspace<T> ws, u32 rec_cap) {
    LoopState* ls = ws.ls;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < num; i += (u64)gridDim.x * blockDim.x) {
        const u64 b = off[i], e = off[i + 1];
        if (e < b) {
            atomicOr(&ls->status, kStatusInternal);
            continue;
        }
        const u64 n = e - b;
        if (n < 2) continue;
        if (n <= (u64)rec_cap) {
            const u32 idx = atomicAdd(&ws.init_count[0], 1u);
            if (idx < ws.init_cap) ws.init_tasks[idx] = Task{b, n};
            else atomicOr(&ls->status, kStatusCapacity);
        } else {
            // the place in its size group (k_seg_scan turned the group counts into starts)
            const u32 idx = atomicAdd(&ws.hist[64 - __clzll((long long)n)], 1u);
            if (idx < ws.next_cap) ls->cur_q[idx] = Task{b, n};
            else atomicOr(&ls->status, kStatusCapacity);
        }
    }
}

// A sort that is one base case: the single task and the loop state.
template <class T>
__global__ void k_plan_base(Workspace<T> ws, u64 n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *ws.ls = LoopState{};
        *ws.ctr = ChunkCounters{};
        const Task t{0, n};
        if (n <= (u64)T::kBaseTiny) {
            ws.base_tiny[0] = t;
            ws.ctr->base_tiny = 1;
        } else if (n <= (u64)T::kBaseSmall) {
            ws.base_small[0] = t;
            ws.ctr->base_small = 1;
        } else {
            ws.base_large[0] = t;
            ws.ctr->base_large = 1;
        }
    }
}

}  // namespace ips4o
