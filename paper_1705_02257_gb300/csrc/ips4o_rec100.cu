// ips4o_rec100.cu — 100-byte records (Section 5 "100Bytes": a 10-byte key
// compared as unsigned bytes, then 90 bytes of payload), two ways.
//
// Key + index indirection (the default).  Moving 100-byte elements through
// the distribution levels costs 100 bytes per element per pass; the paper
// notes that for such large elements its in-place method moves every element
// twice per level (Section 6, comparison with s^3-sort).  Here the records
// are instead represented by 16-byte pairs
//     key     = bytes 0..7 of the record as a big-endian integer,
//     payload = bytes 8..9 as a big-endian 16-bit integer << 48 | record index,
// which are sorted by the pair path; runs of equal 8-byte prefixes are then
// sorted again by payload (bytes 8..9, then index), and finally every record
// is gathered once from a copy of the input to its place.  The result is the
// records in key order, records with equal keys in their input order.
// Extra device memory: 16 bytes (pairs) + 100 bytes (input copy) + 16 bytes
// (run bounds) per record, besides the pair sort's own workspace; not in
// place.
//
// In-place blocks (params.record_path = 1).  The records themselves go
// through the distribution steps of the other types, in blocks of 5 records
// (500 bytes, copied in 4-byte words) with keys (bytes 0..7, bytes 8..9)
// compared by the tree descent, down to a shared-memory base case of up to
// 1024 records; the levels are planned on the host.  In place (workspace
// O(k b t + #subproblems)); not stable.
#include "ips4o_driver.cuh"

#include <algorithm>
#include <vector>

#include "ips4o_common.cuh"
#include "ips4o_host.h"

namespace ips4o {

constexpr int kRecBytes = 100;
constexpr int kRecWords = kRecBytes / 4;

// pairs[i] = {big-endian bytes 0..7, big-endian bytes 8..9 << 48 | i}
__global__ void k_rec_extract(const u32* __restrict__ rec, u64 n, PairElem* __restrict__ pairs) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        const u32* r = rec + i * kRecWords;
        const u32 w0 = r[0], w1 = r[1], w2 = r[2];
        const u64 hi = ((u64)bswap32(w0) << 32) | bswap32(w1);
        const u64 lo16 = ((w2 & 0xffu) << 8) | ((w2 >> 8) & 0xffu);
        pairs[i] = PairElem{hi, (lo16 << 48) | i};
    }
}

// Bounds of the runs of at least two equal keys: begins (first index) and
// ends (one past the last), in no particular order.
__global__ void k_rec_runs(const PairElem* __restrict__ p, u64 n, u64* begins, u64* ends, u32* counts, u64 cap) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        const u64 k = p[i].k;
        const bool same_prev = i > 0 && p[i - 1].k == k;
        const bool same_next = i + 1 < n && p[i + 1].k == k;
        if (same_next && !same_prev) {
            const u32 q = atomicAdd(&counts[0], 1u);
            if (q < cap) begins[q] = i;
        }
        if (same_prev && !same_next) {
            const u32 q = atomicAdd(&counts[1], 1u);
            if (q < cap) ends[q] = i + 1;
        }
    }
}

__global__ void k_rec_swap(PairElem* p, u64 n) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        const PairElem e = p[i];
        p[i] = PairElem{e.p, e.k};
    }
}

// out[i] = in[index of pair i]: one warp per record, 25 lanes of 4 bytes.
__global__ void k_rec_gather(u32* __restrict__ out, const u32* __restrict__ in, const PairElem* __restrict__ p,
                             u64 n) {
    const int lane = threadIdx.x & 31;
    const u64 warps = (u64)gridDim.x * (blockDim.x / 32);
    for (u64 i = ((u64)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < n; i += warps) {
        const u64 src = p[i].p & ((1ull << 48) - 1);
        if (lane < kRecWords) out[i * kRecWords + lane] = in[src * kRecWords + lane];
    }
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// pairs [16 n] | input copy [100 n] | run begins, run ends [n / 2 + 1 each] | counts
size_t rec100_aux_bytes(size_t n) { return align256(n * (16 + kRecBytes)) + 2 * (n / 2 + 1) * 8 + 256; }

// The block path: the records sorted in place by the distribution steps.
// The records moved in place by the strictly in-place recursion (Section 4.6).
ips4o_status sort_strict_rec100(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    return strict_sort_t<TRec>(st, d, n, s);
}
size_t strict_workspace_bytes_rec100(size_t n, int sms) { return strict_workspace_bytes_t<TRec>(n, sms); }

static ips4o_status sort_rec100_blocks(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    Driver<TRec> drv(st, s);
    return drv.run((RecElem*)d, (u64)n, nullptr);
}

ips4o_status sort_rec100(DeviceState& st, void* d, size_t n, cudaStream_t s) {
    if (global_params().record_path == 1) return sort_rec100_blocks(st, d, n, s);
    ips4o_status rc = ensure_device_buffer(&st.d_aux, &st.aux_bytes, rec100_aux_bytes(n));
    if (rc != IPS4O_OK) return rc;
    char* aux = (char*)st.d_aux;
    PairElem* pairs = (PairElem*)aux;
    u32* tmp = (u32*)(aux + n * 16);
    u64* begins = (u64*)(aux + align256(n * (16 + kRecBytes)));
    u64* ends = begins + n / 2 + 1;
    u32* counts = (u32*)(ends + n / 2 + 1);
    const u64 cap = n / 2 + 1;
    const int grid = st.sms * 8;
    auto cuda = [](cudaError_t e, const char* what) -> ips4o_status {
        if (e == cudaSuccess) return IPS4O_OK;
        set_last_cuda_error(e, what);
        return IPS4O_ERR_CUDA;
    };
    u64 launches = 1;
    k_rec_extract<<<grid, 256, 0, s>>>((const u32*)d, n, pairs);
    if ((rc = cuda(cudaGetLastError(), "launch of k_rec_extract")) != IPS4O_OK) return rc;
    rc = sort_pair(st, pairs, n, s, nullptr);
    if (rc == IPS4O_OK) rc = finalize_pending(st);     // the pair sort is enqueued: wait for it, read its status
    if (rc != IPS4O_OK) return rc;
    const ips4o_stats main_sort = st.stats;
    launches += main_sort.kernel_launches;
    // runs of equal 8-byte prefixes: order them by bytes 8..9 (then index)
    if ((rc = cuda(cudaMemsetAsync(counts, 0, 8, s), "cudaMemsetAsync")) != IPS4O_OK) return rc;
    k_rec_runs<<<grid, 256, 0, s>>>(pairs, n, begins, ends, counts, cap);
    ++launches;
    if ((rc = cuda(cudaGetLastError(), "launch of k_rec_runs")) != IPS4O_OK) return rc;
    u32 h_counts[2];
    if ((rc = cuda(cudaMemcpyAsync(h_counts, counts, 8, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync")) != IPS4O_OK)
        return rc;
    if ((rc = cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize")) != IPS4O_OK) return rc;
    if (h_counts[0] != h_counts[1] || h_counts[0] > cap) {
        set_last_message("100-byte records: inconsistent runs of equal keys");
        return IPS4O_ERR_INTERNAL;
    }
    if (h_counts[0] > 0) {
        const size_t m = h_counts[0];
        std::vector<u64> hb(m), he(m);
        if ((rc = cuda(cudaMemcpyAsync(hb.data(), begins, m * 8, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync")) !=
            IPS4O_OK)
            return rc;
        if ((rc = cuda(cudaMemcpyAsync(he.data(), ends, m * 8, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync")) !=
            IPS4O_OK)
            return rc;
        if ((rc = cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize")) != IPS4O_OK) return rc;
        std::sort(hb.begin(), hb.end());
        std::sort(he.begin(), he.end());
        std::vector<Task> runs(m);
        for (size_t q = 0; q < m; ++q) {
            if (he[q] <= hb[q]) {
                set_last_message("100-byte records: inconsistent runs of equal keys");
                return IPS4O_ERR_INTERNAL;
            }
            runs[q] = Task{hb[q], he[q] - hb[q]};
        }
        k_rec_swap<<<grid, 256, 0, s>>>(pairs, n);
        if ((rc = cuda(cudaGetLastError(), "launch of k_rec_swap")) != IPS4O_OK) return rc;
        rc = sort_segments_pair(st, pairs, runs, s);
        if (rc != IPS4O_OK) return rc;
        launches += st.stats.kernel_launches + 2;
        k_rec_swap<<<grid, 256, 0, s>>>(pairs, n);
        if ((rc = cuda(cudaGetLastError(), "launch of k_rec_swap")) != IPS4O_OK) return rc;
    }
    // one gather of the records from a copy of the input
    if ((rc = cuda(cudaMemcpyAsync(tmp, d, n * kRecBytes, cudaMemcpyDeviceToDevice, s), "cudaMemcpyAsync(records)")) !=
        IPS4O_OK)
        return rc;
    k_rec_gather<<<st.sms * 16, 256, 0, s>>>((u32*)d, tmp, pairs, n);
    ++launches;
    if ((rc = cuda(cudaGetLastError(), "launch of k_rec_gather")) != IPS4O_OK) return rc;
    if ((rc = cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize")) != IPS4O_OK) return rc;
    st.stats = main_sort;
    st.stats.kernel_launches = launches;
    st.stats.workspace_bytes = st.ws_bytes + st.aux_bytes;
    return IPS4O_OK;
}

}  // namespace ips4o
