// ips4o_noalloc_driver.cuh — the level loop of ips4o_sort_noalloc over
// fixed task arrays (no std::vector, no allocation).  Included only by the
// per-type translation units, so that every instantiation of a type's
// kernels and driver lives in one translation unit (kernel attributes set by
// the driver then always apply to the kernels it launches).
#pragma once

#include "ips4o_driver.cuh"

namespace ips4o {

// The library defaults (ips4o_set_params(NULL)): the scratch is sized for
// them, so user parameters (e.g. a smaller base case, which creates more
// subproblems) do not apply.
static const ips4o_params kNoAllocParams = kDefaultParams;

// Every next-level subproblem is larger than the recursion threshold, so a
// level of an array of at most kNoAllocMaxN elements has fewer than
// kNoAllocMaxN / (threshold + 1) of them; with the default parameters the
// smallest threshold is the pair base case.
static_assert(kNoAllocMaxN / ((size_t)TPair::kBaseCap + 1) < kNoAllocMaxTasks, "task arrays too small");

template <class T>
struct NoAllocDriver : Driver<T> {
    typedef typename T::elem_t E;
    using Driver<T>::st;
    using Driver<T>::prm;
    using Driver<T>::caps;
    using Driver<T>::h_tasks;
    using Driver<T>::ws;
    using Driver<T>::rec_cap;
    using Driver<T>::stream;

    Task* tasks;   // [2][kNoAllocMaxTasks], owned by the caller

    NoAllocDriver(DeviceState& s, cudaStream_t strm, Task* t) : Driver<T>(s, strm, kNoAllocParams), tasks(t) {}

    ips4o_status run(E* d, u64 n) {
        // the scratch is used as it is: setup never allocates or frees in
        // this mode and answers TOO_LARGE when the workspace or the host
        // staging this sort needs does not fit
        ips4o_status rc = this->setup(n, 0, nullptr, Driver<T>::kFixed);
        if (rc != IPS4O_OK) return rc;
        st.stats.n = n;
        if (n <= (u64)rec_cap) return this->base_only(d, n);
        Task* cur = tasks;
        Task* nxt = tasks + kNoAllocMaxTasks;
        size_t ncur = 1;
        cur[0] = Task{0, n};
        u32 level = 0;
        while (ncur > 0) {
            size_t nnext = 0;
            u64 level_total = 0;
            for (size_t q = 0; q < ncur; ++q) level_total += cur[q].n;
            size_t i = 0;
            while (i < ncur) {
                u32 nsub = 0, nstr = 0;
                const size_t taken = this->plan_chunk(cur, ncur, i, level_total, level, false, &nsub, &nstr);
                if (taken == 0) return IPS4O_ERR_INTERNAL;
                u32 cnt = 0;
                rc = this->run_chunk(d, nsub, nstr, false, &cnt);
                if (rc != IPS4O_OK) return rc;
                if (cnt > 0) {
                    if (cnt > caps.next_cap || nnext + cnt > kNoAllocMaxTasks) return IPS4O_ERR_TOO_LARGE;
                    IPS4O_CUDA(cudaMemcpyAsync(h_tasks, ws.next_tasks, cnt * sizeof(Task), cudaMemcpyDeviceToHost,
                                               stream));
                    IPS4O_CUDA(cudaStreamSynchronize(stream));
                    for (u32 q = 0; q < cnt; ++q) nxt[nnext + q] = h_tasks[q];
                    nnext += cnt;
                }
                i += taken;
            }
            ++level;
            st.stats.levels = level;
            Task* t = cur;
            cur = nxt;
            nxt = t;
            ncur = nnext;
            if (level > 64) return IPS4O_ERR_INTERNAL;
        }
        return IPS4O_OK;
    }
};

template <class T>
ips4o_status noalloc_sort_t(DeviceState& st, void* d, size_t n, cudaStream_t s, Task* tasks) {
    NoAllocDriver<T> drv(st, s, tasks);
    return drv.run((typename T::elem_t*)d, (u64)n);
}

}  // namespace ips4o
