/*
 * ips4o.h — C ABI of the GB300 in-place samplesort library (libips4o_gb300.so).
 *
 * The library sorts an array that lives in GPU memory, in place, by the
 * method of "In-place Parallel Super Scalar Samplesort" (Axtmann, Witt,
 * Ferizovic, Sanders, 2017): recursive distribution steps of sampling,
 * local classification into blocks, block permutation and cleanup
 * (Section 4), with equality buckets for repeated keys (Section 4.4), down
 * to a base case sorted in on-chip shared memory (Section 4.7).
 *
 * Problem statement (Section 1): rearrange A[0..n) so that the keys are
 * non-decreasing under a total order.  The result's key sequence is unique;
 * elements with equal keys (and different payloads) may come out in any
 * order, since the method is not stable.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers (cudaMalloc, torch CUDA tensors);
 *     h_* are host pointers.  The caller owns all of them; the library never
 *     frees or keeps them after the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it.
 *   - The library owns one workspace per (device, stream) pair (see
 *     ips4o_workspace_bytes), allocated on first use with cudaMalloc and
 *     reused; its size is O(k*b*t + number of subproblems) as in Theorem 2,
 *     plus a small host staging area.
 *   - Calls on the same (device, stream) are serialised by the library;
 *     calls on different streams, made from different host threads, run
 *     side by side on the device, each with its own workspace.  ips4o_sort
 *     and ips4o_sort_segmented_async only enqueue work (capturable in a CUDA
 *     graph with a reserved workspace); the other sort calls plan each
 *     recursion level on the host and synchronise the stream per level.
 *   - Return codes: argument errors are detected before any work is queued;
 *     device-side errors (an exhausted bounded wait, a broken internal
 *     invariant) are recorded in a device status word, which the
 *     synchronising calls read at each level and ips4o_stream_status reads
 *     for the enqueue-only ones.
 */
#ifndef IPS4O_GB300_H
#define IPS4O_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types (Section 5 lists 64-bit floating point elements, Pair,
 * Quartet and 100Bytes records; this library also sorts plain uint64). */
typedef enum {
    IPS4O_U64 = 0,         /* 8-byte unsigned integer, natural order; 8-byte aligned */
    IPS4O_F64 = 1,         /* 8-byte IEEE double, ordered by '<'; the bit pattern b is
                              ordered as (b has sign) ? ~b : b | 2^63, a total order that
                              equals '<' on non-NaN values and puts -0.0 before +0.0 */
    IPS4O_PAIR_U64 = 2,    /* 16-byte {uint64 key; uint64 payload}, ordered by key; 16-byte aligned */
    IPS4O_REC100_K10 = 3,  /* 100-byte record, key = bytes [0,10) compared as unsigned bytes
                              (lexicographic), payload = bytes [10,100); 4-byte aligned.
                              Sorted through 16-byte (key prefix, index) pairs and one gather
                              of the records: NOT in place, it needs 132 bytes of extra device
                              memory per record (see ips4o_workspace_bytes); records with equal
                              keys keep their input order.  ips4o_sort and ips4o_sort_host
                              only; the other entry points return IPS4O_ERR_UNSUPPORTED_TYPE. */
    IPS4O_QUARTET_U64 = 4  /* 32-byte quartet {uint64 k0, k1, k2; uint64 payload} (Section 5's
                              Quartet: three key words and one word of associated information),
                              ordered by (k0, k1, k2) lexicographically; 16-byte aligned; sorted
                              in place.  ips4o_partition reports the splitters' k0 words.  Not
                              supported by ips4o_sort_noalloc. */
} ips4o_key_type;

typedef enum {
    IPS4O_OK = 0,
    IPS4O_ERR_INVALID_ARG = 1,      /* null pointer with n > 0, bad sizes or parameters */
    IPS4O_ERR_UNSUPPORTED_TYPE = 2, /* key type not one of ips4o_key_type */
    IPS4O_ERR_MISALIGNED = 3,       /* pointer not aligned as the key type requires */
    IPS4O_ERR_OOM = 4,              /* workspace could not be allocated */
    IPS4O_ERR_CUDA = 5,             /* a CUDA runtime call failed (see ips4o_last_cuda_error) */
    IPS4O_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up */
    IPS4O_ERR_INTERNAL = 7,         /* a device-side invariant check failed */
    IPS4O_ERR_TOO_LARGE = 8         /* request exceeds a fixed capacity of the entry point
                                       (ips4o_sort: more than 16 GiB of elements per call) */
} ips4o_status;

/* Tuning parameters (Section 4.7 gives k <= 256, alpha = 0.2 log n,
 * beta = 1, n0 = 16 and b = 2 KiB for its CPUs; the GPU defaults differ:
 * 512-byte blocks so that the k buffer blocks of a classification CTA fit its
 * shared memory, alpha = 16 because the shared-memory base case has a hard
 * capacity, and a base case of up to 16 Ki elements instead of 16). */
typedef struct {
    int k_max;            /* maximum buckets per distribution step, power of two in [4, 256]; default 256 */
    int alpha;            /* oversampling factor; <= 0 selects the default (max(8, 0.2 log2 n) ... see source) */
    int base_case_max;    /* buckets of at most this many elements are sorted in shared memory
                             (clamped to [16, ips4o_base_case_capacity]); smaller values force
                             deeper recursion; <= 0 selects the capacity */
    int stripes_per_sm;   /* fewest stripes (local-classification work items) per SM tried for a level; default 1 */
    int profile;          /* 1: time every kernel with CUDA events into ips4o_stats.phase_ms */
    uint64_t seed;        /* sampling seed */
    int segment_scheduler;  /* ips4o_sort_segmented / ips4o_sort_batched: 0 automatic (currently
                               level by level, the faster of the two), 1 level by level across
                               all segments, 2 the segment scheduler (one CTA per array, as in
                               ips4o_sort_segmented_async) */
    uint32_t spin_limit;    /* polls of every bounded device wait before it gives up and the call
                               returns IPS4O_ERR_TIMEOUT; 0 selects the default (2^22, about 0.3 s) */
    int record_path;        /* 100-byte records: 0 key + index indirection (default; records with
                               equal keys keep their input order; 132 bytes of extra device memory
                               per record), 1 the records moved in place through the distribution
                               steps in blocks of 5 (not stable; workspace independent of the
                               record size but for the blocks) */
    uint64_t strict_window; /* ips4o_sort_strict: elements scanned per pass of its bucket-head scan
                               (rounded down to a multiple of 2048, at least 2048); 0 selects about
                               1 GiB of elements */
} ips4o_params;

/* Parameters of the distribution steps per size class, as an autotuner picks
 * them (the paper fixes k = 256 and alpha = 0.2 log n for its CPUs, Section
 * 4.7; on the GPU the best choice depends on the subproblem size).  Entry c
 * applies to subproblems of n elements with 2^c <= n < 2^(c+1):
 *   leaves  number of leaves of the step (power of two in [4, 256]; 0 = the
 *           library's rule: about 2n / base-case size, at most k_max);
 *   alpha   oversampling factor (alpha * leaves <= 4096; 0 = the default).
 * The table is process-wide and applies to ips4o_sort, the segmented and
 * batched calls (both forms) and ips4o_sort_segmented_async, not to
 * ips4o_partition or ips4o_sort_noalloc. */
#define IPS4O_NUM_CLASSES 64
typedef struct {
    uint16_t leaves;
    uint16_t alpha;
} ips4o_class_params;

/* Set entries [0, count) of the table (count <= IPS4O_NUM_CLASSES; the rest
 * are reset to 0); NULL resets the whole table.  The device copy used by the
 * segment scheduler is updated on the current device (call it once per
 * device, not while a stream is being captured).  INVALID_ARG if an entry
 * breaks the rules above (nothing is changed then). */
ips4o_status ips4o_set_class_params(const ips4o_class_params* table, size_t count);
ips4o_status ips4o_get_class_params(ips4o_class_params* out, size_t count);

/* Counters of the last completed call on the calling thread's current device. */
#define IPS4O_NUM_PHASES 8
typedef struct {
    uint64_t n;                    /* elements sorted by the last call */
    uint32_t levels;               /* distribution levels executed (deepest level reached) */
    uint32_t chunks;               /* level chunks launched (groups of subproblems) */
    uint64_t subproblems;          /* distribution steps performed */
    uint64_t kernel_launches;      /* kernels this library launched for the call */
    uint64_t blocks_moved;         /* block writes of the block permutation (Section 4.2) */
    uint64_t blocks_skipped;       /* blocks found already in their bucket and left in place */
    uint64_t fix_blocks_moved;     /* blocks moved by the empty-block movement (Appendix A) */
    uint64_t base_case_buckets;    /* buckets sorted by the shared-memory base case */
    uint64_t elements_distributed; /* sum over levels of the elements classified */
    uint64_t workspace_bytes;      /* device workspace held by the library on this device */
    double phase_ms[IPS4O_NUM_PHASES]; /* with params.profile: summed kernel time per phase:
                                      0 sample, 1 classify, 2 prefix, 3 empty-block fix,
                                      4 block permutation (and the segment scheduler),
                                      5 cleanup, 6 base case, 7 other */
    uint64_t phase_launches[IPS4O_NUM_PHASES];
} ips4o_stats;

/* Sort d_ptr[0..n) in place (Section 4: recursive distribution steps down
 * to the base case).  n in {0, 1} is a no-op.
 * Asynchronous: the call only enqueues kernels on `stream` and returns; the
 * recursion levels are planned on the device (each round takes the next
 * chunk of a level's subproblems from a queue in device memory), so the host
 * never waits.  Work on the stream after the call sees the sorted array.
 *   - Argument errors are returned at once, before anything is queued.
 *   - Device-side errors (a bounded wait that gave up, a failed invariant
 *     check) are returned by ips4o_stream_status(stream), which waits for
 *     the stream; after such an error d_ptr holds the same elements,
 *     permuted but not sorted.  ips4o_get_stats also waits for the call.
 *   - The workspace of (current device, stream) grows on the first call of a
 *     size (cudaMalloc).  Reserved beforehand with ips4o_reserve_workspace(n,
 *     1, key_type, stream), a call allocates nothing and can be captured into
 *     a CUDA graph; under capture without a large enough reservation it
 *     returns IPS4O_ERR_TOO_LARGE and queues nothing.
 *   - Extra device memory (Theorem 2): a leftover pool for 2 stripes per SM
 *     (independent of n) plus per-chunk tables, two level queues of
 *     n / (base-case size) entries, and the segment scheduler's per-CTA
 *     areas; see ips4o_workspace_bytes.  ips4o_sort_strict needs no queue. */
ips4o_status ips4o_sort(void* d_ptr, size_t n, int key_type, void* stream);

/* Sort d_ptr[0..n) in place with extra memory independent of n: the strictly
 * in-place recursion of Section 4.6.  Each distribution step moves the
 * largest element of every bucket that must be distributed again to the
 * bucket's first slot; the end of such a bucket is then the first later
 * position holding a larger key, so the remaining work is found by scanning
 * the array (a window of params.strict_window elements at a time) instead of
 * being kept in queues.  Every key type, including 100-byte records (moved in
 * place in blocks of 5, not through key + index pairs).  The result equals
 * ips4o_sort's.
 *   - Synchronous: the host waits on `stream` once per round of subproblems
 *     and once per scanned window, and the call returns when the array is
 *     sorted; device-side errors are returned by the call itself.  Refused
 *     (IPS4O_ERR_INVALID_ARG) while the stream is being captured.
 *   - Extra device memory: ips4o_workspace_bytes_strict(n, key_type), the
 *     same for every n above the base case. */
ips4o_status ips4o_sort_strict(void* d_ptr, size_t n, int key_type, void* stream);

/* Device workspace in bytes that ips4o_sort_strict uses for n elements of
 * key_type with the current parameters (host computation, no device work). */
size_t ips4o_workspace_bytes_strict(size_t n, int key_type);

/* Same as ips4o_sort but for an array in HOST memory: the elements are
 * brought to a device staging buffer (owned by the library and kept for
 * reuse), sorted there, and copied back (all on `stream`); the call returns
 * when h_ptr holds the result.  For pinned host memory the GPU reads and
 * writes the buffer through its device address: for u64, f64 and pair keys
 * the first distribution step samples and classifies the host buffer itself
 * and writes its blocks into the staging buffer (no separate copy to the
 * device), and a kernel copies the result back; inputs no larger than the
 * base case and 100-byte records are copied by a kernel first.  Pageable
 * memory is copied by cudaMemcpyAsync. */
ips4o_status ips4o_sort_host(void* h_ptr, size_t n, int key_type, void* stream);

/* One distribution step (Section 4: sampling, local classification, block
 * permutation, cleanup) on d_ptr[0..n), n > base case, leaving the array
 * partitioned into buckets, followed by nothing else.  Outputs (host):
 *   h_bounds[0..*num_buckets]  bucket boundaries (h_bounds[0] = 0, last = n),
 *                              capacity 257 entries;
 *   h_splitters[0..*num_splitters) the splitter keys of the step in the
 *                              library's comparable form (u64: the value;
 *                              f64: the mapped bits; pair: the key), capacity 256;
 *   *eq                        1 if equality buckets were used (Section 4.4):
 *                              bucket 2i+1 then holds the keys equal to
 *                              splitter i, bucket 2i those strictly between
 *                              splitters i-1 and i.
 * Splitters are padded to a power-of-two tree by repeating the largest one,
 * so some buckets are empty. */
ips4o_status ips4o_partition(void* d_ptr, size_t n, int key_type, void* stream,
                             uint64_t* h_bounds, size_t* num_buckets,
                             uint64_t* h_splitters, size_t* num_splitters, int* eq);

/* Sort many independent segments of one device array, each in place and
 * each as ips4o_sort would sort it alone (the paper has no batched form; its
 * recursion already processes the buckets of a level side by side, Section
 * 4, and this entry point starts that processing from the caller's
 * segments).  Segment i is d_base[offsets[i] .. offsets[i+1]), i <
 * num_segments; offsets holds num_segments + 1 non-decreasing element
 * indices, in host or device memory (it is read once at the start of the
 * call).  Elements outside the segments are not touched.  Segments no
 * larger than the base case (ips4o_base_case_capacity) are sorted in shared
 * memory by one launch; the others go through the distribution levels
 * together, one set of kernel launches per level for all of them.
 * Errors: decreasing offsets or a null d_base with elements -> INVALID_ARG;
 * a segment above the ips4o_sort size limit -> TOO_LARGE (nothing queued).
 * Synchronises the stream; on return the segments are sorted. */
ips4o_status ips4o_sort_segmented(void* d_base, const uint64_t* offsets, size_t num_segments, int key_type,
                                  void* stream);

/* ips4o_sort_segmented without any host work after the call returns:
 * d_offsets (num_segments + 1 element indices) must be in DEVICE memory, the
 * call only enqueues kernels on `stream` (it neither allocates, nor copies
 * to or from the host, nor synchronises), so it can be captured into a CUDA
 * graph and replayed.  The levels are planned on the device as for
 * ips4o_sort: the segments no larger than the base case are sorted by the
 * base case at once, the larger ones form the first level's queue, and each
 * level distributes all its subproblems side by side (Section 4); what is
 * left after the enqueued rounds is sorted by the segment scheduler (one CTA
 * per array).  With params.segment_scheduler = 2 every segment goes to the
 * segment scheduler instead.
 *   - The workspace of (current device, stream) must have been reserved
 *     with ips4o_reserve_workspace(n, num_segments, key_type, stream), n at
 *     least the total number of elements of the segments (the level queues
 *     are sized from it; a larger total makes ips4o_stream_status report
 *     IPS4O_ERR_INTERNAL); without a reservation IPS4O_ERR_TOO_LARGE is
 *     returned and nothing is enqueued.
 *   - Device-side errors (decreasing offsets, a bounded wait that gave up,
 *     a broken invariant) are recorded in the stream's status word:
 *     ips4o_stream_status(stream) waits for the stream and returns them.
 *   - ips4o_get_stats (which waits for the stream) reports the call's
 *     counters, with n = 0 (the total is known on the device only).
 *     u64, f64, pair and quartet keys. */
ips4o_status ips4o_sort_segmented_async(void* d_base, const uint64_t* d_offsets, size_t num_segments,
                                        int key_type, void* stream);

/* Sort `count` separate device arrays, ptrs[i][0 .. lens[i]), each in place,
 * in one call (the same processing as ips4o_sort_segmented).  ptrs and lens
 * are arrays of `count` entries in host or device memory; every ptrs[i] with
 * lens[i] > 0 must be aligned for the key type, and the arrays must not
 * overlap (INVALID_ARG otherwise, before any work).  Arrays of length 0 are
 * skipped. */
ips4o_status ips4o_sort_batched(void* const* ptrs, const uint64_t* lens, size_t count, int key_type,
                                void* stream);

/* Waits for all work on `stream` and reports a CUDA error that it raised
 * (IPS4O_ERR_CUDA, text in ips4o_last_cuda_error), then the device status
 * word of the last ips4o_sort or ips4o_sort_segmented_async call on the
 * stream (IPS4O_ERR_TIMEOUT, IPS4O_ERR_INTERNAL), else IPS4O_OK.  The other
 * sort calls return device-side errors themselves. */
ips4o_status ips4o_stream_status(void* stream);

/* Sort d_ptr[0..n) in place, like ips4o_sort, without allocating any memory.
 * The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory when they sort, such as a service whose device
 * footprint is fixed at start-up (a later allocation could fail or push out
 * other tenants) or a plug-in whose host process owns every allocation.
 * Instead of the workspace it uses a scratch area built into the library: a
 * 16 MiB __device__ array, which every GPU that loads the library holds until
 * the process exits, plus a static host staging buffer.  It calls no
 * cudaMalloc, cudaMallocHost, cudaFree or other allocating routine.
 *   - n is limited to 2^20 elements; larger n returns IPS4O_ERR_TOO_LARGE
 *     before any work is queued.  The library's default parameters are used
 *     (ips4o_set_params does not apply), and ips4o_get_stats does not report
 *     these calls.
 *   - The call synchronises `stream` once per recursion level, so it cannot
 *     be made while the stream is being captured into a CUDA graph: it then
 *     returns IPS4O_ERR_INVALID_ARG before queuing anything (the capture
 *     stays valid).  Work that must be captured can use
 *     ips4o_sort_segmented_async with a reserved workspace.
 *   - The first call on a device looks up the device address of the scratch
 *     array (cudaGetSymbolAddress) with that device current.
 *   - All calls share the scratch array and keep the last call's contents
 *     (counters that must start at zero are cleared by every call); calls are
 *     serialised by the library and each waits for its own work, since calls
 *     that overlapped on the GPU would race on the scratch.
 *   - Same argument checks and return codes as ips4o_sort.  As there, an
 *     error reported after the first level has run (a bounded wait that gave
 *     up, a failed invariant check) leaves d_ptr holding the same elements,
 *     permuted but not sorted. */
ips4o_status ips4o_sort_noalloc(void* d_ptr, size_t n, int key_type, void* stream);

/* Device workspace the library needs for a sort of n elements of the type. */
size_t ips4o_workspace_bytes(size_t n, int key_type);

/* Make the workspace and host staging of (current device, stream) large
 * enough for a call on n elements in num_segments segments (1 for
 * ips4o_sort), so that such calls allocate nothing.  A service reserves its
 * workers' workspaces up front this way: allocation while other streams run
 * costs time, and freeing a smaller workspace synchronises the device.
 * Workspaces only grow; ips4o_release_workspace frees them.  The largest n
 * reserved on (device, stream) for the key type is remembered: the
 * enqueue-only ips4o_sort_segmented_async sizes its level queues from it, so
 * n must be at least the total number of elements of its segments. */
ips4o_status ips4o_reserve_workspace(size_t n, size_t num_segments, int key_type, void* stream);

/* Free the workspaces and staging buffers held on the current device (all streams). */
ips4o_status ips4o_release_workspace(void);

/* Parameters (process-wide).  ips4o_set_params(NULL) restores defaults. */
ips4o_status ips4o_set_params(const ips4o_params* p);
ips4o_status ips4o_get_params(ips4o_params* out);

/* Counters of the last call made by this process on the current device (any stream). */
ips4o_status ips4o_get_stats(ips4o_stats* out);

/* Capacity of the shared-memory base case for a key type, in elements. */
size_t ips4o_base_case_capacity(int key_type);

const char* ips4o_status_string(int status);

/* Self-check of the failure path (no counterpart in the paper): runs, on
 * `stream`, one device wait of the kind the sort uses (a bounded poll of a
 * flag) on a flag that nothing sets, with the given poll limit.  Returns
 * IPS4O_ERR_TIMEOUT when the wait gave up and reported it as the sort
 * kernels do; the context stays usable.  Any other result means the check
 * failed.  Uses a few bytes of device memory built into the library. */
ips4o_status ips4o_check_bounded_wait(uint32_t spin_limit, void* stream);

/* Text of the last CUDA error seen by the library (empty if none). */
const char* ips4o_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IPS4O_GB300_H */
