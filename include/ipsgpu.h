/*
 * ipsgpu.h -- C ABI of the GB300 (sm_103a) in-place samplesort library.
 *
 * The library sorts arrays that already live in device memory, in place,
 * following the in-place parallel super scalar samplesort (IPS4o) and its
 * radix variant (IPS2Ra) of Axtmann, Witt, Ferizovic and Sanders,
 * "Engineering In-place (Shared-memory) Sorting Algorithms":
 *   problem statement        Sec. 2 (sort A[0..n-1] in place by '<')
 *   partitioning step        Sec. 3.1 (sampling, classification into
 *                            b-element buffer blocks, block permutation with
 *                            per-bucket read/write pointers, cleanup)
 *   recursion and base case  Sec. 3.2, Sec. 5
 *   radix variant            Sec. 5 (IPS2Ra: radix extractor on unsigned keys)
 *   sorter object            Sec. 6.6 (setup separated from sorting)
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers of the current CUDA device; the
 *     caller owns them.  Data arrays must be aligned to their element size
 *     (4 bytes for rec100, 16 for quartet) and must not be accessed by other
 *     work while a call on them is in flight.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous with respect to the host unless a
 *     function says it synchronizes.  The sorts (ipsgpu_sort,
 *     ipsgpu_sort_segmented, ipsgpu_sort_batch) plan every recursion level
 *     on the device and never synchronize; the single-level calls wait for
 *     their previous call's descriptor upload.
 *   - Return values are status codes (IPSGPU_OK = 0).  Errors detected by
 *     kernels (a bounded wait that ran out, an inconsistent count) are kept
 *     in a device status word of the sorter and reported by ipsgpu_status.
 *   - A sorter may be used by one host thread at a time.
 */
#ifndef IPSGPU_H
#define IPSGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types (Sec. 6 "data types").  Key order:
 *   U32, U64   numeric
 *   F64        IEEE-754 bits b mapped to (b>>63) ? ~b : b|2^63, compared as
 *              unsigned; this is '<' on non-NaN values with -0.0 before +0.0
 *   PAIR_U64   16 bytes {u64 key, u64 value}; key only
 *   REC100     100 bytes; the first 10 bytes compared lexicographically as
 *              unsigned bytes; 90 bytes of payload
 *   QUARTET    32 bytes {u64 a, u64 b, u64 c, u64 value}; key (a, b, c)
 *              compared lexicographically (the Quartet comparison of
 *              Sec. 6); arrays 16-byte aligned                              */
typedef enum {
    IPSGPU_U32 = 0,
    IPSGPU_U64 = 1,
    IPSGPU_F64 = 2,
    IPSGPU_PAIR_U64 = 3,
    IPSGPU_REC100 = 4,
    IPSGPU_QUARTET = 5
} ipsgpu_dtype;

/* Classifier of the partitioning step: the branchless splitter tree of IPS4o
 * (Sec. 2, Algorithm 1) or the radix extractor of IPS2Ra (Sec. 5; U32, U64
 * and PAIR_U64 keys only).  SAMPLESORT starts each element's tree walk from
 * a lookup table of start nodes addressed by the key's leading bits (the
 * table Sec. 8 proposes); SAMPLESORT_TREE walks every element from the root
 * as Algorithm 1 does.  Both give identical classes and results;
 * SAMPLESORT_TREE exists to measure the table. */
typedef enum {
    IPSGPU_SAMPLESORT = 0,
    IPSGPU_RADIX = 1,
    IPSGPU_SAMPLESORT_TREE = 2
} ipsgpu_algo;

enum {
    IPSGPU_OK = 0,
    IPSGPU_E_INVAL = 1,       /* bad argument (NULL, misaligned, too large)   */
    IPSGPU_E_UNSUPPORTED = 2, /* dtype/algorithm combination not supported    */
    IPSGPU_E_NOMEM = 3,       /* device or pinned host allocation failed      */
    IPSGPU_E_CUDA = 4,        /* a CUDA runtime call failed                   */
    IPSGPU_E_TIMEOUT = 5,     /* a bounded device wait gave up                */
    IPSGPU_E_BUSY = 6,        /* server: request cannot be admitted now       */
    IPSGPU_E_INTERNAL = 7,    /* a kernel found an inconsistent count         */
    IPSGPU_E_CANCELED = 8     /* server: the request was cancelled before it ran */
};

/* Tuning parameters; a zero field takes its default.
 *   k                 max buckets per level incl. equality buckets (256,
 *                     Sec. 5; power of two in [4, 256])
 *   block_bytes       bytes per block (512; the paper's 2 KiB shrinks so that
 *                     k buffer blocks fit in one SM's shared memory).  A
 *                     block holds b elements, b the largest power of two
 *                     with b * element size <= block_bytes (at least 1);
 *                     b * element size must be a multiple of 16, at most
 *                     2 KiB, and k * b * element size at most 128 KiB (the
 *                     k buffer blocks of a classification CTA; with them
 *                     its tile stage and tables fill 227 KiB of shared
 *                     memory): k = 256 takes blocks up to 512 B, 128 up to
 *                     1 KiB, 64 up to 2 KiB
 *   alpha_scale       oversampling alpha = alpha_scale * log2(n') (0.2, Sec. 5)
 *   base_case         largest segment sorted by the shared-memory base case
 *                     (elements; at least 32; default and maximum: as many
 *                     as fit in 184 KiB, 23552 for 8-byte elements, 5888
 *                     Quartets, 1884 100-byte records)
 *   seed              seed of the sampling generator (splitmix64)
 *   algo              ipsgpu_algo
 *   spin_limit        iterations of a bounded device wait before it gives up
 *                     with IPSGPU_E_TIMEOUT (default 1<<22, ~0.5 s)
 *   arena_bytes       device scratch for leftover buffer blocks and cleanup
 *                     staging (default 256 MiB; at least
 *                     (2k + 1) * block + 1 KiB, block = b * element size)
 * A parameter outside these ranges makes ipsgpu_sorter_create return
 * IPSGPU_E_INVAL and ipsgpu_scratch_bytes return 0.                       */
typedef struct {
    uint32_t k;
    uint32_t block_bytes;
    float alpha_scale;
    uint32_t base_case;
    uint64_t seed;
    int32_t algo;
    uint32_t spin_limit;
    uint64_t arena_bytes;
} ipsgpu_params;

typedef struct ipsgpu_sorter ipsgpu_sorter;

/* Create a sorter for one element type (the "sorter object" of Sec. 6.6).
 * Allocates every piece of device scratch the sorter will ever use; the
 * amount depends on the parameters only, never on n (see
 * ipsgpu_scratch_bytes).  params may be NULL (all defaults).  The sorter is
 * bound to the CUDA device current at creation.
 * Errors: E_INVAL (bad params, out NULL), E_UNSUPPORTED (RADIX with F64,
 * REC100 or QUARTET), E_NOMEM, E_CUDA. */
int ipsgpu_sorter_create(const ipsgpu_params *params, int dtype, ipsgpu_sorter **out);

/* Build now what a sorter otherwise builds on its first sort: the CUDA graph
 * of the device-planned recursion (a capture on a private stream).  Call it
 * before capturing other work if the first sort would fall inside a capture
 * window.  Errors: E_INVAL, E_CUDA. */
int ipsgpu_sorter_prepare(ipsgpu_sorter *s);

/* Free a sorter and its scratch (synchronizes the device first). */
int ipsgpu_sorter_destroy(ipsgpu_sorter *s);

/* Device scratch bytes a sorter with these parameters allocates, none of it
 * depending on n or on the number of segments: the arena (arena_bytes; per
 * segment of a wave its cleanup staging, per stripe its leftover buffer
 * blocks) plus tables of fixed capacity for one wave (2^16 segments and
 * stripes, 2^20 (segment, class) pairs, 2^21 base-case entries, 2^22 fix-up
 * moves, a ring of 2^20 waiting segments): 227 MiB for U32, 235 MiB for
 * 8- and 16-byte elements, 251 MiB for REC100, 267 MiB for QUARTET.  The
 * sorter allocates under 64 KiB more (fixed-size state, guard zones).
 * 0 if the parameters are invalid for the dtype. */
uint64_t ipsgpu_scratch_bytes(const ipsgpu_params *params, int dtype);

/* Sort d_data[0..n) in place, ascending in the key order of the sorter's
 * dtype (Sec. 2 problem statement; Sec. 3 and 5).  Detects non-decreasing
 * inputs (left as they are) and non-increasing ones (reversed) first
 * (Sec. 5), on the device.  Asynchronous: never synchronizes, and can be
 * captured into a CUDA graph.
 * For U32/U64/F64 the result is the unique sorted sequence; for PAIR_U64,
 * REC100 and QUARTET records with equal keys may appear in any order.
 * Errors: E_INVAL, E_CUDA; kernel-side errors via ipsgpu_status. */
int ipsgpu_sort(ipsgpu_sorter *s, void *d_data, uint64_t n, void *stream);

/* Sort an array that lives in HOST memory: copy h_in[0..n) to the device
 * buffer d_work (n elements, caller-owned, aligned like d_data above), sort
 * it there as ipsgpu_sort does, and copy the result to h_out[0..n) (h_out
 * may equal h_in).  All three steps are queued on `stream` and the call
 * returns at once when the host buffers are page-locked (cudaHostAlloc /
 * cudaHostRegister); with pageable buffers the CUDA runtime stages the
 * copies and the call may block.  Independent sorts issued this way on two
 * streams (each with its own sorter and d_work) overlap one sort's copies
 * with the other's kernels.
 * Errors: E_INVAL (NULL or misaligned pointers), E_CUDA; kernel-side errors
 * via ipsgpu_status. */
int ipsgpu_sort_host(ipsgpu_sorter *s, const void *h_in, void *h_out, uint64_t n, void *d_work,
                     void *stream);

/* One partitioning step with given splitters (Sec. 3.1.2 - 3.1.4): classify
 * every element with the branchless tree over the sorted splitters
 * d_splitters[0..num_splitters) (elements of the sorter's dtype, only their
 * keys are read), then move the elements in place so that bucket j occupies
 * d_data[d_bucket_begin[j] .. d_bucket_begin[j+1]).  With K =
 * 2^ceil(log2(num_splitters+1)) leaves, the classes are
 *   equal_buckets == 0: class(e) = smallest i < K-1 with e <= s_i, else K-1
 *   equal_buckets != 0: class(e) = 2i + 1 - [e < s_i] over the splitters
 *                       padded to K entries with the largest one (Sec. 2)
 * and B = K or 2K; d_bucket_begin receives B+1 values (u64, device memory).
 * Order inside a bucket is unspecified.  B must be <= the sorter's k.
 * Errors: E_INVAL (num_splitters == 0, B > k, NULL or misaligned data or
 * splitter pointers). */
int ipsgpu_partition_level(ipsgpu_sorter *s, void *d_data, uint64_t n,
                           const void *d_splitters, uint32_t num_splitters,
                           int equal_buckets, uint64_t *d_bucket_begin, void *stream);

/* One IPS2Ra partitioning step (Sec. 5): class(e) = (key >> shift) &
 * (2^bits - 1), bits in [1, 8] with 2^bits <= k; d_bucket_begin receives
 * 2^bits + 1 values.  U32 / U64 / PAIR_U64 only (E_UNSUPPORTED otherwise). */
int ipsgpu_radix_level(ipsgpu_sorter *s, void *d_data, uint64_t n, uint32_t shift,
                       uint32_t bits, uint64_t *d_bucket_begin, void *stream);

/* Sort many independent arrays in one call (segmented sort): segment i is
 * d_data[d_offsets[i] .. d_offsets[i+1]) for i < num_segments, sorted in
 * place exactly as ipsgpu_sort would sort it alone.
 *   - d_offsets: num_segments + 1 u64 element offsets in device memory,
 *     non-decreasing, the last one <= n; n is the length of d_data.  A
 *     segment that violates this is left untouched and E_INVAL is recorded
 *     in the status word.  Elements outside every segment are not touched.
 *   - The recursion of Sec. 3.2 runs on the device over all segments at
 *     once: segments that need a partitioning step wait in a FIFO ring and
 *     are taken in waves sized to the sorter's fixed scratch, so scratch
 *     does not grow with n or with the number of segments.  The waves run
 *     inside one CUDA graph launch (a conditional WHILE node); the call
 *     never synchronizes.  Unlike ipsgpu_sort it does not look for already
 *     sorted or reversed inputs.
 *   - Kernel-side errors go to the status word (ipsgpu_status); after an
 *     error the data still holds a permutation of every segment.
 * Errors: E_INVAL (NULL or misaligned pointers, n > 2^40, num_segments >
 * 2^32 - 1), E_CUDA. */
int ipsgpu_sort_segmented(ipsgpu_sorter *s, void *d_data, uint64_t n,
                          const uint64_t *d_offsets, uint64_t num_segments, void *stream);

/* Sort many separate arrays in one call: array i starts at the device
 * address d_segs[2i] (aligned as for ipsgpu_sort) and has d_segs[2i+1]
 * elements; d_segs holds 2 * num_segments u64 in device memory.  Each array
 * is sorted in place exactly as ipsgpu_sort_segmented would sort it; the
 * arrays must not overlap.  Asynchronous, never synchronizes; an entry with
 * a NULL or misaligned address (and n > 0) or n > 2^40 is skipped and
 * recorded as E_INVAL in the status word.
 * Errors: E_INVAL (NULL or misaligned d_segs, num_segments > 2^32 - 1),
 * E_CUDA. */
int ipsgpu_sort_batch(ipsgpu_sorter *s, const uint64_t *d_segs, uint64_t num_segments,
                      void *stream);

/* A segmented sort over fixed buffers (d_data, d_offsets) as one
 * instantiated CUDA graph: a node that sets up the run, then the WHILE loop
 * over waves.  ipsgpu_graph_launch replays it with one call; it reads the
 * offsets and data at launch time, so the caller may refill both buffers
 * between launches.  The graph uses the sorter's scratch: launches of graphs
 * of one sorter, and its other calls, must not overlap on the GPU.  Errors:
 * as ipsgpu_sort_segmented, plus E_CUDA if building the graph fails. */
typedef struct ipsgpu_graph ipsgpu_graph;
int ipsgpu_segmented_graph_create(ipsgpu_sorter *s, void *d_data, uint64_t n,
                                  const uint64_t *d_offsets, uint64_t num_segments,
                                  ipsgpu_graph **out);
int ipsgpu_graph_launch(ipsgpu_graph *g, void *stream);
/* Number of top-level nodes of the graph (the setup node and the WHILE node). */
int ipsgpu_graph_nodes(ipsgpu_graph *g, uint64_t *nodes);
int ipsgpu_graph_destroy(ipsgpu_graph *g);

/* The classification rule alone (Sec. 2 branchless tree, Algorithm 1):
 * writes class(d_data[i]) to d_class[i] (u32, device) without moving data.
 * Same splitter semantics and errors as ipsgpu_partition_level. */
int ipsgpu_classify(ipsgpu_sorter *s, const void *d_data, uint64_t n,
                    const void *d_splitters, uint32_t num_splitters, int equal_buckets,
                    uint32_t *d_class, void *stream);

/* Synchronize `stream`, return the sorter's device status word (IPSGPU_OK
 * if no kernel reported an error since the last call) and clear it. */
int ipsgpu_status(ipsgpu_sorter *s, void *stream);

/* Static description of a status code. */
const char *ipsgpu_strerror(int code);

/* Per-kernel timing.  When enabled, every kernel launch of the sorter is
 * bracketed by CUDA events on its stream; ipsgpu_kernel_stats synchronizes
 * and reports, for kernel kind i (names from ipsgpu_kernel_name), the number
 * of launches, their summed device time in ms and the algorithmic bytes
 * those launches moved (as defined in the library's design notes).  Arrays
 * have `cap` entries; returns the number of kinds. */
int ipsgpu_set_timing(ipsgpu_sorter *s, int enable);
int ipsgpu_kernel_stats(ipsgpu_sorter *s, uint64_t *launches, double *ms,
                        double *bytes, int cap);
const char *ipsgpu_kernel_name(int kind);

/* Recursion statistics of the sorter's last sort, segmented or batched run
 * made with timing on (the host-driven waves of the device-planned
 * recursion, Sec. 3.2's task structure breadth-first): the number of waves,
 * the largest number of segments waiting in the sorter's fixed ring between
 * two waves (the task metadata the recursion keeps; App. B's strictly
 * in-place variant keeps none), and the ring's capacity.  Zeros if the last
 * run was not timed.  Errors: E_INVAL (s NULL). */
int ipsgpu_wave_stats(ipsgpu_sorter *s, uint64_t *waves, uint64_t *max_pending,
                      uint64_t *ring_capacity);

/* Test hook for failure detection: launches one kernel that waits, with the
 * sorter's bounded-wait helper and at most `spin_limit` polls, on a device
 * flag that nothing sets, so the wait must give up and record
 * IPSGPU_E_TIMEOUT in the status word (read it with ipsgpu_status). */
int ipsgpu_debug_bounded_wait(ipsgpu_sorter *s, uint32_t spin_limit, void *stream);

/* Out-of-bounds write detection without a sanitizer: every device buffer of
 * a sorter lies between two 256-byte guard zones filled with 0xA5 at
 * creation.  Synchronizes the device and checks every guard.  Returns
 * IPSGPU_OK if all are intact; IPSGPU_E_INTERNAL if one changed (a kernel
 * wrote past a buffer's end or before its start), with *first_bad (if not
 * NULL) the index of the first such buffer in creation order (UINT64_MAX
 * when none).  Errors: E_INVAL (s NULL), E_CUDA. */
int ipsgpu_debug_check_guards(ipsgpu_sorter *s, uint64_t *first_bad);

/* ------------------------------------------------------------------ serving
 * A server sorts requests that arrive at any time: it admits them by HBM
 * footprint and runs them on a few CUDA streams ("lanes") while others are
 * in flight.  The caller owns every request's device buffer.
 *   - Footprint: a request of n elements of type t needs n * sizeof(t) bytes,
 *     its own data, because the sort is in place; the server adds the fixed
 *     scratch of one sorter per (lane, served type), allocated at creation.
 *     A request is admitted while the admitted requests plus that scratch
 *     stay within hbm_budget_bytes; the last small_reserve_bytes of it admit
 *     small requests (at most batch_max_elems elements) only, so a large
 *     request that waits for memory does not keep small ones out.
 *   - Batching: started requests wait in one FIFO queue.  Requests of at most
 *     batch_max_elems elements are batched (oldest first, one type per batch,
 *     at most batch_max_requests) into one ipsgpu_sort_batch run at high
 *     stream priority, preferably on the last lane, which takes nothing
 *     else; larger ones run alone (ipsgpu_sort) at low priority on any other
 *     free lane, except a request holding at least half of hbm_budget_bytes,
 *     which runs at high priority (requests waiting for admission wait for
 *     its memory).  A request that cannot run yet does not hold back those
 *     behind it.
 *   - Each request's result is exactly what ipsgpu_sort gives for it alone
 *     (for PAIR_U64, REC100 and QUARTET: the same keys, records with equal
 *     keys in some order).
 * Thread safety: every server call may be made from any host thread. */
typedef struct ipsgpu_server ipsgpu_server;
typedef struct {
    uint64_t hbm_budget_bytes;    /* admitted request bytes + server scratch */
    uint64_t batch_max_elems;     /* 0: 2^22 */
    uint64_t small_reserve_bytes; /* budget only small requests may use; 0: budget / 32 */
    uint32_t lanes;               /* 0: 4 (the last one runs batches only) */
    uint32_t dtype_mask;          /* bit t serves ipsgpu_dtype t; 0: U32|U64|PAIR_U64 */
    uint32_t batch_max_requests;  /* 0: 4096 */
    uint32_t reserved;
} ipsgpu_server_config;

/* Create a server on the current device: lanes, sorters (params as for
 * ipsgpu_sorter_create) and a scheduler thread.
 * Errors: E_INVAL (cfg or out NULL, hbm_budget_bytes 0, more than 64 lanes,
 * a dtype_mask bit above IPSGPU_QUARTET, small_reserve_bytes not below the
 * budget, params invalid for a served dtype, e.g. RADIX with F64), E_NOMEM
 * (the sorters' scratch above the budget, or allocation), E_CUDA.  The
 * argument checks come before any CUDA call. */
int ipsgpu_server_create(const ipsgpu_server_config *cfg, const ipsgpu_params *params,
                         ipsgpu_server **out);
/* Drain, stop the scheduler and free everything. */
int ipsgpu_server_destroy(ipsgpu_server *srv);
/* Admit a request of n elements of dtype: reserves its footprint and
 * returns a ticket.  E_BUSY: it does not fit now (retry after releases);
 * E_NOMEM: it never fits; E_UNSUPPORTED: dtype not served; E_INVAL: NULL
 * arguments, an unknown dtype or n > 2^40. */
int ipsgpu_server_reserve(ipsgpu_server *srv, uint64_t n, int dtype, uint64_t *ticket);
/* Start a reserved request on d_data (n elements, aligned as for
 * ipsgpu_sort).  If ready_stream is not NULL the sort waits for the work
 * enqueued on it so far (the caller may still be filling d_data there). */
int ipsgpu_server_start(ipsgpu_server *srv, uint64_t ticket, void *d_data, void *ready_stream);
/* reserve + start(ready_stream = NULL). */
int ipsgpu_server_submit(ipsgpu_server *srv, void *d_data, uint64_t n, int dtype,
                         uint64_t *ticket);
/* done = 1 once the request's sort has finished on the GPU; status = its
 * status code (IPSGPU_OK, or the error its run reported). */
int ipsgpu_server_poll(ipsgpu_server *srv, uint64_t ticket, int *done, int *status);
/* Block until the request is done; returns its status.  E_INVAL for an
 * unknown ticket or one that was reserved but never started. */
int ipsgpu_server_wait(ipsgpu_server *srv, uint64_t ticket);
/* Host steady-clock times in microseconds: started, launched, seen done. */
int ipsgpu_server_times(ipsgpu_server *srv, uint64_t ticket, double *t_submit_us,
                        double *t_launch_us, double *t_done_us);
/* The clock of ipsgpu_server_times. */
double ipsgpu_server_now_us(void);
/* Return a request's footprint (reserved or done) and forget its ticket.
 * Errors: E_INVAL (unknown ticket), E_BUSY (started and still queued or
 * running: wait for it, or cancel it first while it is queued). */
int ipsgpu_server_release(ipsgpu_server *srv, uint64_t ticket);
/* Cancel a request that has not begun to run: a reserved one, or a started
 * one still waiting in the queue.  It becomes done with status
 * IPSGPU_E_CANCELED (poll / wait report it) and its data is left untouched;
 * release it as usual.  Errors: E_INVAL (unknown or already done ticket),
 * E_BUSY (already running: it will complete normally). */
int ipsgpu_server_cancel(ipsgpu_server *srv, uint64_t ticket);
/* Block until every started request is done. */
int ipsgpu_server_drain(ipsgpu_server *srv);
/* Bytes admitted now (scratch included), the budget, the scratch. */
int ipsgpu_server_usage(ipsgpu_server *srv, uint64_t *used, uint64_t *budget, uint64_t *scratch);

/* One partitioning level with given splitters, like ipsgpu_partition_level,
 * for callers that cannot allocate memory: code running while a CUDA graph is
 * being captured, code inside an allocator or memory-pool callback, or a
 * service that reserves all device memory up front.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *   - No sorter is needed and nothing is allocated: all scratch lives in a
 *     fixed device array inside the library (about 8.2 MiB, held by every GPU
 *     that loads the library until the process exits).  The caller passes the
 *     data, the splitters and d_bucket_begin exactly as for
 *     ipsgpu_partition_level; dtype is an ipsgpu_dtype.
 *   - Limits: n <= 2^32 - 1 elements and B <= 256 classes; larger requests
 *     return IPSGPU_E_INVAL.
 *   - The first call on a device (of any dtype) looks up the array's device
 *     address and sets the kernel attributes of every dtype; make that first
 *     call before any stream capture.
 *   - Every call uses the same array and leaves its contents behind, so calls
 *     whose work overlaps on the GPU (other streams, other host threads) race:
 *     serialize them.
 *   - A kernel-side error (a bounded wait that ran out, an inconsistent count)
 *     is reported by writing ~0 into d_bucket_begin[B], which otherwise
 *     equals n. */
int ipsgpu_partition_level_noalloc(int dtype, void *d_data, uint64_t n, const void *d_splitters,
                                   uint32_t num_splitters, int equal_buckets,
                                   uint64_t *d_bucket_begin, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IPSGPU_H */
