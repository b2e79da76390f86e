/*
 * tdq.h -- C ABI of libtdq, a GB300 (sm_103a) implementation of the distance
 * threshold search over trajectory databases of Gowanlock & Casanova,
 * "Parallel Distance Threshold Query Processing for Spatiotemporal
 * Trajectory Databases on the GPU" (arXiv 1405.7461).
 *
 * Problem (Sec. 3): the database D holds n 4-D line segments (x,y,z,t of a
 * start point and of an end point, a segment id and a trajectory id).  A
 * query is a set of query segments, a distance d and a time window [t0,t1].
 * The result holds, for every (query segment, entry segment) pair that comes
 * within distance d during the common time span of both segments inside the
 * window, that pair and the sub-interval [t_enter, t_exit] in absolute time.
 *
 * Conventions shared by every call:
 *  - Every call returns a tdq_status; on error no output is produced (output
 *    handles are left NULL) and tdq_last_error() gives a message.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work of a call is ordered on that stream.
 *  - Device pointers refer to memory of the CUDA device that is current on
 *    the calling thread; an index is bound to the device it was built on.
 *  - Readings of the paper that these calls implement:
 *      * two segments form a pair only if their common span has positive
 *        length (a < b); segments that only touch at an instant do not;
 *      * "within d" is inclusive (distance <= d);
 *      * the window clips the common span; a window with t0 > t1 is invalid;
 *      * at most one interval per pair (the squared distance of two linearly
 *        moving points is a convex quadratic in time, Sec. 5).
 *  - One search at a time per index (calls on one index must not overlap).
 */
#ifndef TDQ_H
#define TDQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TDQ_OK = 0,
    TDQ_ERR_INVALID = 1,  /* NULL argument, non-finite value, t_end <= t_start, d < 0 or NaN, t0 > t1 */
    TDQ_ERR_NOMEM = 2,    /* a device or host allocation failed; nothing leaked */
    TDQ_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    TDQ_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    TDQ_ERR_OVERFLOW = 5  /* a caller-provided result buffer is too small (see tdq_search_device) */
} tdq_status;

/* A segment set in structure-of-arrays form (Sec. 3).  Columns are float64
 * (start point xs,ys,zs at time ts; end point xe,ye,ze at time te) and int64
 * ids, n entries each.  on_device = 0: host memory; 1: device memory.
 * traj_id may be NULL (ids then read as 0).  The library copies what it
 * needs; the caller keeps ownership of these arrays. */
typedef struct {
    const double *xs, *ys, *zs, *ts;
    const double *xe, *ye, *ze, *te;
    const int64_t *seg_id;
    const int64_t *traj_id;
    uint64_t n;
    int on_device;
} tdq_segments;

/* Temporal-bin index parameters (Sec. 4).  bin_count = m, the number of
 * fixed-width bins over the database's temporal extent; 0 selects 10,000,
 * the value used in the paper's experiments (Sec. 7.2). */
typedef struct {
    uint32_t bin_count;
} tdq_index_params;

/* Opaque index: the entry segments sorted by t_start in device memory (SoA)
 * and the bin table, plus the search workspace.  Owns its device memory. */
typedef struct tdq_index tdq_index;

/* Search modes.  All three return the same pairs and intervals: the
 * pre-tests only drop pairs whose bounding spheres (the query's grown by d)
 * cannot meet, which therefore never come within d (Sec. 3), and the FP64
 * evaluation of Sec. 5 / Algorithm 1 decides the rest. */
enum {
    TDQ_MODE_FP64 = 0,        /* every temporal-overlap pair in FP64 (plain method) */
    TDQ_MODE_FP32_FILTER = 1, /* conservative FP32 pre-test, FP64 for the survivors */
    TDQ_MODE_TC_FILTER = 2    /* the sphere pre-test as an exact integer GEMM on the tensor cores (centers
                                 and radii on an 11-bit grid over the entries' extent, radii rounded up to
                                 cover the snapping), FP64 for the survivors */
};

/* Search tuning.  Zero fields select defaults. */
typedef struct {
    uint32_t query_tile;  /* query segments per tile (multiple of 32, <= 32; default 32) */
    uint32_t entry_chunk; /* entry segments per work item (multiple of 256, <= 2048; default 512) */
    int mode;             /* TDQ_MODE_* (default TDQ_MODE_FP64) */
    uint32_t flags;       /* TDQ_FLAG_* (default 0) */
} tdq_search_params;

/* Pair filters of tdq_search_params.flags (no counterpart in the paper's
 * kernel; they express query (ii) of Sec. 2.1, see tdq_self_join).  Both
 * leave the temporal-overlap count of tdq_stats unchanged (it covers every
 * pair). */
#define TDQ_FLAG_OTHER_TRAJECTORIES 1u /* report only pairs whose query and entry trajectory ids differ
                                          (the queries' traj_id must be given) */
#define TDQ_FLAG_UNORDERED_ONCE 2u     /* report a pair only if entry_seg_id > query_seg_id (with the
                                          database as the query set: each unordered pair once) */

/* Host-side results, owned by the library (release with tdq_results_free).
 * Item k: query segment query_seg_id[k] (the caller's id) is within d of
 * entry segment entry_seg_id[k] over [t_enter[k], t_exit[k]].  Order is
 * unspecified.  The searches place the arrays in page-locked host memory
 * (one block per result set, its size rounded up to a power of two, at least
 * 64 KiB; plain host memory when no page-locked memory can be had) that
 * tdq_results_free keeps for reuse by later results (up to 1 GiB; the rest
 * is released).  Result sets held at the same time each keep their block. */
typedef struct {
    int64_t *query_seg_id;
    int64_t *entry_seg_id;
    double *t_enter;
    double *t_exit;
    uint64_t count;
} tdq_results;

/* Device-side result buffer provided by the caller: four device arrays of
 * `capacity` items each (same meaning as tdq_results). */
typedef struct {
    int64_t *query_seg_id;
    int64_t *entry_seg_id;
    double *t_enter;
    double *t_exit;
    uint64_t capacity;
} tdq_result_buffer;

/* Counters of the last search on an index (Sec. 8.1 splits interactions into
 * hits, temporal misses and temporal-hit/spatial-misses). */
typedef struct {
    uint64_t query_segments;    /* query segments searched (after validation) */
    uint64_t interactions;      /* candidate pairs of the tiles' ranges (tile x chunk; a search of at most
                                   1,024 query segments in the FP32 filter mode tests only the pairs of
                                   each segment's own range among them) */
    uint64_t overlap_pairs;     /* pairs whose common span (inside the window) has positive length */
    uint64_t fp64_pairs;        /* pairs evaluated in FP64 (all overlap pairs in FP64 mode) */
    uint64_t results;           /* pairs within d (alpha * interactions) */
    uint64_t work_items;        /* (query tile, entry chunk) work items */
    uint64_t kernel_launches;   /* CUDA kernels the library launched for the search */
    double pair_kernel_ms;      /* device time of the pair kernel (CUDA events; filter modes: the
                                   pre-test kernel) */
    double total_ms;            /* device time of the whole search on its stream */
    uint64_t filter_survivors;  /* filter modes: pairs that passed the pre-test (0 in FP64 mode) */
    double refine_ms;           /* filter modes: device time of the FP64 refine kernel (pair_kernel_ms then
                                   covers the pre-test kernel alone); ~0 for a search of at most 1,024
                                   query segments in the FP32 filter mode, whose pre-test kernel refines its
                                   own survivors */
    uint64_t mma_issued;        /* TDQ_MODE_TC_FILTER: tensor-core MMAs issued (each 128 entries x 128 query
                                   slots x 16 record elements) */
} tdq_stats;

/*
 * Build the temporal-bin index of Sec. 4 over `entries`: entry segments sorted
 * by non-decreasing t_start (ties by input position), m fixed-width bins over
 * [min t_start, max t_end], per bin the largest t_end and the range of sorted
 * positions.  Sorting, binning and the per-segment velocity are computed on
 * the device.  n = 0 is allowed (every search then returns no results).
 * Errors: TDQ_ERR_INVALID for a NULL argument or an invalid segment
 * (non-finite value, t_end <= t_start).  *out is set only on TDQ_OK.
 */
tdq_status tdq_build_index(const tdq_segments *entries, const tdq_index_params *params, void *stream,
                           tdq_index **out);

/* Release an index and all its device memory (NULL is ignored). */
void tdq_index_free(tdq_index *idx);

/* Number of entry segments in the index. */
uint64_t tdq_index_size(const tdq_index *idx);

/*
 * Copy the bin table of Sec. 4 (Fig. 1) to host arrays of *m items each:
 * bin_start = smallest t_start in the bin, bin_end = largest t_end,
 * bin_first/bin_last = sorted positions of the bin's first and last entry;
 * an empty bin has first = last = -1 and start = end = NaN.  *width receives
 * the bin width b and *t_min the lower end of the extent.  Pass NULL arrays
 * to query *m only.  sorted_index (n items, may be NULL) receives the input
 * position of each sorted entry.  Synchronous.
 */
tdq_status tdq_index_bins(const tdq_index *idx, uint32_t *m, double *width, double *t_min, double *bin_start,
                          double *bin_end, int64_t *bin_first, int64_t *bin_last, int64_t *sorted_index);

/*
 * Search (Sec. 4 lookup + Sec. 5 kernel): every query segment against the
 * candidate entry segments its bins select, with threshold d and window
 * [t0, t1] (use -INFINITY/INFINITY for no window).  Queries may be on the
 * host or the device; results are returned in host memory, owned by the
 * library.  The result buffer is grown and the kernel re-run when the
 * results do not fit (the retry of Sec. 5).  Blocks until done.
 * Errors: TDQ_ERR_INVALID (NULL, invalid query segment, d < 0 or NaN,
 * t0 > t1, NaN window).  n = 0 queries gives an empty result.
 */
tdq_status tdq_search(tdq_index *idx, const tdq_segments *queries, double d, double t0, double t1,
                      const tdq_search_params *params, void *stream, tdq_results **out);

/*
 * Self-join, query (ii) of Sec. 2.1 (every trajectory against all other
 * trajectories) with the database as the query set: `entries` must be the
 * segment set the index was built from (same count, traj_id given).  Reports
 * every pair of segments of different trajectories within d during [t0, t1],
 * each unordered pair once, as (query_seg_id < entry_seg_id).  A search with
 * flags TDQ_FLAG_OTHER_TRAJECTORIES | TDQ_FLAG_UNORDERED_ONCE; other fields of
 * params as for tdq_search.  Errors as tdq_search, and TDQ_ERR_INVALID when
 * the count differs from the index's or traj_id is NULL.  Blocks.
 */
tdq_status tdq_self_join(tdq_index *idx, const tdq_segments *entries, double d, double t0, double t1,
                         const tdq_search_params *params, void *stream, tdq_results **out);

/* Release results from tdq_search (NULL is ignored). */
void tdq_results_free(tdq_results *res);

/*
 * Device-resident search: queries in device memory, results written into the
 * caller's device buffer.  *count receives the number of results; when it
 * exceeds out->capacity only the first capacity items are written and the
 * call returns TDQ_ERR_OVERFLOW, so the caller can grow the buffer and call
 * again (Sec. 5).  Blocks until the count is known.
 */
tdq_status tdq_search_device(tdq_index *idx, const tdq_segments *queries, double d, double t0, double t1,
                             const tdq_search_params *params, void *stream, const tdq_result_buffer *out,
                             uint64_t *count);

/*
 * Same as tdq_search_device with a threshold and a window per query segment:
 * d_per_query, t0_per_query, t1_per_query are device arrays of queries->n
 * items (the batched form, where each query trajectory of a batch carries
 * its own d and window).
 */
tdq_status tdq_search_device_batched(tdq_index *idx, const tdq_segments *queries, const double *d_per_query,
                                     const double *t0_per_query, const double *t1_per_query,
                                     const tdq_search_params *params, void *stream,
                                     const tdq_result_buffer *out, uint64_t *count);

/*
 * Allocation-free variant of tdq_search_device.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * at search time -- for example a process whose device memory is already
 * owned by another allocator (a framework's caching pool), or a
 * latency-critical loop that cannot afford cudaMalloc/cudaFree, which may
 * synchronize the whole device.  Build the index beforehand; then this call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * It runs the plain FP64 kernels of tdq_search_device, with the same
 * arguments, results and errors in that mode, but keeps its per-search
 * scratch in one fixed file-scope device array of about 1.5 MiB, held by the
 * device until the process exits.
 *  - Modes: only TDQ_MODE_FP64 with no pair filters.  The filter modes
 *    (whose survivor list has no fixed bound) and any TDQ_FLAG_* are
 *    rejected with TDQ_ERR_INVALID.
 *  - Synchronous: the call copies the counters back to the host and waits
 *    for its stream before it returns.
 *  - Device code: CUDA loads device code and arrays lazily; tdq_build_index
 *    loads all of the library's device code (this array included) on the
 *    index's device, so that no search call -- this one in particular --
 *    loads any.
 *  - Limit: at most 8192 query segments per call; more is rejected with
 *    TDQ_ERR_INVALID and a message naming the limit.
 *  - The first call on a device resolves the array's device address
 *    (cudaGetSymbolAddress) for that device; make that first call before
 *    any stream capture.
 *  - Every call on a device shares the one array, which keeps the previous
 *    call's contents (the call clears what must start at zero).  Calls that
 *    overlap on the GPU race -- including calls on different indexes or
 *    different streams of the same device; serialize them.
 *  - Does not update the index's counters (tdq_get_stats).
 */
tdq_status tdq_search_device_noalloc(tdq_index *idx, const tdq_segments *queries, double d, double t0, double t1,
                                     const tdq_search_params *params, void *stream, const tdq_result_buffer *out,
                                     uint64_t *count);

/*
 * Batched search plan.  The paper splits a query into batches of query
 * segments processed in sequence, one kernel invocation each (Sec. 4, 6.1).
 * A plan runs one batch -- query segments of uneven trajectories, each with
 * its own threshold d and window [t0, t1] -- as one CUDA graph launch: the
 * whole search (counter reset, query preparation and sort, candidate ranges,
 * tiles, pair kernels, overlap count, counter read-back) is captured once per
 * size class of the batch (powers of two up to the plan's largest batch, and
 * that batch size itself) and replayed.  The plan owns its
 * workspace, staging buffers and a result buffer (device memory, or with
 * host_results page-locked host memory); it keeps a pointer
 * to the index (free the plan before the index).  One search at a time per
 * plan; distinct plans on one index may run concurrently on distinct
 * streams.
 */
typedef struct tdq_plan tdq_plan;

typedef struct {
    uint64_t max_query_segments; /* largest batch (required, < 2^31) */
    uint64_t result_capacity;    /* initial device result capacity in items (0: max(|D|, 65536)); grown and the
                                    batch re-run when a batch overflows it (Sec. 5) */
    uint32_t entry_chunk;        /* as in tdq_search_params (0: mode default) */
    int mode;                    /* TDQ_MODE_* */
    int no_graph;                /* 1: launch the kernels one by one instead of replaying a CUDA graph */
    int host_results;            /* 1: the result buffer is page-locked host memory mapped into the device's address
                                    space: the pair kernels write each result there over the CPU-GPU link, and
                                    tdq_plan_results returns host pointers, readable once tdq_plan_search has
                                    returned (no copy) */
} tdq_plan_params;

tdq_status tdq_plan_create(tdq_index *idx, const tdq_plan_params *params, tdq_plan **out);
void tdq_plan_free(tdq_plan *plan);

/*
 * Search one batch.  queries->n <= max_query_segments; d_per_query,
 * t0_per_query and t1_per_query hold one value per query segment, in the
 * same memory (host or device) as the query columns.  Host inputs are
 * copied into the plan's staging buffers -- unless every array lies in
 * page-locked memory mapped into the device's address space (cudaHostAlloc,
 * cudaHostRegister): then, like device inputs, they are read in place by the
 * replayed graph (over the coherent CPU-GPU link on a Grace-Blackwell node).  The call blocks until the batch is done and returns
 * the number of results in *count.  Errors as tdq_search.
 */
tdq_status tdq_plan_search(tdq_plan *plan, const tdq_segments *queries, const double *d_per_query,
                           const double *t0_per_query, const double *t1_per_query, void *stream, uint64_t *count);

/* View of the plan's results (valid until the next search on the plan or
 * its release): the first *count items of the four arrays -- device
 * pointers, or host pointers for a plan created with host_results. */
tdq_status tdq_plan_results(const tdq_plan *plan, tdq_result_buffer *view, uint64_t *count);

/* Copy the first n results of the plan's last search into caller arrays:
 * host memory (to_device = 0) or device memory (to_device = 1).  Page-locked
 * host arrays (cudaHostAlloc, cudaHostRegister, pinned tensors) are written
 * by one kernel over the CPU-GPU link; others through copies.  Blocks. */
tdq_status tdq_plan_copy_results(const tdq_plan *plan, int64_t *query_seg_id, int64_t *entry_seg_id,
                                 double *t_enter, double *t_exit, uint64_t n, int to_device, void *stream);

/* Counters of the plan's last search (total_ms: device time of the graph). */
tdq_status tdq_plan_get_stats(const tdq_plan *plan, tdq_stats *out);

/*
 * Autotuner: measures, on a sample of query segments (with their own d and
 * windows), the bin count m of the index (Sec. 4), the entry chunk of the
 * pair kernels, and the batch size of a plan, and suggests a per-batch
 * result capacity.  Candidates default to m in {1000, 10000, 100000},
 * chunks {256, 512, 1024}, batches {1024, 4096, 16384, 65536, 262144, the
 * whole sample}; the chosen batch is the smallest whose throughput is within
 * batch_tolerance of the best.  Builds temporary indexes; blocks.
 */
typedef struct {
    const uint32_t *bin_counts;
    int n_bin_counts;
    const uint32_t *entry_chunks;
    int n_entry_chunks;
    const uint64_t *batch_sizes;
    int n_batch_sizes;
    int mode;               /* TDQ_MODE_* to tune for */
    int repeats;            /* timed repetitions per candidate (0: 3, at most 16) */
    double batch_tolerance; /* 0: 0.05 */
} tdq_autotune_params;

typedef struct {
    uint32_t bin_count;
    uint32_t entry_chunk;
    uint64_t batch_query_segments;
    uint64_t result_capacity;          /* suggested for batches of batch_query_segments */
    double ms_per_query_segment;       /* measured at the chosen setting */
    double results_per_query_segment;  /* measured on the sample */
} tdq_tuning;

tdq_status tdq_autotune(const tdq_segments *entries, const tdq_segments *sample, const double *d_per_query,
                        const double *t0_per_query, const double *t1_per_query, const tdq_autotune_params *params,
                        void *stream, tdq_tuning *out);

/*
 * Serving loop with continuous batching.  The paper's setting is online: one
 * database resident on the GPU, many queries, response time as the
 * objective, batches because result memory is reserved up front, and several
 * users competing for that memory (Sec. 3).  A server keeps the index
 * resident and runs `lanes` worker threads, each with its own CUDA stream and
 * batched plan.  Submitted requests (one query trajectory's segments with its
 * own d and window) wait in a FIFO queue; a free lane admits requests from
 * its head while the batch stays within max_batch_query_segments and the
 * estimated result-buffer bytes of all admitted, unfinished requests stay
 * within memory_cap_bytes (at least one request is admitted when nothing is
 * in flight), then searches the batch.  Requests that arrive while batches
 * are running are admitted by free lanes as slots and memory free up, so
 * batches overlap on the device.  A request's results do not depend on the
 * batch it ran in.  The server keeps a pointer to the index; free the
 * server first.
 */
typedef struct tdq_server tdq_server;

typedef struct {
    uint64_t max_batch_query_segments; /* per batch, and the largest request (0: 65536) */
    uint64_t memory_cap_bytes;         /* admission cap on estimated result-buffer bytes (0: 16 GiB) */
    int lanes;                         /* concurrent batches (0: 2, at most 16) */
    int mode;                          /* TDQ_MODE_* */
    uint32_t entry_chunk;              /* 0: mode default */
    double results_per_query_segment;  /* estimate used for admission (0: 4); tdq_autotune measures it */
} tdq_server_params;

typedef struct {
    double queue_ms;    /* submit -> admitted to a batch */
    double run_ms;      /* admitted -> results ready */
    double latency_ms;  /* submit -> results ready */
    uint64_t batch;     /* id of the batch the request ran in */
    uint64_t batch_query_segments;
} tdq_request_info;

typedef struct {
    uint64_t requests_submitted;
    uint64_t requests_completed;
    uint64_t batches;
    uint64_t failed_batches;
    uint64_t query_segments;
    uint64_t max_concurrent_batches; /* most batches running at once */
    double peak_bytes_in_flight;     /* largest estimated bytes admitted at once */
    uint64_t queued;                 /* requests waiting now */
} tdq_server_stats;

tdq_status tdq_server_create(tdq_index *idx, const tdq_server_params *params, tdq_server **out);

/* Queue one request (host memory; copied).  Validated here: TDQ_ERR_INVALID
 * for bad segments, d < 0 or NaN, NaN or reversed window, or more segments
 * than max_batch_query_segments.  *ticket identifies it for tdq_server_wait. */
tdq_status tdq_server_submit(tdq_server *srv, const tdq_segments *queries, double d, double t0, double t1,
                             uint64_t *ticket);

/* Queue `count` requests in one call (the paper's setting of many users
 * querying one resident database, Sec. 3; one call instead of one per
 * request, so that a caller's per-call cost does not bound the server).
 * Request k is query segments [offsets[k], offsets[k+1]) of `queries` (host
 * memory, copied; offsets has count + 1 non-decreasing entries starting at
 * 0 and ending at queries->n) with threshold d[k] and window [t0[k], t1[k]].
 * Every request is validated as by tdq_server_submit before any is queued:
 * on an error nothing is queued and TDQ_ERR_INVALID names the first bad
 * request.  tickets (count entries) receive the requests' tickets, for
 * tdq_server_wait. */
tdq_status tdq_server_submit_many(tdq_server *srv, const tdq_segments *queries, const uint64_t *offsets,
                                  uint64_t count, const double *d, const double *t0, const double *t1,
                                  uint64_t *tickets);

/* Wait (timeout_ms < 0: no limit) until every request submitted so far has
 * finished its search (its results then wait for tdq_server_wait).
 * TDQ_ERR_TIMEOUT if not in time. */
tdq_status tdq_server_drain(tdq_server *srv, int64_t timeout_ms);

/* Wait for a request (timeout_ms < 0: no limit) and take its results (host,
 * library-owned, release with tdq_results_free) and timings.
 * TDQ_ERR_TIMEOUT if not done in time (the request stays queued/running and
 * can be waited for again). */
tdq_status tdq_server_wait(tdq_server *srv, uint64_t ticket, int64_t timeout_ms, tdq_results **out,
                           tdq_request_info *info);

tdq_status tdq_server_get_stats(tdq_server *srv, tdq_server_stats *out);

/* Finish the queued requests, stop the lanes and release the server. */
void tdq_server_free(tdq_server *srv);

/* Counters of the last completed search on idx. */
tdq_status tdq_get_stats(const tdq_index *idx, tdq_stats *out);

/* Fault injection for tests of the error paths: the allocation (device or
 * pinned host) made `after` allocations from now fails as if memory were
 * exhausted, once; after < 0 disables it.  Calls then return TDQ_ERR_NOMEM
 * and release what they had allocated.  Process-wide. */
void tdq_debug_fail_allocations(int64_t after);

/* Message of the last error on the calling thread ("" if none). */
const char *tdq_last_error(void);

/* Library version string. */
const char *tdq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TDQ_H */
