/*
 * grape_walk.h -- C ABI of libgrape_walk, a GB300 (sm_103a) engine for
 * node2vec second-order biased random walks over sorted CSR graphs.
 *
 * The method is GRAPE's (Cappelletti et al., arXiv 2110.06196), Methods,
 * "Implementation of second-order RWs":
 *   a walk at v that arrived from t moves to x in N(v) with un-normalised
 *   probability pi_vx = alpha_pq(t, x) * w_vx                  (eq. alphaRW)
 *   alpha = 1/p if x == t, 1 if x in N(t), 1/q otherwise         (eqs. alpha, beta
 *   and "Efficient computation of the in-out and return bias").
 *   The first step has no t and is first-order, pi_vx = w_vx ("First and
 *   second-order RW-based embedding methods").
 *
 * Sampling is exact rejection sampling, in place of the paper's per-step
 * cumulative sum ("Efficient sampling for Node2Vec RWs"):
 *   - trial k of step s of walk w draws one Philox4x32-10 block (r0, r1, r2, r3),
 *     with key = seed and counter = (w lo, w hi, s, k);
 *   - the proposal is x = row_v[floor((r1:r0) * deg_v / 2^64)];
 *   - it is accepted iff r2 < T_class (unweighted) or
 *     r2 * wmax_v < T_class * w_vx (weighted, compared exactly over the reals).
 *     Here T_class = floor(alpha_class / max(1/p, 1, 1/q) * 2^32) and wmax_v is
 *     the largest weight in the row of v;
 *   - after `trial_cap` rejections the step is drawn by inverse transform over
 *     the cumulative sum of pi in row order, with the Philox block of trial
 *     index trial_cap.
 * A walk is therefore a pure function of (graph, start, walk id, seed, p, q):
 * the same bytes come out of every entry point below, alone, batched or served.
 *
 * Conventions
 *   - CSR: offsets int64[num_nodes + 1] with offsets[0] = 0 and
 *     offsets[num_nodes] = num_entries; dsts int32[num_entries], each row
 *     strictly increasing (sorted, no multi-edges), ids in [0, num_nodes);
 *     weights fp32[num_entries], finite and > 0, or NULL for unweighted.
 *     Self-loops are allowed.  N(t) is the out-row of t ("x in N(t)" is read as
 *     the directed edge t -> x; for undirected graphs, store both directions).
 *   - Output rows: int32, walk_len entries per walk.  Entry 0 is the start and
 *     entry s is the node after s transitions.  Once a walk reaches a node
 *     without out-edges, the rest of its row is -1.  Walk w = r * num_starts + i
 *     is repetition r of starts[i], and its row is row w.
 *   - Device pointers are CUDA device (or managed) addresses on the current
 *     device.  Streams are cudaStream_t values (struct CUstream_st *); NULL is the
 *     legacy default stream.  Every launch is asynchronous on the given stream.
 *   - Errors in arguments are returned synchronously, before anything is
 *     enqueued.  Errors found on the device (a start id out of range) set the
 *     graph's device status word.  Their rows are filled with -1.
 *     grape_stream_status reads the word and clears it.  Kernels never trap.
 *   - Thread safety: a graph is immutable after creation, except through
 *     grape_graph_set_tuning, and may be used from several host threads and
 *     streams at once.  Server calls are thread-safe.
 */
#ifndef GRAPE_WALK_H
#define GRAPE_WALK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* grape_stream_t;   /* identical to cudaStream_t */

typedef enum grape_status {
    GRAPE_OK = 0,
    GRAPE_ERR_INVALID_ARG = 1,    /* bad argument; nothing was enqueued */
    GRAPE_ERR_INVALID_GRAPH = 2,  /* CSR failed validation */
    GRAPE_ERR_NOMEM = 3,          /* device or host allocation failed, or request above the server cap */
    GRAPE_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    GRAPE_ERR_TIMEOUT = 5,        /* a bounded wait ran out */
    GRAPE_ERR_BUSY = 6,           /* server queue full (try again) */
    GRAPE_ERR_CANCELLED = 7,      /* request cancelled or server shut down */
    GRAPE_ERR_DEVICE = 8,         /* the device status word was set (bad start id) */
    GRAPE_ERR_NOT_FOUND = 9       /* unknown ticket */
} grape_status_t;

/* Message for a status code (static storage). */
const char* grape_status_string(grape_status_t status);

/* ------------------------------------------------------------------------ */
/* Graphs                                                                    */
/* ------------------------------------------------------------------------ */

typedef struct grape_graph grape_graph_t;

#define GRAPE_UNDIRECTED 1u  /* caller asserts every row pair is symmetric (with equal weights);
                                membership may then search whichever of N(t), N(x) is shorter */
#define GRAPE_VALIDATE   2u  /* check the CSR on the device before accepting it */

/*
 * Copy a CSR graph into library-owned device memory and build the per-node
 * records the walks read (row offset, degree, largest row weight).  The layout
 * follows GRAPE, Methods, "Graph data structures" (CSR with sorted adjacency).
 *   offsets, dsts, weights: device pointers laid out as in Conventions.  The
 *       caller keeps ownership; they may be freed once `stream` has reached
 *       this call's work (the copies are enqueued on it).
 *   num_nodes in [1, 2^31 - 1]; num_entries in [0, 2^62].  The graph holds
 *   node records (16 bytes per node), the sorted rows and their sector pivots
 *   (4.5 bytes per entry), one 32-byte proposal entry per CSR entry (the
 *   target's degree, row offset and largest row weight, the weight, and the
 *   position of the row's node in the target's row), and an edge hash: every
 *   pair stored once in 32-byte buckets of eight slots at 2 to 3.5 pairs per
 *   bucket (8-16 bytes per undirected edge), so that a membership test reads one
 *   bucket.  The hash is left out when it would exceed twice the sorted rows.
 *   A proposal entry also carries a filter that proves non-memberships: on
 *   undirected graphs with the hash, of N(v) n N(x) for the entry (v -> x) (96
 *   bits unweighted; 32 bits weighted, in place of the reverse weight, which
 *   the GRAPE_UNDIRECTED flag asserts equal); otherwise, on unweighted graphs,
 *   of N(x).  Unweighted graphs need another 16 * num_nodes bytes of scratch,
 *   and the hash 4 bytes per bucket, from the device's stream-ordered pool
 *   during the call.  grape_graph_info reports the bytes held.
 *   flags: GRAPE_UNDIRECTED | GRAPE_VALIDATE.  With GRAPE_VALIDATE the call
 *       synchronises `stream` and returns GRAPE_ERR_INVALID_GRAPH for:
 *       non-monotone offsets, wrong first or last offset, ids out of range,
 *       rows not strictly increasing, weights not finite or <= 0, or (with
 *       GRAPE_UNDIRECTED) a missing or unequal reverse entry.
 *   *out receives the graph on GRAPE_OK, and NULL otherwise.
 */
grape_status_t grape_graph_create(const int64_t* offsets, const int32_t* dsts,
                                  const float* weights, int64_t num_nodes,
                                  int64_t num_entries, uint32_t flags,
                                  grape_stream_t stream, grape_graph_t** out);

/* Free the graph's device memory (synchronises the device first). NULL is a no-op. */
void grape_graph_destroy(grape_graph_t* graph);

typedef struct grape_graph_info {
    int64_t num_nodes;
    int64_t num_entries;
    int32_t max_degree;
    int32_t weighted;        /* 1 when weights were given */
    int32_t undirected;      /* 1 when GRAPE_UNDIRECTED was given */
    int32_t pad;
    int64_t device_bytes;    /* device memory held by the graph */
    int64_t edge_hash_bytes; /* of which the edge hash (0 when the graph has none) */
} grape_graph_info_t;

grape_status_t grape_graph_info(const grape_graph_t* graph, grape_graph_info_t* info);

/*
 * Launch and search policy.  None of these change any output byte; they only
 * change how the work is spread over the GPU.
 */
typedef struct grape_tuning {
    int64_t trial_cap;        /* rejection trials before the exact fallback, in [0, 2^31 - 1]
                                 (default 4096; 0 = always fall back) */
    int32_t shorter_min;      /* undirected graphs: when deg(t) exceeds this, the record of x is
                                 loaded first and the shorter of N(t), N(x) is searched; otherwise
                                 N(t) is searched at once (INT32_MAX: always N(t)) */
    int32_t block_threads;    /* threads per block for walk kernels (multiple of 32, <= 256) */
    int32_t blocks_per_sm;    /* resident blocks per SM for the grid size; 0 = occupancy maximum */
    int32_t chunk_walks;      /* batched and served queues: walks per queue entry */
    int32_t interp_search;    /* membership probes read the aligned 32-byte sector of the list at
                                 the position interpolated between the known value bounds (1,
                                 default), or at the midpoint (0); an interpolated probe that
                                 does not halve the range is followed by a bisecting one */
    int32_t l2_fetch_bytes;   /* 0: leave the L2 fetch granularity as it is; 32, 64 or 128: set
                                 it (cudaLimitMaxL2FetchGranularity, a per-context limit) when
                                 this tuning is applied */
    int32_t pivot_min;        /* membership searches over lists of at least this many entries
                                 first search the list's sector pivots (the first id of every
                                 aligned 32-byte sector of the sorted rows, held beside them),
                                 which leaves one sector of the list to read; INT32_MAX
                                 (default): never */
    int32_t warp_search_min;  /* membership searches over lists of more than this many entries
                                 are first narrowed by the whole warp, 32 probes at once, one
                                 lane's search at a time; INT32_MAX (default): never.
                                 pivot_min or warp_search_min below INT32_MAX selects kernels
                                 that carry these schedules (general p, q specialisation); the
                                 default kernels compile them out.  grape_walks_batched_static
                                 does not use them. */
    int32_t l2_persist_mb;    /* 0: none; else ask the L2 to keep up to this many MB of the
                                 sector pivots resident (a persisting access-policy window on
                                 each walk launch; cudaLimitPersistingL2CacheSize, a per-context
                                 limit, is raised to it when this tuning is applied) */
    int32_t edge_hash;        /* 1 (default): membership tests read the graph's edge hash, one
                                 32-byte bucket, and search the rows only when that bucket
                                 overflowed; 0: always search the rows */
} grape_tuning_t;

grape_status_t grape_graph_get_tuning(const grape_graph_t* graph, grape_tuning_t* tuning);
grape_status_t grape_graph_set_tuning(grape_graph_t* graph, const grape_tuning_t* tuning);

/* ------------------------------------------------------------------------ */
/* Walks                                                                     */
/* ------------------------------------------------------------------------ */

/*
 * walks_per_node * num_starts walks of walk_len entries each, into
 * out[walks_per_node * num_starts][walk_len] (device, caller-owned, int32).
 * This is the per-call path (GRAPE, "Implementation of second-order RWs"),
 * with the p == 1 / q == 1 / unweighted specialisations of that section
 * picked automatically.
 *   starts: device int32[num_starts], or NULL for 0, 1, ..., num_starts - 1
 *           (then num_starts <= num_nodes).
 *   walk_len >= 1; walks_per_node >= 1; p, q finite and > 0; seed any value.
 *   Starts out of range produce -1 rows and set the device status word.
 * Returns after enqueueing on `stream`.
 */
grape_status_t grape_walks(const grape_graph_t* graph, const int32_t* starts,
                           int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                           double p, double q, uint64_t seed, int32_t* out,
                           grape_stream_t stream);

/*
 * A contiguous shard of a grape_walks job: the walks with ids
 * [walk_begin, walk_begin + walk_count) of the job (starts, num_starts,
 * walks_per_node, ...), written to out[walk_count][walk_len] (row j = walk id
 * walk_begin + j).  The rows are byte-identical to the same rows of the whole
 * job, so a job split over several GPUs (one shard each, no communication)
 * reassembles exactly.
 */
grape_status_t grape_walks_range(const grape_graph_t* graph, const int32_t* starts,
                                 int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                 double p, double q, uint64_t seed, int64_t walk_begin,
                                 int64_t walk_count, int32_t* out, grape_stream_t stream);

/*
 * Approximated walks (GRAPE, Methods, "Approximated RWs"): as grape_walks,
 * except that a step at a node of degree above suss_k considers only suss_k
 * neighbours, one drawn uniformly from each of suss_k equal buckets of row
 * positions (Sorted Unique Sub-Sampling), bucket b holding positions
 * [floor(b deg / suss_k), floor((b + 1) deg / suss_k)), and samples among them
 * with the same rule (rejection, then after trial_cap rejections the cumulative
 * sum over the sub-sample in bucket order).  The member of bucket b comes from
 * the Philox block of trial index 2^31 + b of the step, so the sub-sample is
 * fixed for the step.  suss_k = 0 gives grape_walks' rows; suss_k >= 1 otherwise.
 */
grape_status_t grape_walks_approx(const grape_graph_t* graph, const int32_t* starts,
                                  int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                  double p, double q, uint64_t seed, int32_t suss_k, int32_t* out,
                                  grape_stream_t stream);

/*
 * The walks of grape_walks drawn at every step by the paper's own on-the-fly
 * sampler (GRAPE, Methods, "Efficient sampling for Node2Vec RWs"): the
 * un-normalised probabilities alpha(t, x) * w_vx of every neighbour, their
 * cumulative sum in row order, u = ((r1:r0) >> 11) * 2^-53 * total from the
 * Philox block of trial index 0, and the first neighbour whose cumulative sum
 * exceeds u, in fp64 with every product and sum rounded once.  Its rows equal
 * grape_walks' rows with trial_cap = 0.  A step reads all of N(v) and tests each
 * neighbour against N(t), so its cost does not depend on (p, q) or the weights:
 * the alternative to rejection where most proposals would be rejected.
 * Arguments as grape_walks.
 */
grape_status_t grape_walks_cumsum(const grape_graph_t* graph, const int32_t* starts,
                                  int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                  double p, double q, uint64_t seed, int32_t* out,
                                  grape_stream_t stream);

/*
 * The same walks as grape_walks, with `starts` and `out` in HOST memory
 * (pageable or page-locked).  The call copies the starts in, walks the whole
 * job in one launch and copies the rows out, and returns once `out` holds them
 * (it synchronises `stream`).  The rows are cut into up to 64 slices of walk
 * ids (64 MB or more each); the walk that completes a slice raises the slice's
 * flag in mapped host memory, and the calling thread then copies that slice
 * out on one of the library's per-device copy streams while the launch goes
 * on.  Device scratch for the starts and rows is taken from, and given back to,
 * the device's default stream-ordered memory pool inside the call.
 * Page-locked host buffers let the copies run at the host link's rate.
 */
grape_status_t grape_walks_host(const grape_graph_t* graph, const int32_t* starts,
                                int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                double p, double q, uint64_t seed, int32_t* out,
                                grape_stream_t stream);

/*
 * Give back device scratch that grape_walks_host and grape_walk_contexts keep
 * for reuse in the current device's default stream-ordered memory pool, down
 * to keep_bytes (>= 0).  Synchronises the device first.
 */
grape_status_t grape_trim_scratch(int64_t keep_bytes);

/* ------------------------------------------------------------------------ */
/* Context windows (SkipGram / CBOW input)                                   */
/* ------------------------------------------------------------------------ */

#define GRAPE_MAX_CONTEXT_WINDOW 64

/*
 * Context windows of walk rows, the input the shallow SkipGram and CBOW models
 * learn from (GRAPE, Methods, "First and second-order RW-based embedding
 * methods": windows of a given size sliding over the walks).  For row r and
 * position i:
 *     contexts[r][i][j]          = rows[r][i - window + j]   j = 0 .. window-1
 *     contexts[r][i][window + j] = rows[r][i + 1 + j]        j = 0 .. window-1
 * and -1 where that position lies outside the row, holds -1 (after a dead
 * end), or the centre rows[r][i] is -1.  SkipGram pairs are (centre, entry)
 * over the entries that are not -1.
 *   rows: device int32[num_rows][walk_len]; contexts: device
 *   int32[num_rows][walk_len][2 * window]; window in [1, GRAPE_MAX_CONTEXT_WINDOW].
 * Enqueued on `stream`.
 */
grape_status_t grape_contexts_from_rows(const int32_t* rows, int64_t num_rows, int32_t walk_len,
                                        int32_t window, int32_t* contexts, grape_stream_t stream);

/*
 * Walks [walk_begin, walk_begin + walk_count) of the job that grape_walks(starts,
 * num_starts, walk_len, walks_per_node, p, q, seed) describes, turned into
 * their context windows as in grape_contexts_from_rows.  The walk rows go to
 * `centres` (device int32[walk_count][walk_len]) when it is not NULL; otherwise
 * they live only in scratch taken from, and given back to, the device's
 * stream-ordered pool.  Calling this for consecutive ranges streams a job's
 * windows to a trainer without holding all of its walks.  Enqueued on `stream`.
 */
grape_status_t grape_walk_contexts(const grape_graph_t* graph, const int32_t* starts,
                                   int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                   double p, double q, uint64_t seed, int32_t window,
                                   int64_t walk_begin, int64_t walk_count, int32_t* centres,
                                   int32_t* contexts, grape_stream_t stream);

/* One walk request: rows as in grape_walks. */
typedef struct grape_walk_request {
    const int32_t* starts;    /* device int32[num_starts] for batched calls; HOST for the server */
    int64_t num_starts;       /* >= 1 (NULL starts: 0..num_starts-1) */
    int32_t walk_len;         /* >= 1 */
    int32_t walks_per_node;   /* >= 1 */
    double p, q;              /* finite, > 0 */
    uint64_t seed;
    int32_t* out;             /* device rows (batched); HOST rows or NULL (server) */
} grape_walk_request_t;

/*
 * Batched walks: all requests in one persistent launch, replayed from a CUDA
 * graph.  Each request's rows are byte-identical to a grape_walks call with
 * the same arguments.  Workers take `chunk_walks` walks at a time from one
 * queue that spans the requests, so requests of uneven size, length and
 * (p, q) share the GPU without a launch per request.
 * A plan uploads the request table once and can be launched many times; the
 * request arrays must stay valid while the plan is in use.
 */
typedef struct grape_batch_plan grape_batch_plan_t;

grape_status_t grape_batch_plan_create(const grape_graph_t* graph,
                                       const grape_walk_request_t* requests,
                                       int32_t num_requests, grape_stream_t stream,
                                       grape_batch_plan_t** out);
grape_status_t grape_batch_plan_launch(grape_batch_plan_t* plan, grape_stream_t stream);
void grape_batch_plan_destroy(grape_batch_plan_t* plan);

/* Plan, launch and free in one call (the plan is freed after the launch is enqueued). */
grape_status_t grape_walks_batched(const grape_graph_t* graph,
                                   const grape_walk_request_t* requests,
                                   int32_t num_requests, grape_stream_t stream);

/*
 * grape_walks_batched without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need walks (an allocator of their own owns the memory budget, or
 * allocation is not allowed at that point of their program).  It writes the
 * request table, per-request queue bounds and the queue head into one
 * file-scope device array of fixed size (about 480 KB, held on every GPU that
 * loads the library until the process exits), then runs the same walks as
 * grape_walks_batched: each request's rows are byte-identical.
 *   num_requests must be in [1, 4096]; larger batches return
 *   GRAPE_ERR_INVALID_ARG before anything is enqueued.
 *   The first call on a device, with that device current, looks up the
 *   array's device address (cudaGetSymbolAddress) and the kernel's occupancy;
 *   make that first call before any stream capture.
 *   Every call, on every stream, shares the one array per device.  The queue
 *   head is cleared on each call; the rest keeps the last call's contents.
 *   Calls whose work overlaps on the GPU (two streams, or a second call
 *   before the first finished on another stream) race on it: order them on
 *   one stream or synchronise between them.
 *   No cudaMalloc, cudaFree or other allocating routine is called.  The table
 *   is written by small launches that each carry 32 requests as kernel
 *   parameters, so no host buffer has to outlive the call.  The graph's
 *   tuning (chunk_walks, block_threads, blocks_per_sm, trial_cap, search
 *   policy) and its work counters apply as for grape_walks_batched.
 */
grape_status_t grape_walks_batched_static(const grape_graph_t* graph,
                                          const grape_walk_request_t* requests,
                                          int32_t num_requests, grape_stream_t stream);

/*
 * Autotune the batched path for this graph with CUDA events on the given
 * requests, in two stages: first (chunk_walks, shorter_min, interp_search) over
 * a grid, then, from the best of those, the hub thresholds (pivot_min,
 * warp_search_min).  Stores the fastest in the graph's tuning (also returned in
 * *best when not NULL).  Writes into the requests' out buffers.  Synchronises
 * `stream`.
 */
grape_status_t grape_autotune_batched(grape_graph_t* graph,
                                      const grape_walk_request_t* requests,
                                      int32_t num_requests, grape_stream_t stream,
                                      grape_tuning_t* best);

/*
 * Synchronise `stream`, then read and clear the graph's device status word:
 * GRAPE_OK, or GRAPE_ERR_DEVICE when a kernel saw a start id out of range.
 */
grape_status_t grape_stream_status(const grape_graph_t* graph, grape_stream_t stream);

/*
 * Work counters, summed over every walk kernel that ran on this graph while
 * counting was on (off by default; enabling costs one atomic per warp per
 * counter per kernel).  Used for the bytes-per-step roofline accounting.
 */
typedef struct grape_walk_counters {
    int64_t steps;        /* transitions taken */
    int64_t trials;       /* proposals drawn */
    int64_t gathers;      /* proposals whose entry had to be read (the rest were decided
                             without a read: rejected whatever the target, or the return) */
    int64_t searches;     /* membership tests, deciding acceptance, run on the sorted rows */
    int64_t probes;       /* 32-byte row sectors read by those tests */
    int64_t fallbacks;    /* steps drawn by the exact inverse-transform fallback */
    int64_t walks;        /* rows written */
    int64_t filtered;     /* membership tests settled by the neighbour filters of an
                             unweighted graph, without reading a row */
    int64_t pivot_probes; /* of the probes, 32-byte sectors of the sector pivots */
    int64_t hash_probes;  /* of the probes, 32-byte buckets of the edge hash */
} grape_walk_counters_t;

grape_status_t grape_counters_enable(grape_graph_t* graph, int32_t enable);
/* Synchronises the device, copies the counters out and resets them. */
grape_status_t grape_counters_read(grape_graph_t* graph, grape_walk_counters_t* out);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching with the graph resident on the device         */
/* ------------------------------------------------------------------------ */

typedef struct grape_server grape_server_t;

typedef struct grape_server_config {
    int64_t output_cap_bytes;   /* device bytes for admitted requests' rows and starts (e.g. 40 GB) */
    int32_t max_inflight;       /* requests admitted at once (ring slots), <= 65536 */
    int32_t chunk_walks;        /* walks per work-queue entry; 0 = per request: the graph's
                                   tuned size, raised for a large request so that its
                                   entries give each resident lane up to 16 walks */
    int64_t max_chunks;         /* capacity of the device work queue, in entries */
    int64_t idle_exit_us;       /* the resident kernel is stopped once the server has had nothing
                                   in flight for this long (relaunched with the next request) */
    int32_t admit_timeout_ms;   /* submit waits this long for memory/slots, then GRAPE_ERR_BUSY */
    int32_t kernel_wait_ms;     /* bound on the resident kernel's wait for work while no host
                                   heartbeat arrives (the host beats several times within it);
                                   0 = 2000 */
} grape_server_config_t;

typedef struct grape_server_stats {
    int64_t submitted, admitted, completed, cancelled, rejected;
    int64_t inflight;            /* admitted, not yet complete */
    int64_t bytes_reserved;      /* output arena bytes in use */
    int64_t kernel_launches;     /* resident-kernel launches so far */
    int64_t steps;               /* transitions of completed requests (counted on the device) */
    int64_t kernel_timeouts;     /* resident-kernel launches that ended because their bounded
                                    wait ran out without a host heartbeat */
} grape_server_stats_t;

/*
 * Create a server on `graph` (which must outlive it).  The server owns a
 * device arena of output_cap_bytes, a device request ring and work queue, a
 * compute and a copy stream, and two host threads (scheduler, completion).
 * Requests are admitted while arena bytes and ring slots allow; each is cut
 * into queue entries of chunk_walks walks, appended to the queue that a
 * resident kernel is draining.  Work that arrives while other requests run is
 * picked up by the running kernel.  Finished rows are copied to the host on the
 * copy stream while the kernel keeps running.  The server stops the resident
 * kernel after idle_exit_us without work in flight (all its warps leave
 * together) and relaunches it with the next request.  The kernel's own waits
 * are bounded should the host stop: a warp that has waited kernel_wait_ms
 * without a host heartbeat raises bit 2 of the graph's status word (read by
 * grape_stream_status as GRAPE_ERR_DEVICE) and leaves.  A kernel that ends that
 * way is counted in stats.kernel_timeouts, requests it left unfinished fail
 * with GRAPE_ERR_TIMEOUT, and the next request relaunches it.
 */
grape_status_t grape_walk_server_create(const grape_graph_t* graph,
                                        const grape_server_config_t* config,
                                        grape_server_t** out);

/*
 * Submit a request.  req->starts is HOST memory (copied before return, so it
 * may be reused at once).  req->out is the HOST destination of the rows
 * (walks_per_node * num_starts * walk_len int32).  It must stay valid until
 * grape_walk_server_wait returns for this ticket.  It may be NULL, and then
 * the rows are handed over by wait's host_out.
 * Returns GRAPE_ERR_NOMEM for a request larger than the whole cap, and
 * GRAPE_ERR_BUSY when admission did not succeed within admit_timeout_ms.
 */
grape_status_t grape_walk_server_submit(grape_server_t* server,
                                        const grape_walk_request_t* req,
                                        uint64_t* ticket);

/*
 * Wait up to timeout_ms (< 0: no limit) for a ticket.  On GRAPE_OK the rows
 * are in the host buffer given at submit, or in host_out when that was NULL.
 * Once wait has returned GRAPE_OK, GRAPE_ERR_CANCELLED or a device error,
 * the ticket is retired.  GRAPE_ERR_TIMEOUT leaves it pending.
 */
grape_status_t grape_walk_server_wait(grape_server_t* server, uint64_t ticket,
                                      int64_t timeout_ms, int32_t* host_out);

/*
 * Wait up to timeout_ms (< 0: no limit) for ANY submitted ticket to finish,
 * retire it and return it in *ticket.  *latency_ns (if not NULL) gets the time
 * from submit to the rows being in host memory.  host_out is used as in
 * grape_walk_server_wait.  Returns the ticket's status, or GRAPE_ERR_TIMEOUT.
 */
grape_status_t grape_walk_server_wait_any(grape_server_t* server, int64_t timeout_ms,
                                          uint64_t* ticket, int64_t* latency_ns,
                                          int32_t* host_out);

/* Cancel a pending ticket (its rows are not delivered; wait returns GRAPE_ERR_CANCELLED). */
grape_status_t grape_walk_server_cancel(grape_server_t* server, uint64_t ticket);

grape_status_t grape_walk_server_stats(grape_server_t* server, grape_server_stats_t* stats);

/*
 * Host-side fault injection, for testing the bounded waits.
 * GRAPE_FAULT_NO_HEARTBEAT stops the heartbeat that renews the resident
 * kernel's wait, as a host that has stopped responding would; 0 restores it.
 * Other bits return GRAPE_ERR_INVALID_ARG.
 */
#define GRAPE_FAULT_NO_HEARTBEAT 1u
grape_status_t grape_walk_server_inject_fault(grape_server_t* server, uint32_t faults);

/* Stop admitting, let admitted work finish (bounded), cancel the rest, free everything. */
void grape_walk_server_destroy(grape_server_t* server);

/* ------------------------------------------------------------------------ */
/* Elias-Fano graph store                                                    */
/* ------------------------------------------------------------------------ */

/*
 * A graph held as the Elias-Fano representation of its edge codes (GRAPE,
 * Methods, "Succinct data structures for adjacency matrices"), for graphs whose
 * CSR and proposal entries would not fit the device: about
 * 2 + floor(log2(u / m)) bits per CSR entry plus the indexes and 8 bytes per
 * node of row pointers, against 36 bytes per entry for grape_graph_t.
 *   - Edge Encoding: k = ceil(log2 num_nodes); the entry (a, b) is the code
 *     phi_k(a, b) = a * 2^k + b; u = num_nodes * 2^k.
 *   - Elias-Fano of the m sorted codes: l = floor(log2(u / m)) low bits per
 *     code (0 when u <= m), packed least significant bit first, code i at bits
 *     [i l, (i + 1) l) of the low array; the high parts in the high array as
 *     the inverted unary codes of their gaps, code i's one at bit
 *     (code_i >> l) + i, followed by the zeros that close every bucket up to
 *     (u - 1) >> l (Z = ((u - 1) >> l) + 1 zeros in all, zero j closing bucket j).
 *     Bit b of an array is bit b mod 64 of its 64-bit word b / 64.
 *   - Indexes ("Efficient implementation of Elias-Fano"): the positions of one
 *     number j * quantum (j < ceil(m / quantum)) and of zero number j * quantum
 *     (j < ceil(Z / quantum)).  The paper uses quantum 1024.
 *   - rank(c) = number of codes below c; select(i) = the i-th smallest code
 *     (0-based); deg(a) = rank(phi(a + 1, 0)) - rank(phi(a, 0)) ("Operations on
 *     Elias-Fano").
 *   - Row pointers: rank(phi(a, 0)) for every node (the CSR offsets), so a walk
 *     learns a degree from one read instead of two ranks, which scan the dense
 *     high bits of hub rows.  Rows much longer than their 2^(k - l) buckets
 *     (deg + 2^(k-l) > 448 and deg >= 8 * 2^(k-l)) also get a bucket directory:
 *     the bit offset of each bucket's start, so a membership test in a hub row
 *     reads two offsets instead of scanning.
 */
typedef struct grape_ef_graph grape_ef_graph_t;

#define GRAPE_EF_PAPER_QUANTUM 1024

/*
 * Build the store from a device CSR laid out as in Conventions (the same
 * arguments as grape_graph_create), on `stream`, synchronising it.  The CSR is
 * always checked first (the store's layout is computed from the ids):
 * GRAPE_ERR_INVALID_GRAPH for bad offsets, ids out of range, rows not strictly
 * increasing, or weights not finite or <= 0.  The caller keeps its buffers.
 *   quantum: a power of two in [1, 65536].  num_entries < 2^40.
 *   flags: GRAPE_UNDIRECTED (the caller asserts every entry has its reverse with
 *       the same weight; a membership test may then search the shorter row),
 *       GRAPE_VALIDATE (with GRAPE_UNDIRECTED: check that assertion too).
 *   Weighted graphs also hold the weights (fp32 per entry) and each row's
 *   largest weight (fp32 per node) uncompressed.
 *   *out receives the store on GRAPE_OK, and NULL otherwise.
 */
grape_status_t grape_ef_graph_create(const int64_t* offsets, const int32_t* dsts,
                                     const float* weights, int64_t num_nodes,
                                     int64_t num_entries, int32_t quantum, uint32_t flags,
                                     grape_stream_t stream, grape_ef_graph_t** out);

/* Free the store (synchronises the device first).  NULL is a no-op. */
void grape_ef_graph_destroy(grape_ef_graph_t* graph);

typedef struct grape_ef_info {
    int64_t num_nodes;
    int64_t num_entries;       /* m, the number of codes */
    int64_t universe;          /* u = num_nodes * 2^k */
    int64_t num_zeros;         /* Z */
    int64_t high_bits;         /* m + Z */
    int64_t low_words;         /* ceil(m l / 64) 64-bit words */
    int64_t high_words;        /* ceil((m + Z) / 64) 64-bit words */
    int64_t ones_index_len;    /* ceil(m / quantum) */
    int64_t zeros_index_len;   /* ceil(Z / quantum) */
    int64_t structure_bytes;   /* device bytes of the bit arrays (padding included), indexes, row
                                  pointers and bucket directories */
    int64_t device_bytes;      /* structure_bytes plus the weights and row maxima */
    int32_t code_bits;         /* k */
    int32_t low_bits;          /* l */
    int32_t quantum;
    int32_t weighted;
    int32_t max_degree;
    int32_t directory_rows;    /* rows with a bucket directory */
} grape_ef_info_t;

grape_status_t grape_ef_graph_info(const grape_ef_graph_t* graph, grape_ef_info_t* info);

/*
 * Copy the store's arrays into caller-owned device buffers of the lengths in
 * grape_ef_info_t (low_words, high_words, ones_index_len, zeros_index_len
 * elements; the padding is not copied).  Any pointer may be NULL to skip that
 * array.  Enqueued on `stream`.
 */
grape_status_t grape_ef_graph_export(const grape_ef_graph_t* graph, uint64_t* low,
                                     uint64_t* high, int64_t* ones_index, int64_t* zeros_index,
                                     grape_stream_t stream);

/*
 * out[j] = select(idx[j]), the idx[j]-th smallest code, for n indexes (device
 * int64 arrays).  An index outside [0, m) gives -1 and sets the status word.
 */
grape_status_t grape_ef_select(const grape_ef_graph_t* graph, const int64_t* idx, int64_t n,
                               int64_t* out, grape_stream_t stream);

/* out[j] = rank(values[j]), the number of codes below values[j] (0 for values <= 0, m for values >= u). */
grape_status_t grape_ef_rank(const grape_ef_graph_t* graph, const int64_t* values, int64_t n,
                             int64_t* out, grape_stream_t stream);

/*
 * The walks of grape_walks (same arguments, same rule, byte-identical rows for
 * the same CSR, starts, p, q, seed and trial_cap) read from the Elias-Fano
 * store: each proposal is a select, each degree two ranks, each membership
 * test a rank.  trial_cap in [0, 2^31 - 1] (grape_tuning_t's default is 4096).
 * Starts out of range give -1 rows and set the store's status word.
 */
grape_status_t grape_ef_walks(const grape_ef_graph_t* graph, const int32_t* starts,
                              int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                              double p, double q, uint64_t seed, int64_t trial_cap,
                              int32_t* out, grape_stream_t stream);

/* Synchronise `stream`, read and clear the store's status word (GRAPE_ERR_DEVICE if set). */
grape_status_t grape_ef_stream_status(const grape_ef_graph_t* graph, grape_stream_t stream);

/* Work counters of grape_ef_walks (counting launches only; enabling clears them). */
typedef struct grape_ef_counters {
    int64_t steps;             /* transitions taken */
    int64_t trials;            /* proposals drawn (Philox blocks) */
    int64_t codes_read;        /* proposals whose code was selected */
    int64_t membership_tests;  /* class-deciding tests x in N(t) */
    int64_t sectors;           /* distinct 32-byte sectors each walk step reads (row pointers,
                                  directories, high and low bits, indexes, weights), summed */
    int64_t fallbacks;         /* steps drawn by the cumulative-sum fallback */
    int64_t walks;             /* walks started from a valid start */
} grape_ef_counters_t;

grape_status_t grape_ef_counters_enable(grape_ef_graph_t* graph, int32_t enable);
/* Synchronises the device, copies the counters out and clears them. */
grape_status_t grape_ef_counters_read(grape_ef_graph_t* graph, grape_ef_counters_t* out);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */

/*
 * The device Philox4x32-10 generator the walks use (Salmon et al., SC 2011),
 * evaluated on n counter/key pairs: ctr_key is device uint32[n][6]
 * (c0 c1 c2 c3 k0 k1), out is device uint32[n][4].  Enqueued on `stream`.
 */
grape_status_t grape_philox4x32_10(const uint32_t* ctr_key, int64_t n, uint32_t* out,
                                   grape_stream_t stream);

/*
 * Random 32-byte-sector gather probe: the ceiling of independent random
 * sector reads on this device, the denominator the walk kernels' gathers are
 * compared with.  Each read fetches one aligned 32-byte sector of `buf`
 * (device, `buf_bytes` long, 32-byte aligned) at a position drawn by a hash of
 * (seed, thread, read).  The launch shape is swept by the caller:
 *   mode: the load's cache path: 0 read-only through L1 (ld.global.nc),
 *       1 L2 only (ld.global.cg), 2 streaming (ld.global.cs);
 *   load_bytes: 4, 16 or 32 (a 32-, 128- or 256-bit load at the sector start),
 *       or 64 (both sectors of a random aligned 64-byte block, two 256-bit
 *       loads; a read then counts as two sectors);
 *   loads_in_flight: independent reads each thread issues before it waits:
 *       8/16/32/64 for 4-byte loads, 8/16/32 for 16-byte loads, 4/8/16 for
 *       32-byte loads, 4/8 for 64-byte reads; other pairs return
 *       GRAPE_ERR_INVALID_ARG;
 *   blocks_per_sm: resident 256-thread blocks per SM, capped at what the
 *       kernel's registers allow (0: that maximum).
 * n_reads is rounded up to whole rounds of the grid.  The XOR of what was read
 * lands in *sink (device uint32) so nothing is optimised away.
 * buf_bytes >= 64.  *resident_blocks_per_sm and *reads_done (host, either may
 * be NULL) receive the blocks per SM launched and the number of 32-byte
 * sectors the launch reads.
 */
grape_status_t grape_sector_probe(const void* buf, int64_t buf_bytes, int64_t n_reads,
                                  uint64_t seed, int32_t mode, int32_t load_bytes,
                                  int32_t loads_in_flight, int32_t blocks_per_sm, uint32_t* sink,
                                  int32_t* resident_blocks_per_sm, int64_t* reads_done,
                                  grape_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GRAPE_WALK_H */
