/*
 * libeic — single-source shortest paths on undirected graphs with positive
 * integer weights by the EIC heuristic method of Yu, Wang and Luo, "A
 * Heuristic Algorithm for Shortest Path Search" (arXiv 2506.19349), on one
 * NVIDIA GB300 (sm_103a).
 *
 * Plain C ABI: no C++ or PyTorch types cross it. Every call returns an int
 * status (EIC_OK or an EIC_E* code); no call aborts, traps or exits the
 * process. Device pointers are CUDA global-memory addresses on the current
 * device; host pointers are ordinary process memory. A "stream" argument is a
 * cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Distances are uint32 with +infinity = EIC_INF (0xFFFFFFFF), the paper's
 * "+inf" for unreachable vertices (Section 2). Results are exact: dist[v] is
 * lsp(s, v), the length of the shortest path, identical to Dijkstra's.
 */
#ifndef EIC_H
#define EIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EIC_INF 0xFFFFFFFFu
#define EIC_RATIO_NUM 4096 /* entries of the RtoW weight-quantile table (Section 4.1) */

/* Status codes. */
#define EIC_OK 0
#define EIC_EINVAL 1    /* bad argument: NULL pointer, vertex id >= n, weight 0, size limit */
#define EIC_ENOMEM 2    /* device or host allocation failed, or a fixed capacity was exceeded */
#define EIC_ECUDA 3     /* a CUDA runtime call failed (no device, launch error, ...) */
#define EIC_EOVERFLOW 4 /* the largest shortest distance plus the largest weight reaches 2^32-1 */
#define EIC_ETIMEOUT 5  /* a bounded device-side wait (grid barrier) ran out; the context stays usable */
#define EIC_EBUSY 6     /* the object is in use by another call */
#define EIC_ESIZE 7     /* the graph exceeds the fixed limits of eic_sssp_noalloc */
#define EIC_EABORT 8    /* batch: not run to the end, every block group stopped at an earlier error */

/* Opaque, device-resident graph owned by the library (create/destroy). */
typedef struct eic_graph eic_graph;

/* Tunable parameters. eic_params_default() fills the paper's settings
 * (Section 4.1): alpha = 3, beta = 0.9, ST_NUM = 1024; RATIO_NUM is fixed at
 * EIC_RATIO_NUM when the graph is created.
 *   alpha, beta   Eq. 1-3 constants (beta in (0, 1)).
 *   st_num        size of the Function 2 candidate grid (Section 4.1), in
 *                 [1, 65536].
 *   gap_shift     step-width multiplier 2^gap_shift applied to Eq. 3's gap
 *                 (0 = the paper; any value keeps distances exact).
 *   block_threads threads per block of the relaxation kernel (0 = library
 *                 choice; else a multiple of 32 in [128, 512]).
 *   heavy_min     window length above which a vertex's edges are cut into
 *                 64-entry tasks spread over the whole grid instead of being
 *                 relaxed by one warp (0 = library choice, 32; else 16..4096).
 *   max_spin_log2 bound on each grid-barrier wait, 2^max_spin_log2 polls of
 *                 about 100 ns (0 = library choice, about 2 s); exceeding it
 *                 returns EIC_ETIMEOUT.
 *   flags         EIC_FLAG_* bits.
 *   batch_groups  batches only: number of block groups that run queries at
 *                 the same time (0 = library choice from the graph sizes;
 *                 capped by the number of queries, the co-resident blocks and
 *                 free device memory). */
typedef struct {
  uint32_t alpha;
  double beta;
  uint32_t st_num;
  uint32_t gap_shift;
  uint32_t block_threads;
  uint32_t heavy_min;
  uint32_t max_spin_log2;
  uint32_t flags;
  uint32_t batch_groups;
  uint32_t reserved[7];
} eic_params;

#define EIC_FLAG_NO_PULL 1u /* force st = lb (disable traversal optimisation; still exact) */
#define EIC_FLAG_NO_FUSE 2u /* no fused rounds (bucket fusion): every round of a step is a grid-wide round */

/* Per-step trace row: the thresholds a step ran with and the statistics of
 * Section 3 that produced them. */
typedef struct {
  int64_t lb, ub, st;  /* step window [lb, ub) and selection threshold st; step 1 reports its final ub */
  int64_t gap_lb;      /* gap(lb) of Eq. 3 */
  uint64_t sumd_lb;    /* sumD(lb): total degree of {v : lsp(s, v) >= lb} */
  uint64_t highd_lb;   /* highD(lb) */
  uint64_t rounds;     /* relaxation rounds (synchronisations) in the step */
  uint64_t settled;    /* vertices whose distance fell in [lb, ub) */
  uint32_t flags;      /* EIC_STEP_* : how the step's first round was formed */
  uint32_t reserved;
} eic_step;

#define EIC_STEP_PULL 1u  /* Function 1's pull ran (st < lb) */
#define EIC_STEP_SWEPT 2u /* ... over the unsettled vertices in vertex order (its set held >= half of them) */

/* Counters of one query (Section 4: nSync, nFrontier, nTrav before
 * normalisation). trace/trace_cap are inputs: when trace is a host array of
 * trace_cap rows, up to trace_cap rows are written and trace_len reports the
 * number of steps. */
typedef struct {
  uint64_t steps;
  uint64_t rounds;     /* nSync */
  uint64_t frontier;   /* vertices relaxed from (nFrontier, leaves excluded) */
  uint64_t traversed;  /* nTrav: window entries relaxed plus pull requests */
  uint64_t pulls;      /* pull requests (entries examined by Function 1's pull) */
  uint64_t improved;   /* successful relaxations */
  uint64_t heavy;      /* 64-entry tasks spread over the grid */
  uint64_t pull_items; /* unsettled vertices whose light prefix a pull read */
  eic_step* trace;
  uint64_t trace_cap;
  uint64_t trace_len;
  /* Diagnostic timeline: when timeline is a host array of 2 * timeline_cap
   * uint64, it receives (device globaltimer ns, tag) pairs: one per grid
   * barrier and around each step-boundary evaluation. tag = kind << 32 |
   * round id, kind 0 kernel start, 1 round, 2 heavy phase, 3 step, 4/5
   * step-boundary begin/end; kind 8 and 9 carry the round's item and task
   * counts in place of the round id. */
  uint64_t* timeline;
  uint64_t timeline_cap;
  uint64_t timeline_len;
  /* Device time of the query kernel alone (the persistent relaxation launch,
   * without the setup memsets and the output pass), from CUDA events recorded
   * around its launch on the call's stream. */
  double kernel_ms;
} eic_stats;

/* Fill *p with the paper's defaults (Section 4.1). Returns EIC_EINVAL if p is NULL. */
int eic_params_default(eic_params* p);

/* Human-readable text for a status code (static storage, never NULL). */
const char* eic_strerror(int status);

/* Library version as major*10000 + minor*100 + patch. */
int eic_version(void);

/*
 * Build a device graph from num_tuples raw undirected tuples (src[i], dst[i],
 * w[i]) over vertices 0..num_vertices-1 (preprocessing of Section 4.1).
 * Self-loops are dropped, a pair given several times keeps its smallest
 * weight, every pair is stored in both directions, each vertex's neighbours
 * are sorted by (weight, neighbour), and the weight quantile table RtoW and
 * the degree statistics are computed on the device.
 *   src, dst, w    arrays of num_tuples uint32; device pointers when
 *                  ptrs_on_device != 0, else host pointers. Caller-owned,
 *                  read only, copied; may be freed when the call returns.
 *   num_vertices   n >= 1, n < 2^32 - 1.
 *   stream         work is enqueued here; the call synchronises it before
 *                  returning.
 *   out            receives the new graph (NULL on failure).
 * Errors: EIC_EINVAL (NULL pointer, endpoint >= n, weight 0, n out of
 * range, num_tuples >= 2^31 directed entries per 2), EIC_ENOMEM, EIC_ECUDA.
 */
int eic_graph_create(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t num_tuples,
                     uint32_t num_vertices, int ptrs_on_device, void* stream, eic_graph** out);

/* Graph facts: vertex count, undirected edge count m (after dedup), largest
 * degree, largest and smallest weight, highD(0). Any output may be NULL. */
int eic_graph_info(const eic_graph* g, uint32_t* n, uint64_t* m, uint32_t* max_deg, uint32_t* max_w,
                   uint32_t* min_w, uint32_t* highd0);

/* Copy the CSR to host arrays: row_ptr[n+1] (uint64), nbr[2m], w[2m]; and
 * RtoW[EIC_RATIO_NUM] when rtow is non-NULL. Any array may be NULL. */
int eic_graph_export(const eic_graph* g, uint64_t* row_ptr, uint32_t* nbr, uint32_t* w, uint32_t* rtow);

/* Copy the CSR as the queries read it on the device, in internal vertex ids
 * 0..ni-1 (the vertices of degree >= 1 ordered by degree descending, then
 * original id): *ni = ni; int2orig[ni] maps an internal id to the caller's id;
 * row[ni+1] (uint32) row offsets; nbr[2m] internal neighbour ids and w[2m]
 * weights, each row sorted by (weight, the neighbour's original id): the
 * weight order is what the window searches of the relaxation rely on
 * (Section 4.1 sorts rows by weight). Any output may be NULL; host arrays,
 * caller-owned. */
int eic_graph_export_internal(const eic_graph* g, uint32_t* ni, uint32_t* int2orig, uint32_t* row, uint32_t* nbr,
                              uint32_t* w);

/* Device bytes held by the graph and by its query workspace. */
int eic_graph_memory(const eic_graph* g, uint64_t* graph_bytes, uint64_t* workspace_bytes);

/* Free the graph and its workspace. NULL is accepted. Must not race a query
 * on the same graph. */
int eic_graph_destroy(eic_graph* g);

/*
 * One single-source query by Algorithm 1 (dynamic stepping, Eq. 1-3;
 * traversal optimisation, Function 1/2), exact distances.
 *   source   0 <= source < n.
 *   dist     array of n uint32, caller-owned; receives lsp(source, v) or
 *            EIC_INF. Device memory of the graph's GPU, managed memory, or
 *            page-locked host memory mapped for the device (cudaHostAlloc,
 *            or cudaHostRegister with a device mapping): the output kernel
 *            then writes the host array directly across the host link, so
 *            the result is in host memory when the call returns. Any other
 *            pointer (pageable host memory, another GPU's memory) is
 *            rejected with EIC_EINVAL before anything is launched.
 *   parent   NULL, or an array of n uint32 with the same rules as dist;
 *            receives the smallest-id u with dist[u] + w(u, v) == dist[v]
 *            (parent[source] = source, EIC_INF where unreachable).
 *   params   NULL for eic_params_default().
 *   stats    NULL, or a host struct that receives the counters (and the
 *            trace rows when stats->trace is set).
 *   stream   the work is enqueued on it; the call synchronises the stream
 *            before returning the status.
 * The graph's workspace is allocated on first use (device memory about 30
 * bytes per vertex plus the heavy-window and step tables); concurrent calls
 * on one graph are serialised.
 * Errors: EIC_EINVAL, EIC_ENOMEM, EIC_ECUDA, EIC_EOVERFLOW (dist is then
 * unspecified), EIC_ETIMEOUT.
 */
int eic_sssp(const eic_graph* g, uint32_t source, uint32_t* dist, uint32_t* parent, const eic_params* params,
             eic_stats* stats, void* stream);

/*
 * num_queries queries (graphs[i], sources[i]) -> dists[i], with the same
 * results as eic_sssp, in one cooperative persistent launch. The paper runs
 * its trials one after another; this entry point adds query-level
 * parallelism for many sources and many graphs of uneven size. The grid is
 * cut into params->batch_groups groups of blocks (0 = library choice); each
 * group claims the next query from a device work queue (largest graphs
 * first), runs Algorithm 1 for it with its own scratch and a barrier over its
 * own blocks, writes dists[i] and claims again.
 *   graphs, sources   host arrays of num_queries; every graph on the current
 *                     device. A graph may appear many times.
 *   dists             host array of device pointers, one n_i-element uint32
 *                     buffer per query, caller-owned; must not overlap.
 *   statuses          host array of num_queries ints, or NULL; receives each
 *                     query's status.
 * The call reuses a per-device scratch pool (about 40 bytes per vertex plus
 * one byte per adjacency entry of the largest graph, per group; grown when a
 * batch needs more), launches on stream and synchronises it before
 * returning. Returns the first non-OK status in query order, or EIC_OK.
 * A group stops at its first failing query (that query reports the error);
 * the other groups go on with the remaining queries. A query that no group
 * finished reports EIC_EABORT.
 * Errors: EIC_EINVAL, EIC_ENOMEM, EIC_ECUDA, and per query those of eic_sssp.
 */
int eic_sssp_batch(const eic_graph* const* graphs, const uint32_t* sources, uint32_t num_queries,
                   uint32_t* const* dists, const eic_params* params, int* statuses, void* stream);

/*
 * A prepared batch for repeated runs (the batched form of eic_sssp_batch,
 * replayed as a CUDA graph). It holds its own scratch, query table and
 * status buffers; graphs and dists must stay valid until it is destroyed.
 *
 * eic_batch_create  validates and stores the queries (arguments as in
 *                   eic_sssp_batch), allocates the scratch for the group
 *                   count of params->batch_groups (0 = library choice).
 *                   Synchronous. Errors: EIC_EINVAL, EIC_ENOMEM, EIC_ECUDA.
 * eic_batch_run     enqueues one run of every query on stream and returns
 *                   without waiting. The first run captures the launch
 *                   sequence into a CUDA graph (on a private stream) and
 *                   later runs replay it; where capture is unavailable the
 *                   kernels are launched directly. Runs of one batch must not
 *                   overlap on the GPU.
 * eic_batch_wait    waits for stream, copies each query's status into
 *                   statuses (host array of num_queries, or NULL) and
 *                   returns the first non-OK one.
 * eic_batch_tune    autotuner: runs the whole batch for group counts from
 *                   the most down (divisors of the co-resident grid and
 *                   powers of two) until two in a row are 20% slower than
 *                   the best; then, at the best count, step-width scalings
 *                   gap_shift + 1, + 2, ... while they help (up to 8),
 *                   window-class thresholds heavy_min 64 and 256, and a
 *                   256-thread block. Each configuration gets a warm-up run
 *                   and, when that is within 2x of the best, a timed run
 *                   (CUDA events on stream); the fastest is kept for later
 *                   runs and the scratch shrinks to its group count. Every
 *                   tried configuration computes the same exact distances;
 *                   dists hold a complete result afterwards. best (or NULL)
 *                   receives the chosen configuration. Synchronous.
 * eic_batch_info    the current configuration.
 * eic_batch_gap_shifts  each query's step-width scaling in use (host array
 *                   of num_queries, in the caller's query order; the tuner
 *                   chooses it per graph): the value to give eic_sssp in
 *                   eic_params.gap_shift for the same schedule.
 * eic_batch_destroy frees the batch (NULL accepted); no run may be in flight.
 */
typedef struct eic_batch eic_batch;

typedef struct {
  uint32_t groups;            /* block groups running queries at the same time */
  uint32_t blocks_per_group;
  uint32_t block_threads;
  uint32_t cuda_graph;        /* 1 when runs replay a captured CUDA graph */
  uint32_t gap_shift;         /* step-width scaling in use (eic_params.gap_shift) */
  uint32_t heavy_min;         /* window-class threshold in use (eic_params.heavy_min) */
  uint32_t queries;
  uint32_t reserved;
  uint64_t scratch_bytes;     /* device bytes of the groups' scratch */
  double tuned_ms;            /* fastest run seen by eic_batch_tune, 0 if not tuned */
} eic_batch_config;

int eic_batch_create(const eic_graph* const* graphs, const uint32_t* sources, uint32_t num_queries,
                     uint32_t* const* dists, const eic_params* params, eic_batch** out);
int eic_batch_run(eic_batch* b, void* stream);
int eic_batch_wait(eic_batch* b, void* stream, int* statuses);
int eic_batch_tune(eic_batch* b, void* stream, eic_batch_config* best);
int eic_batch_info(const eic_batch* b, eic_batch_config* out);
int eic_batch_gap_shifts(const eic_batch* b, uint32_t* gap_shifts);
int eic_batch_destroy(eic_batch* b);

/*
 * Serving: a request loop with continuous batching (no counterpart in the
 * paper). Graphs stay resident; (graph, source) requests are submitted at any
 * time and run as soon as a block group of the persistent serving kernel is
 * free, while other requests are in flight. Results are exact and identical
 * to eic_sssp's.
 *
 * Admission: requests are admitted in arrival order while the result-buffer
 * budget (config.output_bytes, a device arena allocated at creation; a result
 * takes 4n bytes, rounded up to 256) and the request ring (config.
 * ring_entries in flight) have room; the rest wait in a host queue. A result's
 * memory returns to the budget at eic_server_release. The serving kernel runs
 * while there is work: after config.idle_us without a request, once no
 * request runs, a block group registers as idle, and when every group is
 * registered they leave together; the runtime relaunches the kernel when
 * requests arrive again. The width of a launch follows the backlog: with at
 * most 4 (8, 16) waiting requests it runs 4 (8, 16) groups that share the
 * co-resident blocks, else config.groups groups; a launch with fewer groups
 * ends (each group after its current request) once twice its group count of
 * admitted requests wait, and the runtime relaunches wider. A lone request
 * thus runs on a quarter of the GPU, not on one small group. Scratch: one
 * slot per group (config.groups slots) sized for the largest resident graph
 * (as a batch's).
 *
 * eic_server_create   graphs (host array of num_graphs, all on one device)
 *                     stay owned by the caller and must outlive the server;
 *                     params as eic_sssp's (NULL = defaults); config may be
 *                     NULL. Starts the runtime's pump thread. Errors:
 *                     EIC_EINVAL, EIC_ENOMEM, EIC_ECUDA.
 * eic_server_submit   enqueues (graph index, source); *ticket identifies it.
 *                     Never blocks. EIC_EINVAL for a bad index or source,
 *                     EIC_ENOMEM if the result cannot fit the whole budget.
 * eic_server_poll     EIC_OK and *status once done; EIC_EBUSY while pending.
 * eic_server_wait     waits up to timeout_ms: EIC_OK and *status once done,
 *                     EIC_ETIMEOUT if still pending.
 * eic_server_result   for a done request: copies the n distances to
 *                     host_dist (if non-NULL), returns the device buffer in
 *                     *device_dist (if non-NULL; valid until release) and the
 *                     latency from submit to completion in *latency_ms. Returns
 *                     the request's status (EIC_EBUSY while pending).
 * eic_server_release  forgets a done request and frees its result buffer.
 * eic_server_stats    counters and the latency percentiles of the requests
 *                     completed since creation or the last reset.
 * eic_server_tune     autotuner for the resident graphs: for each graph k it
 *                     picks the step-width scaling (gap_shift, exact for every
 *                     value) that runs sample_sources[k] fastest in one of the
 *                     server's block groups, trying params->gap_shift + 0, 1,
 *                     2, ... while the time falls by 2% (up to 8); one copy of
 *                     the sample runs per group and each setting is timed
 *                     twice. gap_shifts (host array of num_graphs, or NULL)
 *                     receives the choices. The server must be idle (nothing
 *                     queued or in flight: EIC_EBUSY otherwise); submissions
 *                     wait until it returns. Synchronous.
 * eic_server_destroy  stops the kernel and the pump; pending requests are
 *                     dropped. NULL accepted.
 */
typedef struct eic_server eic_server;

typedef struct {
  uint32_t groups;        /* block groups serving at the same time (0 = about 8 blocks per group) */
  uint32_t ring_entries;  /* admitted requests in flight at most, a power of two (0 = 1024) */
  uint64_t output_bytes;  /* device budget for result buffers (0 = 64 results of the largest graph) */
  uint32_t idle_us;       /* idle time before a block group registers as idle (0 = 2000, at most 100000) */
  uint32_t reserved[5];
} eic_server_config;

typedef struct {
  uint64_t submitted, admitted, completed, queued, in_flight, max_in_flight;
  uint64_t kernel_launches;
  uint64_t output_bytes_used, output_bytes, scratch_bytes;
  uint32_t groups, blocks_per_group;
  double latency_p50_ms, latency_p99_ms, latency_mean_ms;  /* submit to completion */
  uint64_t latency_count;
} eic_server_report;

int eic_server_create(const eic_graph* const* graphs, uint32_t num_graphs, const eic_params* params,
                      const eic_server_config* config, eic_server** out);
int eic_server_submit(eic_server* s, uint32_t graph, uint32_t source, uint64_t* ticket);
int eic_server_poll(eic_server* s, uint64_t ticket, int* status);
int eic_server_wait(eic_server* s, uint64_t ticket, uint32_t timeout_ms, int* status);
int eic_server_result(eic_server* s, uint64_t ticket, uint32_t* host_dist, const uint32_t** device_dist,
                      double* latency_ms);
int eic_server_release(eic_server* s, uint64_t ticket);
int eic_server_stats(eic_server* s, eic_server_report* out);
int eic_server_reset_stats(eic_server* s);
int eic_server_tune(eic_server* s, const uint32_t* sample_sources, uint32_t* gap_shifts);
int eic_server_destroy(eic_server* s);

/*
 * Allocation-free single-source query. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc at query time,
 * for example a serving process that plans its whole device-memory budget up
 * front and treats any allocation as a failure, code running inside another
 * framework's memory pool, or a latency-critical loop that cannot afford
 * cudaMalloc's implicit device synchronisation.
 *
 * Same result as eic_sssp (exact distances, paper's default parameters), but
 * the query's scratch (frontier queues, settled list, statistics, tasks,
 * control block) lives in one fixed-size device array inside libeic instead of
 * the graph's workspace. That array (about 13.4 MB) is held on every GPU where
 * the library is loaded, until the process exits. The call allocates nothing:
 * no cudaMalloc, cudaFree or allocating library routine; the caller supplies
 * the graph (created beforehand with eic_graph_create) and the output buffer.
 *   source   0 <= source < n.
 *   dist     device array of n uint32, caller-owned.
 *   stream   the work is enqueued here; the call waits for it to finish.
 * Limits: n <= EIC_NOALLOC_MAX_VERTICES, 2m <= EIC_NOALLOC_MAX_ENTRIES,
 * largest weight <= EIC_NOALLOC_MAX_WEIGHT, at most EIC_NOALLOC_MAX_DEGREES
 * distinct degrees; a larger graph returns EIC_ESIZE. A query needing more than
 * EIC_NOALLOC_MAX_STEPS steps returns EIC_ENOMEM.
 * The first call on a device sets up that device (looks up the scratch
 * address and clears it); make that first call before any stream capture.
 * Every call uses the same scratch, which keeps the previous call's contents
 * (the call clears what must start at zero): calls whose work overlaps on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.
 * Errors: EIC_EINVAL, EIC_ESIZE, EIC_ECUDA, EIC_EOVERFLOW, EIC_ETIMEOUT,
 * EIC_ENOMEM (step limit).
 */
#define EIC_NOALLOC_MAX_VERTICES (1u << 18)
#define EIC_NOALLOC_MAX_ENTRIES (1u << 22)
#define EIC_NOALLOC_MAX_WEIGHT 65535u
#define EIC_NOALLOC_MAX_DEGREES 4096u
#define EIC_NOALLOC_MAX_STEPS (1u << 14)
int eic_sssp_noalloc(const eic_graph* g, uint32_t source, uint32_t* dist, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* EIC_H */
