/*
 * dfpr.h - Dynamic Frontier PageRank on one GPU (sm_103a), C ABI.
 *
 * The library keeps a directed graph resident in device memory, applies
 * batches of edge deletions and insertions to it, and updates the PageRank
 * vector incrementally with the Dynamic Frontier (DF) approach of
 * arXiv 2407.19562 ("Lock-Free Computation of PageRank in Dynamic Graphs"):
 * after a batch, the out-neighbours of every changed edge's source are marked
 * affected (Sec. 4.1), their ranks are recomputed from their in-edges with
 * Eq. 1, and any vertex whose rank moves by more than the frontier tolerance
 * marks its own out-neighbours (Sec. 4.1, Alg. 1, Alg. 2), until every rank
 * moves by at most the iteration tolerance.
 *
 * Conventions for every entry point:
 *  - Vertex ids are int32 in [0, n). Edge counts and offsets are int64.
 *  - Size limits: a graph (or a set) holds at most 2^32 - 2 edges, self-loops
 *    included, since edge keys are counted with 32-bit prefix sums
 *    (dfpr_graph_load and dfpr_apply_batch return EINVAL beyond it). The
 *    update calls (static, ND, DF, autotune) need every in- and out-degree at
 *    most 2^25 - 1, since a warp adds the degrees of its 32 rows in 32-bit
 *    integers; they return EINVAL otherwise. Degrees are tracked only when n
 *    exceeds 2^25 - 1 (a degree never exceeds n).
 *  - Pointer arguments marked "host or device" are host pointers when
 *    on_device == 0 and device pointers of the graph's device when
 *    on_device != 0. The library copies inputs before returning; the caller
 *    keeps ownership of every array it passes.
 *  - The library owns all graph, rank and scratch memory. It allocates with
 *    cudaMalloc unless an allocator was installed with dfpr_set_allocator.
 *  - Work is issued on the graph's stream (given to dfpr_graph_load or
 *    dfpr_graph_set_stream). Calls that return counts or statuses to the host
 *    synchronise that stream before returning. Calls on one graph must not
 *    overlap; distinct graphs may be used from distinct host threads.
 *  - No entry point aborts, traps or exits. Failures return a status code and
 *    leave a message for dfpr_last_error() (thread-local). A graph on which a
 *    call failed with DFPR_ECUDA should be freed.
 */
#ifndef DFPR_H
#define DFPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dfpr_graph dfpr_graph; /* opaque, owned by the library */

typedef enum dfpr_status {
  DFPR_OK = 0,
  DFPR_EINVAL = 1,   /* bad argument: null pointer, id outside [0, n), bad size */
  DFPR_ENOMEM = 2,   /* device or host allocation failed */
  DFPR_ECUDA = 3,    /* a CUDA call failed; the message names it */
  DFPR_ENOTCONV = 4, /* the iteration cap was reached before convergence */
  DFPR_ETIMEOUT = 5, /* the time budget ran out; ranks are valid but unconverged */
  DFPR_EBUSY = 6     /* another call on this graph is in progress */
} dfpr_status;

/* Rank storage and arithmetic. */
enum {
  DFPR_FP64 = 0, /* ranks and gather in FP64, as in the paper (Sec. 5.1.2) */
  DFPR_FP32 = 1  /* ranks in FP32, compensated per-vertex sums, FP64 reductions */
};

/* Dead-end handling. */
enum {
  DFPR_SELF_LOOPS = 0, /* a self-loop on every vertex, kept through every batch
                          (Sec. 5.1.3, Sec. 5.1.4); deleting a self-loop is a no-op */
  DFPR_TELEPORT = 1    /* no self-loops added; the rank of dead ends is spread
                          uniformly (alpha * D / n added to every vertex, D the
                          FP64 sum of dead-end ranks, recomputed every
                          iteration). Jacobi schedule only. In a DF update the
                          frontier rule covers the shared term: when D differs
                          by more than tol_f * n / alpha from the D that the
                          unaffected ranks were computed with (taken by the
                          first dfpr_apply_batch after the ranks were computed
                          or set), every vertex is recomputed from then on.
                          This is a reading; the paper's runs use self-loops
                          (Sec. 5.1.3). */
};

/* Schedules of the rank iteration. */
enum {
  DFPR_MODE_WORKLIST = 0, /* persistent kernel fed by a device work queue: only
                             vertices flagged not-converged are recomputed,
                             in place, with no grid-wide barrier */
  DFPR_MODE_ROUND = 1,    /* Alg. 2 schedule: every affected vertex is recomputed
                             in each pass, in place, chunks claimed dynamically
                             per pass, no grid-wide barrier */
  DFPR_MODE_JACOBI = 2    /* Alg. 1 / Alg. 3 schedule: two rank vectors and an
                             L-inf reduction per iteration (barrier-based) */
};

/* Graph options fixed at load time. */
typedef struct dfpr_graph_config {
  int32_t precision;  /* DFPR_FP64 (default) or DFPR_FP32 */
  int32_t dead_end;   /* DFPR_SELF_LOOPS (default) or DFPR_TELEPORT */
  double row_slack;   /* extra capacity per row as a fraction of its degree, so
                         batches update rows in place (default 0.125) */
  int32_t min_slack;  /* minimum extra capacity per row (default 2) */
  int32_t reorder;    /* 1 (default): number vertices internally by decreasing degree,
                         so that frequently read ranks share memory sectors; ids at the
                         interface stay the caller's. 0: keep the caller's numbering */
  double tail_slack;  /* spare edge capacity for rows that outgrow their slot,
                         as a fraction of the edge count (default 0.125) */
} dfpr_graph_config;

/* Parameters of one rank computation (defaults: the paper's, Sec. 5.1.2, 4.5). */
typedef struct dfpr_params {
  double alpha;        /* damping factor (0.85) */
  double tol;          /* iteration tolerance tau, per-vertex change (1e-10);
                          in FP32 mode a relative tolerance (change <= tol * R[v]) */
  double frontier_tol; /* frontier tolerance tau_f; <= 0 selects tol / 1000 (Sec. 4.5);
                          relative in FP32 mode */
  int32_t max_iter;    /* MAX_ITERATIONS (500): iterations or passes; in worklist
                          mode the cap is max_iter * n recomputations in total */
  int32_t mode;        /* DFPR_MODE_* */
  int32_t normalize;   /* 1: rescale ranks to sum 1 (FP64 sum) after convergence */
  int32_t grid_ctas;   /* persistent grid size; 0 = the schedule's own: worklist about
                          sqrt(n)/4 CTAs (at least 8, at most 4 per SM and one wave),
                          round at most n/2048, jacobi one wave */
  double timeout_ms;   /* wall-clock budget on the device; <= 0 means 60000 */
  /* Simulated faults (Sec. 5.1.6; experiments of Sec. 5.3 and 5.4). All 0 by
     default. A warp stands for one of the paper's threads; every draw comes
     from a counter-based hash of fault_seed, so a run is reproducible.
     - Thread delay: after a warp finishes the rank computation of a batch of
       vertices, it sleeps fault_delay_us microseconds with probability
       1 - (1 - fault_delay_prob)^k, k = the vertices in the batch, i.e.
       fault_delay_prob per vertex. The sleep is a bounded loop of
       __nanosleep that also ends when timeout_ms runs out.
     - Crash-stop: fault_crash_warps warps of the launch (chosen by the hash)
       stop taking part at a random batch boundary, without finishing any
       bookkeeping, like a thread that never runs again. The round schedule
       (Alg. 2) finishes without them: its passes and R_C flags let the
       other warps recompute what they left. The worklist schedule finishes
       without them too while helping is on (see helping below): idle warps
       return a crashed warp's claimed vertices to the queue. With helping
       off, the crashed warp's claim keeps the global count of open work
       unbalanced, so the call stops at timeout_ms with DFPR_ETIMEOUT
       (valid, partly updated ranks). The jacobi schedule rejects crashes
       with DFPR_EINVAL: its iteration barrier could never complete
       (Sec. 5.4).
     Limits: 0 <= fault_delay_prob <= 1, 0 <= fault_delay_us <= 1e6,
     0 <= fault_crash_warps < the warps of the launch. */
  double fault_delay_prob;
  double fault_delay_us;
  int32_t fault_crash_warps;
  uint32_t fault_seed;
  /* Degree classes: an in-row longer than gather_split edges is summed as
     gather_split-edge tokens that any warp takes (worklist and round
     schedules; the jacobi schedule sums such rows in gather_split-edge
     chunks, 2048 by default, spread over every warp after each iteration's
     shorter rows), and
     an out-row longer than mark_split edges is marked the
     same way (worklist schedule); shorter rows are gathered and marked by one
     warp, edge-balanced over its 32 vertices. 0 selects the defaults (4096
     and 8192); otherwise max(256, edges / 2^20) <= value <= 2^24, so that
     the tokens of a launch fit the device's token ring (2^21 entries).
     dfpr_autotune picks them by timing. */
  int32_t gather_split;
  int32_t mark_split;
  /* Helping (worklist schedule; Sec. 4.4: threads help each other so that a
     slow or crashed thread does not hold up the rest). 1 (the default): every
     warp publishes the vertices it claims, and an idle warp that sees the same
     claim unchanged in two of its scans at least 10 ms apart returns those
     vertices to the queue, so a crash-stopped warp's work is done by the
     others. 0: off; a crashed warp's claim then keeps the update open until
     timeout_ms. Other schedules ignore it. */
  int32_t helping;
} dfpr_params;

/* Counters of one call. */
typedef struct dfpr_stats {
  int64_t processed;      /* vertex rank recomputations */
  int64_t edges_gathered; /* in-edges read by those recomputations */
  int64_t expansions;     /* recomputations that marked their out-neighbours */
  int64_t edges_marked;   /* out-edges visited by marking and expansion */
  int64_t pushes;         /* work-queue insertions (worklist mode) */
  int64_t affected;       /* distinct vertices recomputed at least once */
  int32_t passes;         /* iterations (jacobi) or passes (round); 0 for worklist */
  int32_t status;         /* dfpr_status of the call */
  double residual_linf;   /* jacobi: last L-inf iterate difference; worklist and round:
                             the largest change of one recomputation in the call (not a
                             residual; dfpr_residual gives max_v |Eq. 1 (v) - R[v]|) */
  double rank_sum;        /* FP64 sum of the ranks after the call when normalize = 1,
                             else NaN */
  double ms;              /* device time (CUDA events): the persistent kernel alone in
                             worklist mode, all kernels of the call otherwise */
  int64_t batches;        /* worklist: batches of up to 32 vertices taken from the queue */
  int64_t tokens;         /* worklist: chunk tokens processed (pieces of long rows) */
  int64_t jobs;           /* worklist: recomputations whose in-row was split into tokens */
  int64_t phase_cycles[5];/* worklist: SM cycles summed over warps spent idle (queue empty),
                             claiming items, gathering, marking out-neighbours, and
                             finishing (state updates, queue insertions) */
} dfpr_stats;

/* Fills *cfg / *p with the defaults listed above. */
void dfpr_default_config(dfpr_graph_config* cfg);
void dfpr_default_params(dfpr_params* p);

/*
 * Builds the snapshot G^0 from m raw edges src[i] -> dst[i] (host or device;
 * duplicates allowed; ids in [0, n)): out-rows (CSR) and in-rows (CSC) with
 * sorted unique rows, self-loops added under DFPR_SELF_LOOPS (Sec. 5.1.3).
 * Ranks start at 1/n (Sec. 3.1). cuda_stream is a cudaStream_t (NULL: the
 * library creates one). cfg NULL selects the defaults. On success *out owns
 * the graph until dfpr_graph_free. Errors: EINVAL (n <= 0, m < 0, null
 * arrays with m > 0, more than 2^32 - 2 edges with the self-loops, an id out
 * of range; the size check comes before the arrays are read), ENOMEM, ECUDA.
 */
dfpr_status dfpr_graph_load(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            int on_device, void* cuda_stream, const dfpr_graph_config* cfg,
                            dfpr_graph** out);

/*
 * Loads k independent graphs as one device-resident set (a disjoint union):
 * graph i owns the global vertex ids [vertex_offsets[i], vertex_offsets[i+1])
 * (host array of k + 1 entries, vertex_offsets[0] = 0, nondecreasing, each
 * graph non-empty), and src/dst (host or device, m entries) use global ids.
 * An edge joining two graphs is an error (EINVAL). Eq. 1 (Sec. 3.1) is
 * applied per graph: the teleport term of a vertex is (1 - alpha) / n_i of
 * its own graph, and static ranks start at 1 / n_i. Every later call works on
 * all graphs at once: one dfpr_apply_batch takes the batches of every graph
 * (global ids) and one dfpr_df_pagerank runs all their frontiers in a single
 * persistent launch. Not supported with DFPR_TELEPORT or normalize = 1.
 */
dfpr_status dfpr_graph_load_parts(int32_t k, const int32_t* vertex_offsets, int64_t m,
                                  const int32_t* src, const int32_t* dst, int on_device,
                                  void* cuda_stream, const dfpr_graph_config* cfg,
                                  dfpr_graph** out);

/* Number of graphs in the set (1 for dfpr_graph_load). */
dfpr_status dfpr_graph_parts(const dfpr_graph* g, int32_t* k);

/*
 * Per-graph completion times of the last worklist update, in ms after its
 * persistent kernel started (host array of k doubles): the time the last
 * recomputation of a vertex of graph i ended, 0 when graph i had no work.
 */
dfpr_status dfpr_get_part_times(const dfpr_graph* g, double* ms);

/* Releases every device and host resource of g (NULL is a no-op). Returns
   EBUSY, and frees nothing, while another call on g is in progress. */
dfpr_status dfpr_graph_free(dfpr_graph* g);

/* Makes later calls on g issue their work on cuda_stream (a cudaStream_t; NULL:
   a new stream of the library's). A stream the library created is kept until
   dfpr_graph_free, since arrays allocated on it may name it when released. */
dfpr_status dfpr_graph_set_stream(dfpr_graph* g, void* cuda_stream);

/* n, current edge count m (self-loops included) and device id of g. */
dfpr_status dfpr_graph_info(const dfpr_graph* g, int32_t* n, int64_t* m, int32_t* device);

/*
 * Applies a batch update (Sec. 3.4): G^t = (G^{t-1} minus deletions) plus
 * insertions, deletions taken first. Duplicate entries collapse; deleting an
 * absent edge, inserting a present edge and (DFPR_SELF_LOOPS) deleting a
 * self-loop are no-ops, not errors. Rows stay sorted and unique. The real
 * changes Delta- = E^{t-1} \ E^t and Delta+ = E^t \ E^{t-1} are kept for the
 * next dfpr_df_pagerank, which marks the out-neighbours of their sources
 * (Sec. 4.1). n_applied (host, may be NULL) receives {|Delta-|, |Delta+|}.
 * Arrays are host or device. Applying a second batch before dfpr_df_pagerank
 * merges both into the pending change set. Errors: EINVAL (an id out of range,
 * or n_del + n_ins or the graph's edges plus n_ins above 2^32 - 2; the graph
 * is left unchanged), ENOMEM, ECUDA, EBUSY.
 */
dfpr_status dfpr_apply_batch(dfpr_graph* g, int64_t n_del, const int32_t* del_src,
                             const int32_t* del_dst, int64_t n_ins, const int32_t* ins_src,
                             const int32_t* ins_dst, int on_device, int64_t* n_applied);

/*
 * Dynamic Frontier update (Sec. 4; Alg. 1 for DFPR_MODE_JACOBI, Alg. 2 for
 * DFPR_MODE_ROUND, the work-queue schedule for DFPR_MODE_WORKLIST): starting
 * from the current ranks R^{t-1}, marks the affected vertices of the pending
 * change set and iterates Eq. 1 over them until convergence, in place. Clears
 * the pending change set. A recomputed vertex marks its out-neighbours when
 * its rank moved by more than tau_f (Alg. 1, Alg. 2). The worklist schedule
 * recomputes only marked vertices, so there a vertex also marks them once its
 * rank has drifted by more than 10 tau_f since it last did (in FP32 mode:
 * by more than tau_f, the only rule), which bounds what a dependant misses.
 * With no pending changes it returns at once with 0 recomputations. p NULL
 * selects the defaults; stats may be NULL.
 * Returns ENOTCONV / ETIMEOUT when the cap / budget stopped the iteration
 * (ranks are then valid but not converged), EINVAL for bad parameters or a
 * vertex whose in- or out-degree exceeds 2^25 - 1 (ranks untouched).
 */
dfpr_status dfpr_df_pagerank(dfpr_graph* g, const dfpr_params* p, dfpr_stats* stats);

/*
 * Autotuner of the degree-class boundaries (no counterpart in the paper):
 * runs the pending update once per candidate (gather_split, mark_split) pair,
 * each time from the same ranks and the same pending change set, times the
 * rank kernel of each trial with CUDA events, then restores that state once
 * more and runs the update with the fastest pair, which stays applied.
 * Cost: n_candidates + 1 updates.
 * p: in, the parameters of every trial (worklist or round mode); out, the
 * same with gather_split / mark_split set to the chosen pair.
 * candidates: host, 2 * n_candidates int32 (gather_split, mark_split pairs),
 * or NULL for the built-in set {(2048, 2048), (4096, 8192), (8192, 8192),
 * (16384, 16384)} (n_candidates is then ignored).
 * trial_ms: host, n_candidates doubles (may be NULL): the rank kernel time
 * of each trial; a trial that did not converge gets +inf.
 * stats (may be NULL): the final update's counters.
 * Errors: EINVAL (no pending changes, jacobi mode, bad pair), ENOMEM (no room
 * for the ranks' snapshot), ECUDA, EBUSY; otherwise the final update's status.
 */
dfpr_status dfpr_autotune(dfpr_graph* g, dfpr_params* p, int32_t n_candidates,
                          const int32_t* candidates, double* trial_ms, dfpr_stats* stats);

/*
 * Naive-dynamic update (Sec. 3.5.1; Alg. 5 / Alg. 6): iterates Eq. 1 over
 * every vertex starting from the current ranks. Clears the pending change set.
 */
dfpr_status dfpr_nd_pagerank(dfpr_graph* g, const dfpr_params* p, dfpr_stats* stats);

/*
 * Static PageRank (Sec. 3.3; Alg. 3 / Alg. 4): resets every rank to 1/n and
 * iterates Eq. 1 over every vertex until convergence. Clears the pending
 * change set.
 */
dfpr_status dfpr_static_pagerank(dfpr_graph* g, const dfpr_params* p, dfpr_stats* stats);

/* Copies the n ranks out as FP64 (host or device; FP32 ranks are widened),
 * in the caller's vertex numbering. out: n doubles, caller-owned; on_device
 * 1: a device pointer on the graph's device, 0: host memory. Page-locked
 * host memory the device can address (cudaMallocHost, cudaHostAlloc, mapped
 * registrations) is written directly by the device; other host memory goes
 * through a device staging vector of n doubles that the graph keeps after
 * the first such call. Returns when the ranks are in `out`. Errors: EINVAL
 * (NULL argument), EBUSY, ECUDA. */
dfpr_status dfpr_get_ranks(const dfpr_graph* g, double* out, int on_device);

/* Replaces the n ranks (host or device FP64), e.g. to resume from saved ranks. */
dfpr_status dfpr_set_ranks(dfpr_graph* g, const double* ranks, int on_device);

/*
 * Copies the graph out in packed form (host or device): offsets[n + 1]
 * (int64) and idx[m] (int32); out-rows (CSR) for dfpr_get_csr, in-rows (CSC)
 * for dfpr_get_csc. Rows are sorted ascending; self-loops included.
 */
dfpr_status dfpr_get_csr(const dfpr_graph* g, int64_t* offsets, int32_t* idx, int on_device);
dfpr_status dfpr_get_csc(const dfpr_graph* g, int64_t* offsets, int32_t* idx, int on_device);

/*
 * Initial marking of the DF approach (Sec. 4.1; Alg. 1 and Alg. 2 marking
 * loops) for the pending change set, without updating ranks or clearing the
 * set: affected[v] (n bytes, host or device) is 1 when v is an out-neighbour,
 * in G^{t-1} or G^t, of the source of a real change (with self-loops, the
 * source itself). Returns the count in *count (host, may be NULL).
 */
dfpr_status dfpr_initial_affected(dfpr_graph* g, uint8_t* affected, int on_device,
                                  int64_t* count);

/*
 * Serving with continuous batching. A server keeps one or more units resident
 * (a unit is a graph, or a set of graphs from dfpr_graph_load_parts) and
 * serves update requests: each request is one batch of edge deletions and
 * insertions for one graph. Every unit has its own worker thread and uses its
 * own stream (load the units with distinct streams, e.g. cuda_stream NULL, for
 * their launches to overlap). A unit's worker admits the unit's queued
 * requests in arrival order whenever the unit is idle, a slot is free (at most
 * max_slots requests are in flight over the whole server) and their batch
 * memory fits in mem_fraction of the device's free memory minus what earlier
 * admissions hold (with nothing else in flight one request is always
 * admitted); it applies them (requests for the same graph in arrival order)
 * and updates the unit with one dfpr_df_pagerank call, i.e. one persistent
 * launch for all admitted requests of the unit. So a request for an idle unit
 * starts at once, even while other units' updates run on the GPU, and their
 * work overlaps on the device. A unit never changes while its own update
 * reads it (read-only snapshot, Sec. 3.4): requests arriving for a busy unit
 * join its next update. While the server exists, other calls on its units
 * return DFPR_EBUSY; dfpr_server_drain waits until it is idle. Times are host
 * monotonic-clock ms since the server was created.
 */
typedef struct dfpr_server dfpr_server;

typedef struct dfpr_request_info {
  int32_t status;         /* dfpr_status of the update that served it */
  int32_t cycle_requests; /* requests served by the same update */
  int64_t cycle;          /* index of that update (numbered over the server) */
  double submit_ms;       /* when dfpr_server_submit queued it */
  double admit_ms;        /* when it was admitted (its update started) */
  double done_ms;         /* when its update finished */
} dfpr_request_info;

/* A server over k units (graphs or sets, distinct). Parts are numbered over
 * the units in order: unit 0's graphs first. grid_share > 0 caps every
 * worklist launch at that many CTAs (when params->grid_ctas is 0), so that
 * updates of several units are resident on the GPU together; 0 leaves each
 * launch its schedule's own grid. EINVAL (k < 1, a NULL or repeated unit, max_slots < 1,
 * mem_fraction outside (0, 1], grid_share < 0), EBUSY (a unit is in use),
 * ENOMEM. */
dfpr_status dfpr_server_create_units(int32_t k, dfpr_graph* const* units, const dfpr_params* p,
                                     int32_t max_slots, double mem_fraction, int32_t grid_share,
                                     dfpr_server** out);

/* A server over one unit (dfpr_server_create_units with k = 1, grid_share 0):
 * every update of that unit batches all of its admitted requests. */
dfpr_status dfpr_server_create(dfpr_graph* g, const dfpr_params* p, int32_t max_slots,
                               double mem_fraction, dfpr_server** out);

/* Queues a request for graph `part` (local ids of that graph; host arrays,
 * copied). Thread-safe. *request_id identifies it for dfpr_server_wait.
 * EINVAL for a bad part or id (checked here, before queueing). */
dfpr_status dfpr_server_submit(dfpr_server* s, int32_t part, int64_t n_del,
                               const int32_t* del_src, const int32_t* del_dst, int64_t n_ins,
                               const int32_t* ins_src, const int32_t* ins_dst,
                               int64_t* request_id);

/* Blocks until the request is done; fills *info (may be NULL). */
dfpr_status dfpr_server_wait(dfpr_server* s, int64_t request_id, dfpr_request_info* info);

/* Blocks until every queued request is done and the server is idle. */
dfpr_status dfpr_server_drain(dfpr_server* s);

/* Drains, stops the worker threads and frees the server (the units stay). */
dfpr_status dfpr_server_destroy(dfpr_server* s);

/*
 * Installs the device allocator used for all later allocations (NULL, NULL
 * restores cudaMalloc / cudaFree). alloc(bytes, stream, ctx) returns a device
 * pointer or NULL; free(ptr, bytes, stream, ctx) releases it. Memory already
 * held by existing graphs is returned through the allocator that provided it.
 */
typedef void* (*dfpr_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*dfpr_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
dfpr_status dfpr_set_allocator(dfpr_alloc_fn alloc, dfpr_free_fn free_fn, void* ctx);

/* Message of the last failed call on this host thread ("" if none). */
const char* dfpr_last_error(void);

/*
 * CUDA-graph replay of the DF update (no counterpart in the paper; for the
 * many-graph step of a set, whose update is one persistent launch). With
 * enable = 1, dfpr_df_pagerank on the worklist schedule runs its device work
 * (marking items of the pending change set, control block, per-vertex
 * records, the persistent kernel, ranks back) as one replay of a CUDA graph
 * that the library captures on the graph's stream at the first such call and
 * again whenever a buffer, the grid or a parameter it depends on changes; the
 * pending counts reach the replay through pinned host memory, so a replay
 * serves any batch. The stream must not be the legacy default stream (such
 * calls run eagerly), and the first call captures, so it must not itself be
 * made while the stream is being captured. dfpr_apply_batch stays eager: its
 * allocation sizes depend on the batch. Results and stats are those of the
 * eager path; stats.ms is the persistent kernel's time. enable = 0 frees the
 * graph. Errors: EINVAL (NULL graph), EBUSY, ECUDA.
 */
dfpr_status dfpr_graph_set_capture(dfpr_graph* g, int32_t enable);

/* Captures made and replays launched so far by dfpr_graph_set_capture's
 * path (host int64 each, may be NULL). EINVAL for a NULL graph. */
dfpr_status dfpr_graph_capture_info(const dfpr_graph* g, int64_t* captures, int64_t* replays);

/*
 * Autotuner over plans (no counterpart in the paper): a plan is the schedule
 * and the tile choices of an update, four int32: mode (DFPR_MODE_*), grid_ctas
 * (0: the schedule's own), gather_split and mark_split (0: the defaults; they
 * bound the degree classes: rows gathered or marked by one warp against rows
 * cut into tokens). Like dfpr_autotune it runs the pending update once per
 * plan from the same ranks, contributions and pending change set, times each
 * whole call with CUDA events, restores that state once more and runs the
 * fastest plan, which stays applied; cost: plans + 1 updates.
 * plans: host, 4 * n_plans int32, or NULL for the built-in set: the worklist
 * schedule at the graph's own grid, at half of it and at a full wave (size
 * classes), at its own grid with split pairs (2048, 2048) and (16384, 16384)
 * (degree classes; pairs below the graph's minimum split are left out), and
 * the jacobi schedule (DF_BB, Alg. 1); repeated plans are timed once;
 * teleport graphs: the jacobi schedule alone. At most 8 built-in plans.
 * p: in, the parameters of every trial; out, the same with the chosen plan's
 * four fields. Outputs (host, may be NULL): *n_run the plans timed;
 * plans_run[4 * n_run] those plans; trial_ms[n_run] their times (INFINITY
 * for a trial that did not converge); *stats the final update's counters.
 * Returns the final update's status. Errors: EINVAL (NULL graph or p, no
 * pending change, an invalid plan), EBUSY, ENOMEM, ECUDA.
 */
dfpr_status dfpr_autotune_plans(dfpr_graph* g, dfpr_params* p, int32_t n_plans,
                                const int32_t* plans, int32_t* n_run, int32_t* plans_run,
                                double* trial_ms, dfpr_stats* stats);

/*
 * FP64 residual of the stored ranks (the L-inf test of Alg. 1, taken on the
 * final state rather than on consecutive iterates): for every vertex,
 * r'(v) = (1 - alpha)/n + alpha * sum over in-edges (u, v) of R[u] / |out(u)|
 * (Eq. 1, Sec. 3.1; plus alpha * D / n under DFPR_TELEPORT, D the rank held
 * by dead ends; n of the vertex's own graph in a set), summed in FP64 from the
 * ranks themselves, not from the stored contributions. *linf receives
 * max_v |r'(v) - R[v]|; *linf_rel (may be NULL) max_v |r'(v) - R[v]| / R[v].
 * One sweep over every in-edge on the graph's stream; the ranks are not
 * changed. Errors: EINVAL (NULL graph or linf, alpha outside (0, 1)), EBUSY,
 * ECUDA.
 */
dfpr_status dfpr_residual(const dfpr_graph* g, double alpha, double* linf, double* linf_rel);

/*
 * Static PageRank over a graph the caller already holds on the device,
 * without allocating any device memory: every rank starts at 1/n and each
 * iteration recomputes all of them from the previous iterate,
 * r_v = (1 - alpha)/n + alpha * (sum over in-edges (u, v) of r_u / d_out(u)
 * + D/n), where D is the rank held by vertices without out-edges (0 when
 * every vertex has one, e.g. a self-loop), until the largest change is
 * <= tol or max_iter iterations have run. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc / cudaFree, for
 * example code working inside a memory budget that another component (a
 * framework's pool allocator, a server's fixed arena) owns entirely, or code
 * that must not trigger the device-wide synchronisation those calls imply.
 *
 * Arguments (all arrays are device pointers on the current device):
 *   n           vertices, 1 <= n <= 1,048,576 (larger n returns EINVAL)
 *   in_offsets  int64[n + 1], in-edge row offsets (CSC); in_idx int32[m] the
 *               sources of each vertex's in-edges; out_degree int32[n]
 *   ranks       double[n], output
 *   iterations  host int32 (may be NULL): iterations performed
 *   cuda_stream the cudaStream_t to run on (NULL: the legacy default stream)
 * Scratch (a second rank vector, two contribution vectors and three control
 * words) lives in one fixed __device__ array of 24 MiB + 256 bytes that every
 * GPU loading this library keeps until the process exits. The first call on a
 * device looks up that array's device address (with the device current); a
 * cudaDeviceReset after it invalidates the address. All calls share the array: calls that overlap on
 * the GPU race and give wrong results. Returns OK, ENOTCONV (cap reached;
 * ranks are the last iterate), EINVAL, ECUDA.
 */
dfpr_status dfpr_static_pagerank_noalloc(int32_t n, const int64_t* in_offsets,
                                         const int32_t* in_idx, const int32_t* out_degree,
                                         double alpha, double tol, int32_t max_iter,
                                         double* ranks, int32_t* iterations, void* cuda_stream);

/* Number of CUDA kernels the library has launched in this process so far
 * (a diagnostic counter; no paper counterpart). */
int64_t dfpr_kernel_launches(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t dfpr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DFPR_H */
