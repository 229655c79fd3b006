/*
 * gsmart.h — C ABI of the B300 engine for SPARQL basic graph patterns by
 * grouped incident-edge evaluation over a sparse RDF matrix.
 *
 * Model (paper Sec. 1, Sec. 2.2): an RDF data set of M triples (s, p, o) is
 * an N x N sparse matrix A whose entry A(s, o) is the predicate id p. Vertex
 * ids are 0-based and predicate ids 1-based, 0 meaning "no entry"
 * (Sec. 6.2.1 step 2). Several predicates between one (s, o) pair are
 * several entries. A query is a basic graph pattern: a set of triple
 * patterns whose subject / object is a constant vertex or a variable and
 * whose predicate is a constant (Sec. 2.2.1); its answer is the set of
 * variable bindings that satisfy all patterns together (Sec. 2.2.3).
 *
 * Conventions shared by every call:
 *   - Every call returns a gs_status and never aborts, traps or exits.
 *     gs_last_error() returns a message for the calling thread's last
 *     failure (valid until that thread's next call).
 *   - "cuda_stream" is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream. Work is enqueued on it; calls that must see results
 *     synchronize it and say so.
 *   - Inputs are copied in; the caller keeps ownership of its buffers.
 *     Objects returned through an out-pointer belong to the caller, who
 *     releases them with the matching gs_free_* call (NULL is accepted).
 *   - Device memory comes from the gs_allocator when one is given (for
 *     example a framework's caching allocator), else from stream-ordered
 *     cudaMallocAsync.
 *   - Not thread-safe per object: one object must not be used by two host
 *     threads at once. Distinct objects may be used concurrently.
 */
#ifndef GSMART_H
#define GSMART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_graph gs_graph;
typedef struct gs_plan gs_plan;
typedef struct gs_result gs_result;

typedef enum {
    GS_OK = 0,
    GS_EINVAL = 1,     /* bad argument, triple or query */
    GS_ENOMEM = 2,     /* device or host allocation failed */
    GS_ECUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error) */
    GS_EOVERFLOW = 4,  /* a caller buffer is too small (nothing written) */
    GS_ETIMEOUT = 5,   /* a bounded device-side wait ran out */
    GS_ENOTIMPL = 6    /* not supported for these arguments (the call says which) */
} gs_status;

/* Device allocation hook. alloc returns NULL on failure, else memory
 * aligned to 256 bytes as cudaMalloc's is (a less aligned block is handed
 * back to free and the call fails as out of memory); both run on the host
 * thread that made the library call, with the stream the memory is used
 * on. */
typedef struct {
    void* (*alloc)(size_t bytes, void* cuda_stream, void* ctx);
    void (*free)(void* ptr, void* cuda_stream, void* ctx);
    void* ctx;
} gs_allocator;

/* ------------------------------------------------------------------ */
/* Store (Sec. 6.2, LSpM): the RDF matrix resident on the device twice,
 * row-wise (CSR, rows = subjects) and column-wise (CSC, columns =
 * objects). Every stored nonzero carries its uint32 predicate label.
 * Within a row the entries are sorted by (label, column), within a column
 * by (label, row), so the entries of one predicate in one row / column
 * form one contiguous, sorted range. Exact duplicate triples are dropped.
 * Unlike the paper's per-query LSpM, no predicate or empty row is
 * dropped: one store serves every query.
 *
 *   s, p, o            n triples; host pointers, or device pointers when
 *                      inputs_on_device != 0
 *   n_vertices         N: every s and o must be < N; N <= 2^31
 *   n_predicates       P: every p must be in 1..P
 *   alloc              optional allocation hook (copied; ctx must outlive
 *                      the graph)
 * Synchronizes cuda_stream. GS_EINVAL on a bad triple, N = 0, P = 0, or
 * when 2*ceil(log2 N) + ceil(log2 (P+1)) > 64 (packed sort keys). */
gs_status gs_load_triples(const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n,
                          uint32_t n_vertices, uint32_t n_predicates, int inputs_on_device,
                          const gs_allocator* alloc, void* cuda_stream, gs_graph** out);

/* Sizes of a loaded graph: M (after deduplication), N, P. Any out pointer
 * may be NULL. */
gs_status gs_graph_info(const gs_graph* g, uint64_t* n_triples, uint32_t* n_vertices,
                        uint32_t* n_predicates);

/* Copy one orientation of the store out (for inspection and tests).
 *   by_column = 0: ptr[N+1] row pointers, idx[M] object of each entry,
 *                  lab[M] predicate; entries grouped by subject
 *   by_column = 1: the column-wise copy: ptr by object, idx = subject
 * Buffers are host memory unless dst_on_device. Synchronizes cuda_stream. */
gs_status gs_graph_export(const gs_graph* g, int by_column, uint32_t* ptr, uint32_t* idx,
                          uint32_t* lab, int dst_on_device, void* cuda_stream);

/* ------------------------------------------------------------------ */
/* Planner (Sec. 6.1): the query graph and the order in which the
 * incident edges of its vertices are evaluated, group by group.
 *
 *   patterns     n_patterns x 3 int64 in row order (s, p, o), host memory:
 *                s, o >= 0 is a constant vertex id (< N); s, o < 0 is the
 *                variable -(k+1), variables numbered densely 0..K-1;
 *                p is a predicate id in 1..P
 *   flags        GS_PLAN_DEGREE (Sec. 6.1.2, the default) or
 *                GS_PLAN_DIRECTION (Sec. 6.1.1; queries with constants
 *                use the degree-driven order, as the paper prescribes),
 *                optionally | GS_PLAN_LISTS (the list frontier form; a
 *                plan that has no such form keeps candidate vectors)
 * g may be NULL: the plan is then made without a graph and its ids are
 * checked by gs_eval_query against the graph it runs on.
 * GS_EINVAL when there is no variable, the variables are not dense, an id
 * is out of range, or n_patterns > GS_MAX_PATTERNS; GS_ENOTIMPL when a
 * variable has more than 8 distinct patterns to bound ends or 8 self-loops, or a
 * scan would test more than 16 distinct predicates in one direction.
 * Host only. */
#define GS_PLAN_DEGREE 0u
#define GS_PLAN_DIRECTION 1u
#define GS_PLAN_PATHS 4u      /* option bit: evaluate with one binding tree per
                                 path of the traversal (Sec. 7.1), reconciled
                                 by local and global tree-pruning (Sec. 8.1,
                                 8.2) and joined into the answers */
#define GS_PLAN_LISTS 2u      /* option bit: for a plan with a triple scan, only
                                 the levels listed from the scan (roots) get a
                                 candidate vector; later levels check the
                                 predicates of their pending edges by a search
                                 of each candidate's label-sorted row / column
                                 (the pre-pruning of Sec. 7.2.2) instead */
#define GS_MAX_PATTERNS 32
#define GS_MAX_VARS 31
gs_status gs_plan_query(const gs_graph* g, const int64_t* patterns, uint32_t n_patterns,
                        uint32_t flags, gs_plan** out);

/* The plan as int32 words, for inspection:
 *   [n_groups, then per group: vertex, n_edges, edge indices...,
 *    n_roots, roots...]
 * where a vertex is the variable index k >= 0, or -(1 + c) for constant
 * vertex id c. *len receives the word count; GS_EOVERFLOW (nothing
 * written) when cap is smaller. */
gs_status gs_plan_describe(const gs_plan* plan, int32_t* buf, uint32_t cap, uint32_t* len);

/* The binding-tree paths of the plan (Sec. 7.1, Ex. 7.1) as int32 words:
 *   [n_paths, then per path: n_vertices, variable indices...]
 * from each root, each edge of a group is followed to its other end, and
 * into that end's group when this edge first reached it, else the path
 * ends; self-loops and edges to constants do not extend a path, and a
 * variable no path reaches is a path of its own. *len receives the word
 * count; GS_EOVERFLOW (nothing written) when cap is smaller. */
gs_status gs_plan_paths(const gs_plan* plan, int32_t* buf, uint32_t cap, uint32_t* len);

/* ------------------------------------------------------------------ */
/* Evaluation (Sec. 5, Sec. 7): grouped incident-edge evaluation of the
 * plan, fully on the device. Candidate vectors of the variables are the
 * AND of the predicate selections of all their incident edges (Eq. 17,
 * Eq. 21); bindings are expanded level by level into a tree stored as
 * device arrays (Sec. 7.1), pruned as soon as an edge has no match
 * (Sec. 7.2.2) and enumerated into tuples.
 *
 * gs_eval_query enqueues the work on cuda_stream and returns without
 * waiting. A plan without a full triple scan whose first level is small
 * runs first in one CTA; if that CTA's budgets do not hold the query, the
 * grid path continues from the levels it completed (this happens inside
 * gs_result_info / gs_fetch_bindings, on the same stream). The result holds
 * device memory until gs_free_result. */
gs_status gs_eval_query(gs_graph* g, const gs_plan* plan, void* cuda_stream, gs_result** out);

/* Root-range evaluation: the first-stage partition of Sec. 6.3.1. Every
 * answer has exactly one binding of the plan's root variable (the variable
 * of its first level, gs_plan_root), so evaluating the query once per
 * range of a partition of the vertex ids [0, N) and concatenating the
 * answers gives the whole answer set, each row once; replicas each holding
 * the full graph can take one range apiece and exchange only the answers
 * at the end. gs_eval_query_roots returns the answers of plan whose root
 * binding lies in [root_lo, root_hi) (root_hi may exceed N; an empty range
 * gives no answers). It runs on the grid path (the root filter sits in the
 * level-0 kernels); the result is used and freed like gs_eval_query's.
 * GS_EINVAL for NULL arguments, root_lo > root_hi, or a GS_PLAN_PATHS plan
 * (one root per path). gs_plan_root writes the root variable's index (its
 * answer column); GS_EINVAL for a GS_PLAN_PATHS plan. Host only. */
gs_status gs_eval_query_roots(gs_graph* g, const gs_plan* plan, uint32_t root_lo, uint32_t root_hi,
                              void* cuda_stream, gs_result** out);
gs_status gs_plan_root(const gs_plan* plan, uint32_t* var);

/* Estimated device memory of evaluating the plan alone on g (*bytes: the
 * binding-tree levels of Sec. 7.1 with their scratch, the answer rows, and
 * for a plan with a triple scan its candidate vectors and masks) and its
 * estimated answer rows (*rows). Made on the host from per-predicate counts
 * taken when the graph was loaded (entries per label, rows and columns
 * holding each label), taking labels as independent of the structure: a
 * level's nodes are the previous level's times the mean range length of
 * the edge it expands, times the share of candidates that hold the
 * predicates of the variable's other edges. It is an estimate, not a
 * bound. The server admits queries by it, and gs_eval_query sizes its first
 * workspace by it when it exceeds the default. Either out pointer may be
 * NULL. */
gs_status gs_plan_estimate(const gs_graph* g, const gs_plan* plan, uint64_t* bytes, double* rows);

/* Number of answer rows and variables. Waits for the result's own work on
 * its stream (work enqueued on the stream after it is not waited for).
 * When the evaluation ran out of its device workspace it is re-run with a
 * larger one; GS_ENOMEM when the device cannot hold it. The first
 * workspace is 512 MiB (at most 1/8 of free memory, at least 64 MiB), or
 * the byte count in the environment variable GS_ARENA_BYTES. */
gs_status gs_result_info(gs_result* r, uint64_t* n_rows, uint32_t* n_vars);

/* Copy the answers out: n_rows x n_vars int32, row-major, column k holds
 * variable k. Rows are distinct; with sort_rows != 0 they are in ascending
 * lexicographic order, else in an unspecified order. dst is host memory
 * unless dst_on_device. GS_EOVERFLOW (nothing written) when
 * cap_rows < n_rows. Synchronizes the result's stream. */
gs_status gs_fetch_bindings(gs_result* r, int32_t* dst, uint64_t cap_rows, int dst_on_device,
                            int sort_rows);

/* The binding tree of r's last grid-path evaluation (Sec. 7.1): nodes per
 * level into nodes[0 .. *n_levels) (waits like gs_result_info).
 * GS_EOVERFLOW when cap < the plan's levels; GS_ENOTIMPL when the query
 * ran in the single-CTA kernel (its levels are not kept). */
gs_status gs_result_tree(gs_result* r, uint64_t* nodes, uint32_t cap, uint32_t* n_levels);

/* Tracing (the phase breakdown of Sec. 9.1.2, on the device). With
 * gs_graph_set_trace(g, 1), every grid-path evaluation on g records CUDA
 * events between its phases: setup and triple scan, then each level of
 * the binding tree (Sec. 7.1), then the enumeration of the answers.
 * gs_result_phases writes their device milliseconds into ms[0 ..
 * *n_phases) in that order (*n_phases = levels + 2; waits like
 * gs_result_info). The events may keep consecutive kernels from
 * overlapping, so traced times can exceed untraced ones. GS_ENOTIMPL when
 * the result has no phase events (tracing was off when it was enqueued, or
 * it ran in the single-CTA kernel); GS_EOVERFLOW (with *n_phases set) when
 * cap < *n_phases. Host entry points also mark NVTX ranges (store build,
 * planning, evaluation enqueue and waits, answer fetches, batch launches,
 * server admissions), visible to a profiler that records them. */
gs_status gs_graph_set_trace(gs_graph* g, int on);
gs_status gs_result_phases(gs_result* r, float* ms, uint32_t cap, uint32_t* n_phases);

/* Statistics of the last evaluation of r (synchronizes): device time in
 * milliseconds from CUDA events around the enqueued work, and the number of
 * kernels it launched. For a query the single CTA handed back, both cover
 * the grid-path part only. Either out pointer may be NULL. */
gs_status gs_result_stats(gs_result* r, float* device_ms, uint32_t* kernel_launches);

/* ------------------------------------------------------------------ */
/* Batched evaluation: the same evaluation (Sec. 5, Sec. 7) of many plans in
 * one persistent launch. Every CTA takes the next query from a device work
 * counter and evaluates it on its own; answers of all queries share one
 * device pool. Plans that need the full triple scan, and queries that
 * outgrow one CTA's budget, are evaluated with the grid path of
 * gs_eval_query on side streams of the graph (the former from the start,
 * the latter after the batch kernel). Answers are identical to
 * gs_eval_query's.
 *
 *   plans        n plan pointers (host array; plans must outlive the batch)
 * Enqueued on cuda_stream; gs_batch_info synchronizes. The pool starts at
 * min(4 GiB, 1/4 of free memory) or the byte count in the environment
 * variable GS_BATCH_POOL_BYTES; a query that does not fit it is handed to
 * the grid path. */
typedef struct gs_batch gs_batch;
gs_status gs_eval_batch(gs_graph* g, const gs_plan* const* plans, uint32_t n, void* cuda_stream,
                        gs_batch** out);

/* Tunables of a batched evaluation; a zero field takes its default. */
typedef struct {
    uint32_t blocks_per_sm;  /* resident CTAs per SM of the batch kernel
                                (0: as many as fit) */
    uint32_t grid_streams;   /* streams on which grid-path queries run side by
                                side (0: 4; at most 16) */
    uint64_t cand_budget;    /* candidates a CTA takes at one level before
                                handing its query to the grid path (0: 65,536) */
    uint64_t row_budget;     /* answer rows a CTA writes before handing its
                                query to the grid path (0: 65,536) */
    uint64_t pool_bytes;     /* answer pool (0: min(4 GiB, free / 4), or
                                GS_BATCH_POOL_BYTES) */
    uint32_t scan_share;     /* triple scans of the plans that need one
                                (constant-free plans): 0 or 1, shared: plans
                                are packed into passes of at most 32
                                predicates per direction (each plan into the
                                pass it adds the fewest predicates to) and
                                each pass reads the labels once (Sec. 5
                                grouping applied across queries); 2, one
                                scan per plan */
    uint32_t frontier;       /* candidate sets those plans test later levels
                                against: 0 or 1, bitmaps (the scan writes
                                one candidate vector per variable; a test is
                                one bit); 2, lists (the scan writes only the
                                vectors the plan's roots are listed from;
                                later candidates are checked by a search of
                                their label-sorted row or column) */
} gs_batch_config;

/* gs_eval_batch under cfg (NULL: all defaults). Grid-path queries run on
 * up to cfg->grid_streams streams of the graph side by side and are joined
 * before gs_batch_info returns. GS_EINVAL on a NULL graph, plan array or
 * out pointer. */
gs_status gs_eval_batch_cfg(gs_graph* g, const gs_plan* const* plans, uint32_t n,
                            const gs_batch_config* cfg, void* cuda_stream, gs_batch** out);

/* Autotuner: evaluates the n plans (a sample of the workload) under a fixed
 * set of candidate configurations, each twice, and returns in *best the one
 * with the smallest wall time from enqueue to the last answer count (of
 * those within 3% of it, the one that hands the fewest queries to the grid
 * path), whose time goes to *best_ms (may be NULL). Stage 1 tries CTAs per SM x candidate
 * budget x row budget; stage 2, when the sample holds plans with a triple
 * scan, tries shared or per-plan scans x bitmap or list frontier x 4 or 16
 * grid-path streams under the stage-1 choice. The choice is kept for the life of the process, keyed by
 * the device name, the graph's N, M and P and the sample's shape classes
 * (scan or seeded, levels, leaves); a later call with the same key returns
 * it without timing. Synchronizes cuda_stream; answers are discarded.
 * Every configuration gives identical answers; only time differs. */
gs_status gs_batch_autotune(gs_graph* g, const gs_plan* const* plans, uint32_t n,
                            void* cuda_stream, gs_batch_config* best, float* best_ms);

/* Triple scans the batch ran (*n_scans) and the plans they served
 * (*n_scan_plans); with shared scans n_scans is the number of passes.
 * Either out pointer may be NULL. Does not synchronize. */
gs_status gs_batch_scans(gs_batch* b, uint32_t* n_scans, uint32_t* n_scan_plans);

/* Non-blocking: *done = 1 once everything gs_eval_batch enqueued has
 * finished on the device (gs_batch_info then returns without waiting for the
 * batch kernel; queries handed to the grid path still run there). */
gs_status gs_batch_poll(gs_batch* b, int* done);

/* Answer row counts: rows[q] for each query (rows may be NULL) and their sum.
 * Synchronizes the batch's stream. */
gs_status gs_batch_info(gs_batch* b, uint64_t* rows, uint64_t* total_rows);

/* Answers of query q, as gs_fetch_bindings (row-major int32, n_vars columns;
 * GS_EOVERFLOW when cap_rows is short). */
gs_status gs_batch_fetch(gs_batch* b, uint32_t q, int32_t* dst, uint64_t cap_rows,
                         int dst_on_device, int sort_rows);

/* Device time from the batch's first enqueued operation to its last result,
 * kernels launched, and queries handed to the grid path. Any out pointer may
 * be NULL. Synchronizes. */
gs_status gs_batch_stats(gs_batch* b, float* device_ms, uint32_t* kernel_launches,
                         uint32_t* n_escalated);

void gs_free_batch(gs_batch* b);

/* ------------------------------------------------------------------ */
/* Serving loop (continuous batching). The server keeps the graph resident
 * and owns a worker thread and a pool of CUDA streams. Submitted plans wait
 * in arrival order; when the device is idle, when max_batch / 8 plans
 * wait, or when the oldest has waited max_wait_us or half the running mean
 * time of the server's batches (whichever is longer), the worker admits
 * waiting plans into a batch (as in gs_eval_batch) while a stream is free
 * and the batch's estimated device bytes fit the memory budget together
 * with the batches in flight. A plan's bytes are its estimated
 * intermediate results (gs_plan_estimate's model): for a plan the batch
 * kernel evaluates, its estimated answer bytes (at most
 * pool_bytes_per_query) as its share of the answer pool; for a grid-path
 * plan, its candidate vectors and the first workspace it will take. A
 * batch adds its CTA workspaces and, with plans that need a triple scan,
 * the scan's masks. A plan that does not fit waits and later plans that do
 * fit pass it, until it has waited 50 x max_wait_us (then nothing passes
 * it); a plan too large for the budget on its own runs alone once nothing
 * else is in flight. Batches admitted while others run overlap on the
 * device; queries a batch hands to the grid path run on the graph's side
 * streams without holding up the worker. Answers are identical to
 * gs_eval_query's; they stay on the device until the ticket is released.
 * Submit / poll / fetch / release may be called from any host thread. */
typedef struct gs_server gs_server;
typedef struct {
    uint32_t max_batch;              /* queries per batch (0: 1024) */
    uint32_t n_streams;              /* batches in flight (0: 4) */
    uint64_t memory_budget;          /* bytes of device memory (0: 40 GiB) */
    uint32_t max_wait_us;            /* while batches run, the least time a
                                        queued query waits for more arrivals
                                        before it starts a batch (0: 200;
                                        half the mean batch time when that
                                        is longer) */
    uint64_t pool_bytes_per_query;   /* largest answer-pool share of one
                                        query (0: 16 MiB) */
    gs_batch_config batch;           /* tunables of every batch (zero fields:
                                        defaults; pool_bytes is ignored) */
} gs_server_config;

gs_status gs_server_start(gs_graph* g, const gs_server_config* cfg, gs_server** out);
/* Queue one plan (the plan must outlive its ticket). */
gs_status gs_server_submit(gs_server* s, const gs_plan* plan, uint64_t* ticket);
/* Queue n plans at once, in array order (the worker sees all or none of
 * them); tickets[i] receives plan i's ticket. */
gs_status gs_server_submit_many(gs_server* s, const gs_plan* const* plans, uint32_t n,
                                uint64_t* tickets);
/* Non-blocking: *done = 1 when the answer is ready; then *rows and
 * *latency_us (submission to completion, host clock) are set (may be NULL). */
gs_status gs_server_poll(gs_server* s, uint64_t ticket, int* done, uint64_t* rows,
                         double* latency_us);
/* Answers of a finished ticket, as gs_fetch_bindings. */
gs_status gs_server_fetch(gs_server* s, uint64_t ticket, int32_t* dst, uint64_t cap_rows,
                          int dst_on_device, int sort_rows);
/* Drop a finished ticket and its device memory share. */
gs_status gs_server_release(gs_server* s, uint64_t ticket);
/* The batch that took a ticket (1-based sequence number, 0 while it waits)
 * and the ticket's estimated device bytes. Either out pointer may be NULL. */
gs_status gs_server_ticket(gs_server* s, uint64_t ticket, uint64_t* batch_seq,
                           uint64_t* est_bytes);
/* Admissions so far that took a plan ahead of an older waiting one, and the
 * estimated bytes of the batches in flight now. Either may be NULL. */
gs_status gs_server_admission(gs_server* s, uint64_t* passed, uint64_t* inflight_bytes);
/* Queries completed, batches launched, peak admitted device bytes. */
gs_status gs_server_stats(gs_server* s, uint64_t* completed, uint64_t* batches,
                          uint64_t* peak_bytes);
/* Finish the queued work, free everything. */
void gs_server_stop(gs_server* s);

/* Load replay (a measuring aid, no counterpart in the paper): submits n
 * queries, query i being plans[i % n_plans], each at arrival_s[i] seconds
 * after the call starts (non-decreasing), from the calling thread; polls
 * and releases them as they finish. latency_us[i] (may be NULL) receives
 * the time from the scheduled arrival to completion as the server's worker
 * saw it, done_s[i] (may be NULL) the completion time since the call
 * started. With fetch_buf (host memory of fetch_cap_rows rows of the
 * widest plan; may be NULL) every finished query's answers are copied
 * there before its release, and *fetched_bytes (may be NULL) gets their
 * total. Returns when every query has finished; GS_ETIMEOUT if that takes
 * longer than timeout_s; GS_EOVERFLOW when an answer does not fit
 * fetch_buf; a failed query's status otherwise. */
gs_status gs_server_replay(gs_server* s, const gs_plan* const* plans, uint32_t n_plans,
                           const double* arrival_s, uint64_t n, double timeout_s,
                           double* latency_us, double* done_s, int32_t* fetch_buf,
                           uint64_t fetch_cap_rows, uint64_t* fetched_bytes);
/* Kernel launches, triple scans and plans served by those scans, summed
 * over the batches completed so far. Any out pointer may be NULL. */
gs_status gs_server_work(gs_server* s, uint64_t* launches, uint64_t* scans, uint64_t* scan_plans);

/* ------------------------------------------------------------------ */
/* One grouped predicate selection on its own (Eq. 17, Eq. 21):
 *     v = AND_i  (dir_i == 0 ? A (x) u_{p_i} : A^T (x) u_{p_i})
 * i.e. bit x of v is 1 when row x of A holds every predicate p_i with
 * dir_i == 0 and column x holds every p_i with dir_i == 1 (Eq. 4, Eq. 5).
 *   preds, dirs   n host arrays (n >= 1), at most 16 distinct predicates per
 *                 direction
 *   out_bits      device buffer of ceil(N/32) uint32 words; bit x of the
 *                 vector is bit (x % 32) of word x / 32; bits >= N are 0
 * Enqueued on cuda_stream (no synchronization). */
gs_status gs_scan_candidates(gs_graph* g, const uint32_t* preds, const uint8_t* dirs, uint32_t n,
                             uint32_t* out_bits, void* cuda_stream);

/* Did the standalone scans on g complete? Synchronizes cuda_stream, then
 * returns GS_ETIMEOUT when a bounded wait for the bulk copies of a scan
 * enqueued by gs_scan_candidates or gs_scan_candidates_noalloc on g (on any
 * stream, since the last call of gs_scan_status) ran out; that scan's bits
 * are incomplete. The report is then cleared. GS_OK otherwise. Scans that
 * gs_eval_query runs report a stall through gs_result_info instead.
 * Allocates nothing. The wait lasts about 2 s; the environment variable
 * GS_SCAN_STALL_CYCLES (a clock-cycle count, 0: give up at once) shortens
 * it, for failure tests. */
gs_status gs_scan_status(gs_graph* g, void* cuda_stream);

/* gs_scan_candidates without any device allocation on the call path (the
 * paper has no counterpart; it is an engineering variant for callers that
 * must not allocate). Same arguments, result and errors as
 * gs_scan_candidates, plus:
 *   - the scan's workspace, a little over 4 (N + 256) bytes for a graph of
 *     N vertices, lives in one static device array of
 *     gs_noalloc_scratch_bytes() bytes (48 MiB: graphs up to about 12
 *     million vertices); a graph that needs more gets GS_EINVAL and a
 *     message naming both sizes;
 *   - nothing in that array has to start at zero (each call zeroes what it
 *     accumulates into);
 *   - the first call on a device looks the array up (cudaGetSymbolAddress)
 *     and caches its address: make it before any stream capture (a first
 *     call on a capturing stream returns GS_EINVAL);
 *   - a stalled scan is reported by gs_scan_status, as for
 *     gs_scan_candidates;
 *   - the current device must be the graph's (else GS_EINVAL);
 *   - all calls on one device share the array: calls whose work overlaps in
 *     time (other streams, unordered host threads) race and corrupt each
 *     other's results; calls on one stream are ordered and safe. */
gs_status gs_scan_candidates_noalloc(gs_graph* g, const uint32_t* preds, const uint8_t* dirs,
                                     uint32_t n, uint32_t* out_bits, void* cuda_stream);
/* Size in bytes of the static workspace of gs_scan_candidates_noalloc. */
size_t gs_noalloc_scratch_bytes(void);

/* ------------------------------------------------------------------ */
/* Per-query light-weight sparse matrix (LSpM, Sec. 6.2): the RDF matrix
 * reduced on the device, from the resident store, to the predicates a query
 * uses. Row-wise it keeps the entries whose predicate is in row_preds and
 * drops the rows left empty (Sec. 6.2.1 steps 1, 3, 4; Sec. 6.2.2's CSR
 * part); column-wise it does the same with col_preds (Sec. 6.2.2's CSC
 * part). Reduced rows keep the (label, other end) order.
 *   row_preds, col_preds   host arrays of predicate ids in 1..P (repeats
 *                          allowed; either may be empty)
 * Synchronizes cuda_stream. The LSpM holds device memory until
 * gs_free_lspm and must not outlive g. */
typedef struct gs_lspm gs_lspm;
gs_status gs_lspm_build(gs_graph* g, const uint32_t* row_preds, uint32_t n_row,
                        const uint32_t* col_preds, uint32_t n_col, void* cuda_stream,
                        gs_lspm** out);
/* The LSpM of one plan (the degree-driven storage of Sec. 6.2.2): row-wise
 * the predicates its evaluation reads from rows (edges expanded from or
 * checked against a subject's row, pre-pruning of a variable's out-edges,
 * the triple scan's row predicates), column-wise those it reads from
 * columns. */
gs_status gs_lspm_for_plan(gs_graph* g, const gs_plan* plan, void* cuda_stream, gs_lspm** out);
/* Rows (by_column = 0) or columns (1) kept, and entries kept. Either out
 * pointer may be NULL. */
gs_status gs_lspm_info(const gs_lspm* l, int by_column, uint64_t* kept, uint64_t* nnz);
/* The reduced orientation in the paper's arrays:
 *   m[N+1]      Mr (Mc): m[i+1] - m[i] = 1 when row i is kept, and it is
 *               then row m[i] of the reduced matrix
 *   ptr[kept+1] Pr (Pc): the kept rows' entry ranges
 *   val[nnz]    predicate of each entry; idx[nnz] its column (row) id
 * Buffers are host memory unless dst_on_device. Synchronizes cuda_stream. */
gs_status gs_lspm_export(const gs_lspm* l, int by_column, uint32_t* m, uint32_t* ptr,
                         uint32_t* val, uint32_t* idx, int dst_on_device, void* cuda_stream);
/* gs_eval_query on the LSpM instead of the full store (same answers).
 * GS_EINVAL when l was built for another graph or lacks a (predicate,
 * orientation) pair the plan reads. */
gs_status gs_eval_query_lspm(gs_graph* g, const gs_lspm* l, const gs_plan* plan, void* cuda_stream,
                             gs_result** out);
void gs_free_lspm(gs_lspm* l);

/* Frees the graph. Stop every server started on it (gs_server_stop) and
 * free its results, batches and LSpMs first: they use its store. */
void gs_free_graph(gs_graph* g);
void gs_free_plan(gs_plan* plan);
void gs_free_result(gs_result* r);

const char* gs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GSMART_H */
