// Executor structures shared by gs_exec.cu and the C ABI.
#pragma once

#include "gs_internal.h"

namespace gs {

constexpr uint32_t kStHuge = 4u;      // a tree node has more than 2^40 answer rows
constexpr uint32_t kStEscalate = 8u;  // the single-block kernel handed the query back

// Control block at the start of the workspace: level sizes and the
// partial sums of the device-wide scans. Zeroed before each evaluation.
struct Ctl {
    uint64_t n[kMaxLevels];        // nodes per level
    uint64_t list_n[kMaxLevels];   // candidate-list length of a list-fed level
    uint64_t cand;                 // candidates of the level being expanded
    uint64_t one;                  // 1: node count of the virtual parent of level 0
    uint64_t rows;                 // answer rows
    uint32_t status;               // kSt* bits
    uint32_t dead;                 // a pattern with two constant ends has no match
    uint32_t arrive;               // blocks of the running count kernel that are done
    uint32_t roff_chunk;           // its blocks took roff_chunk consecutive items each
    uint32_t levels_done;          // single-block kernel: complete levels when it handed back
    uint32_t pad;
    uint64_t bsum[kBlocks];
    uint64_t boff[kBlocks];
};
constexpr uint64_t kCtlBytes = ((sizeof(Ctl) + 255) / 256) * 256;
constexpr uint64_t kCtlHead = offsetof(Ctl, bsum);   // bytes the host reads back

struct ExecDev {
    uint8_t* arena;
    uint64_t arena_bytes;
    Ctl* ctl;
    DStore out, in;
    uint32_t* bits;           // candidate vector of level l at bits + l * words
    uint64_t words;
    uint32_t* lists;          // candidate list of level l at lists + l * list_stride
    uint64_t list_stride;
    // root range (first-stage partition of Sec. 6.3.1): with root_cut set,
    // level 0 keeps only vertices in [root_lo, root_hi)
    uint32_t root_cut, root_lo, root_hi;
};

struct ConstChecks {
    uint32_t n;
    uint32_t t[3 * kMaxPatterns];
};

struct EnumSpec {
    int32_t n_leaves;
    int32_t n_vars;
    LeafSpec leaf[kMaxVars];
    int32_t var_src[kMaxVars];
    int32_t col_of_level[kMaxLevels];   // answer column of each level's variable
    int32_t col_of_leaf[kMaxVars];      // answer column of each leaf
};

// The whole schedule of one query, passed by value to single-block kernels.
struct QueryDev {
    int32_t n_levels;
    ConstChecks cc;
    EnumSpec F;
    LevelSpec lv[kMaxLevels];
};

inline void make_query_dev(const gs_plan* P, QueryDev* Q) {
    Q->n_levels = P->n_levels;
    Q->cc.n = (uint32_t)(P->const_triples.size() / 3);
    if (Q->cc.n > (uint32_t)kMaxPatterns) Q->cc.n = kMaxPatterns;
    for (uint32_t i = 0; i < 3 * Q->cc.n; ++i) Q->cc.t[i] = P->const_triples[i];
    Q->F.n_leaves = P->n_leaves;
    Q->F.n_vars = P->n_vars;
    for (int j = 0; j < P->n_leaves; ++j) Q->F.leaf[j] = P->leaves[j];
    for (int v = 0; v < P->n_vars; ++v) Q->F.var_src[v] = P->var_src[v];
    for (int l = 0; l < P->n_levels; ++l) Q->lv[l] = P->levels[l];
}

// One query's answer in a batch: rows at pool + off, or escalated.
struct BatchResult {
    uint64_t off;
    uint64_t rows;
    uint32_t status;      // 0, or kStEscalate (run again on the grid path)
    uint32_t pad;
};

// Parameters of the persistent batch kernel.
struct BatchDev {
    DStore out, in;
    const uint8_t* recs;          // packed query records
    const uint64_t* rec_off;      // byte offset of each record
    uint32_t n;
    uint8_t* slots;               // one workspace per CTA
    uint64_t slot_bytes;
    uint8_t* pool;                // answer rows of all queries
    uint64_t pool_bytes;
    unsigned long long* pool_top;
    uint32_t* next;               // work counter
    BatchResult* res;
    uint64_t cand_budget, row_budget;
};

gs_status enqueue_batch(const BatchDev& B, int blocks, cudaStream_t st);
int batch_blocks_per_sm();
gs_status sort_rows_on_device(const gs_graph* g, const int32_t* rows, uint64_t n, uint32_t k,
                              int32_t* out, cudaStream_t st);
gs_status eval_query_path(gs_graph* g, const gs_plan* plan, void* cuda_stream, int force_grid,
                          gs_result** out);
// gs_eval_batch with the tunables of cfg (NULL or zero fields: defaults)
// and at most max_blocks CTAs (0: no cap).
gs_status eval_batch_ex(gs_graph* g, const gs_plan* const* plans, uint32_t n, void* cuda_stream,
                        const gs_batch_config* cfg, int max_blocks, gs_batch** out);
uint64_t batch_device_bytes(const gs_batch* b);
// Does a batch under cfg evaluate plan P in its persistent kernel (else on
// the grid path)?
bool batch_in_kernel(const gs_graph* g, const gs_plan* P, const gs_batch_config* cfg);
// Device bytes a batch under cfg holds whatever its queries: the CTA
// workspaces of n_kernel kernel queries, and the triple scan's masks when
// it holds a plan with a scan.
uint64_t batch_fixed_bytes(const gs_graph* g, const gs_batch_config* cfg, uint32_t n_kernel,
                           bool has_scan);
// Non-blocking progress of a batch: *done = 1 once every answer count is
// known (the grid-path queries it handed on included).
gs_status batch_advance(gs_batch* b, int* done);
// Non-blocking: *done = 1 once a result's enqueued work has finished.
gs_status result_ready(gs_result* r, int* done);
// Waits for the result, then moves its answer rows into a right-sized
// allocation and frees its workspace (fetches read the rows from there).
gs_status result_compact(gs_result* r);

// Estimated sizes of one evaluation of a plan, from the graph's
// per-predicate statistics (labels taken as independent of the structure):
// tree nodes per level, answer rows and the device bytes they take.
struct Estimate {
    double nodes[kMaxLevels];
    double rows;
    uint64_t arena;      // control block, levels, their scratch, answer rows
    uint64_t vectors;    // candidate vectors of a plan with a triple scan
    uint64_t answer;     // answer rows alone
    uint64_t total;      // arena + vectors (+ the scan's masks for a query alone)
};
void plan_estimate(const gs_graph* g, const gs_plan* P, Estimate* e);
// The first workspace a grid-path evaluation of a plan with estimate e takes.
uint64_t first_arena_bytes(gs_graph* g, const Estimate& e);

// Grids of k_range and k_expand on a device with sm_count SMs: the blocks
// that fit at once (k_range's at most kBlocks, the size of its block sums).
void level_grids(int sm_count, int* range_blocks, int* expand_blocks);

uint64_t host_level_off(const uint64_t* n, int l);
bool small_eligible(const gs_plan* P);
// An upper bound on the plan's first-level candidates from its constants'
// row / column lengths (UINT64_MAX without a constant seed).
uint64_t first_level_bound(const gs_graph* g, const gs_plan* plan);
gs_status enqueue_small(const gs_plan* P, const ExecDev& E, uint32_t* launches, cudaStream_t st);
// The grid path. start_level > 0 resumes a query the single-block kernel
// handed back, whose levels 0 .. start_level - 1 are complete in E's
// workspace (a plan without triple scan). scanned != NULL: the candidate
// vectors are already in E.bits (a triple scan shared with other queries,
// whose status word `scanned` is); the query runs no scan of its own.
// phase_ev (NULL: none): P->n_levels + 2 events recorded after the setup
// and triple scan, after each level, and after the enumeration.
gs_status enqueue_eval(const gs_graph* g, const gs_plan* P, const ExecDev& E, void* scan_work, uint32_t* launches,
                       cudaStream_t st, int start_level = 0, const uint32_t* scanned = nullptr,
                       const Store* so = nullptr, const Store* si = nullptr,
                       const cudaEvent_t* phase_ev = nullptr);
// As eval_query_prescanned, but bits stay the caller's (several results
// read one set of candidate vectors).
gs_status eval_query_borrowed(gs_graph* g, const gs_plan* plan, void* cuda_stream, uint32_t* bits,
                              cudaEvent_t ready, const uint32_t* scan_status, gs_result** out);
// A result whose answers are a table built outside the executor: created
// (its start event recorded on st), then given the rows (device memory the
// result takes over, n rows of the plan's variables in order).
gs_result* result_new_table(gs_graph* g, const gs_plan* plan, cudaStream_t st);
gs_status result_set_table(gs_result* r, int32_t* rows, uint64_t bytes, uint64_t n,
                           uint32_t launches, const std::vector<uint64_t>& path_nodes);
void result_free(gs_result* r);
// The device rows of a finished result (waits for it; NULL on failure).
const int32_t* result_rows(gs_result* r);
// Per-path evaluation (gs_paths.cu) of a plan made with GS_PLAN_PATHS.
gs_status eval_paths(gs_graph* g, const gs_plan* plan, void* cuda_stream, gs_result** out);
// Per-query LSpM (gs_lspm.cu): the (predicate, orientation) pairs a plan's
// evaluation reads; an LSpM's orientation; whether an LSpM holds every pair
// a plan reads.
void plan_store_preds(const gs_plan* P, std::vector<uint32_t>* rows, std::vector<uint32_t>* cols);
const Store* lspm_side(const gs_lspm* L, int dir);
bool lspm_covers(const gs_lspm* L, const gs_plan* P);
const gs_graph* lspm_graph(const gs_lspm* L);
// A grid-path evaluation of a plan whose candidate vectors a shared triple
// scan writes into `bits` (n_levels vectors of ceil(N/32) words, taken over
// by the result); its stream waits for `ready` before the first kernel, and
// `scan_status` is that scan's status word.
gs_status eval_query_prescanned(gs_graph* g, const gs_plan* plan, void* cuda_stream, uint32_t* bits,
                                cudaEvent_t ready, const uint32_t* scan_status, gs_result** out);

}  // namespace gs
