// Internal declarations of the engine: store, plan and executor structures
// shared by the host code and the sm_103a kernels.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gsmart.h"

namespace gs {

constexpr int kMaxVars = GS_MAX_VARS;        // 31: one bit per variable in 32-bit masks
constexpr int kMaxPatterns = GS_MAX_PATTERNS;
constexpr int kMaxLevels = 32;               // one materialized level per variable at most
constexpr int kMaxBinders = 8;               // edges joining a level's variable to bound ends
constexpr int kMaxProbes = 16;               // presence tests on a level's candidates
constexpr int kMaxSelf = 8;                  // self-loop patterns ?w p ?w per variable
constexpr int kMaxSlots = 16;                // distinct predicates per direction in one query's scan
constexpr int kMaxSlotsWide = 32;            // ... in one scan shared by several queries (32-bit masks)
constexpr int kBlocks = 1024;                // upper bound of the fixed grid (blocks)
constexpr int kThreads = 256;

// Triple-scan work items. Each orientation is cut into items of equal cost
// along the merge of its row ends and its labels (merge path): an item
// holds at most kScanItemCost units, one per label and one per row end,
// so it fits one shared-memory buffer and one pass of a warp whose 32 lanes
// take kScanLabPer labels each.
constexpr uint32_t kScanLabPer = 33;                       // labels per lane (odd: no bank conflicts)
constexpr uint32_t kScanItemCost = 32 * kScanLabPer - 2;

// Status bits written by kernels into the control block.
constexpr uint32_t kStOverflow = 1u;  // a level or the output did not fit the workspace
constexpr uint32_t kStBadInput = 2u;
constexpr uint32_t kStStall = 16u;    // a bulk copy of the triple scan did not complete in time

const char* last_error();

void set_error(const char* fmt, ...);
gs_status cuda_fail(cudaError_t e, const char* what);

#define GS_CUDA(call)                                            \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return ::gs::cuda_fail(_e, #call); \
    } while (0)

// Launch with programmatic stream serialization: the kernel may be
// scheduled while the previous kernel in the stream is still running; it
// must wait for that one (griddepcontrol.wait) before touching what it
// writes.
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                           cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Device memory through the caller's hook or stream-ordered cudaMallocAsync.
struct Alloc {
    gs_allocator hook{};
    bool has_hook = false;
    void* get(size_t bytes, cudaStream_t st) const;
    void put(void* p, cudaStream_t st) const;
};

// One orientation of the RDF matrix. Row r holds entries [ptr[r], ptr[r+1])
// of idx (the other end) and lab (the predicate), sorted by (lab, idx).
// ptr, idx and lab are padded with 4 zero words so aligned 16-byte loads
// and bulk copies that start inside the array stay inside the allocation.
// A named NVTX range over a host-side step (a no-op unless a profiler is
// attached): the store build, planning, evaluation enqueue, waits, batch
// and server admission.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Store {
    uint32_t* ptr = nullptr;
    uint32_t* idx = nullptr;
    uint32_t* lab = nullptr;
    // scan items: items[c] = (rows completed, labels consumed) before item c,
    // c = 0..n_items (items[n_items] = (N, M))
    uint2* items = nullptr;
    uint32_t n_items = 0;
    // bit k of heads: entry k is the first entry of its row
    // (M / 32 + 8 words, zero past the last entry)
    uint32_t* heads = nullptr;
    // label directory of the rows longer than kDirMin entries: the runs of
    // equal labels of row r are dir_lab / dir_pos [dir_off[r], dir_off[r+1])
    // (label, first entry); shorter rows have none. NULL when not built.
    uint32_t* dir_off = nullptr;
    uint32_t* dir_lab = nullptr;
    uint32_t* dir_pos = nullptr;
    uint64_t dir_runs = 0;
};

constexpr uint32_t kDirMin = 32;   // rows up to this long are searched directly

// Device view passed to kernels by value.
struct DStore {
    const uint32_t* __restrict__ ptr;
    const uint32_t* __restrict__ idx;
    const uint32_t* __restrict__ lab;
    const uint32_t* __restrict__ dir_off;   // NULL: no label directory
    const uint32_t* __restrict__ dir_lab;
    const uint32_t* __restrict__ dir_pos;
};

inline DStore dview(const Store& s) {
    return DStore{s.ptr, s.idx, s.lab, s.dir_off, s.dir_lab, s.dir_pos};
}

}  // namespace gs

struct gs_graph {
    uint32_t N = 0, P = 0;
    uint64_t M = 0;
    gs::Store out;   // rows = subjects, idx = objects
    gs::Store in;    // rows = objects,  idx = subjects
    gs::Alloc alloc;
    int sm_count = 148;
    int n_blocks = 592;
    // grids of the level kernels: as many blocks as fit on the SMs at once
    int range_blocks = 592, expand_blocks = 592;
    int device = 0;
    // streams on which batched evaluations run their grid-path queries
    // side by side (created on first use, destroyed with the graph)
    cudaStream_t side[16] = {};
    int n_side = 0;
    std::atomic<uint32_t> side_rr{0};   // where the next batch starts on the side streams
    std::atomic<int> trace{0};          // grid-path evaluations record per-phase events
    // host copies of the row lengths (out = CSR, in = CSC), used to route
    // queries whose first level is certainly large away from the
    // single-CTA evaluator
    std::vector<uint32_t> deg_out, deg_in;
    // per predicate label l and orientation (0 = CSR, 1 = CSC): entries with
    // label l (lab_cnt) and rows / columns holding it (lab_rows); the
    // memory estimates of queries are made from these
    std::vector<uint64_t> lab_cnt[2], lab_rows[2];
    // per-query host resources kept for reuse: timing events and pinned
    // slots the control-block head of a result is copied into
    std::mutex res_mu;
    std::vector<cudaEvent_t> ev_free;
    std::vector<uint8_t*> head_free;
    std::vector<uint8_t*> head_blocks;
    // device word into which the standalone scan calls OR kStStall
    // (read and cleared by gs_scan_status)
    uint32_t* scan_status = nullptr;
    uint64_t free_seen = 0;   // free device memory at free_seen_at
    std::chrono::steady_clock::time_point free_seen_at{};
};

namespace gs {

// An edge joining the variable w bound at a level to an end that is
// already bound (a variable of an earlier level, or a constant vertex).
struct Binder {
    uint32_t label;
    uint32_t c;          // constant vertex id when from_const
    int16_t level;       // level of the bound variable when !from_const
    uint8_t from_const;
    uint8_t dir;         // 0: w is the object -> candidates in the CSR row of the bound end
                         // 1: w is the subject -> candidates in the CSC column of the bound end
};

// Candidate x of a level must have predicate `label` in its row (dir 0)
// or its column (dir 1): a pre-pruning test (Sec. 7.2.2) for edges whose
// other end is bound later.
struct Probe {
    uint32_t label;
    uint32_t dir;
};

enum : int32_t { kSrcBinders = 0, kSrcList = 1 };

struct LevelSpec {
    int32_t var;
    int32_t src;           // kSrcBinders: candidates from the shortest binder range;
                           // kSrcList: candidates = the variable's compacted candidate vector
    int32_t n_binders;
    int32_t n_probes;
    int32_t n_self;
    int32_t use_bitmap;    // test candidates against the variable's candidate vector
    int32_t vec;           // that vector: bits + vec * words (the level's own index
                           // in an ordinary plan)
    Binder b[kMaxBinders];
    Probe pr[kMaxProbes];
    uint32_t self_label[kMaxSelf];
};

// A variable with exactly one incident pattern whose other end is a
// variable: never materialized, its bindings are the entries of one range
// per tree node, expanded only when the tuples are written.
struct LeafSpec {
    int32_t var;
    int32_t level;       // level of its only neighbour
    uint32_t label;
    uint32_t dir;        // as Binder::dir
};

struct ScanSpec {
    int32_t n_out, n_in;               // distinct predicates tested on rows / columns
    uint32_t out_pred[kMaxSlots];
    uint32_t in_pred[kMaxSlots];
    int32_t n_bvars;                   // candidate vectors produced
    int32_t bvar[kMaxVars];            // which variable each vector belongs to
    int32_t blevel[kMaxVars];          // its level (the vector goes to bits + level * words)
    uint32_t need_out[kMaxVars];       // slot masks that must all be present
    uint32_t need_in[kMaxVars];
};

}  // namespace gs

struct gs_plan {
    uint32_t N = 0, P = 0;
    std::vector<int64_t> patterns;     // n x 3 as given
    int n_vars = 0;
    uint32_t flags = 0;
    // planner output (Sec. 6.1): groups of (vertex, edge indices) and roots;
    // vertex >= 0 is a variable, < 0 is -(1 + constant id)
    std::vector<std::pair<int64_t, std::vector<int>>> groups;
    std::vector<int64_t> roots;
    // schedule for the executor
    int n_levels = 0;
    gs::LevelSpec levels[gs::kMaxLevels];
    int n_leaves = 0;
    gs::LeafSpec leaves[gs::kMaxVars];
    int32_t var_src[gs::kMaxVars];    // >= 0: level of the variable; < 0: -(leaf + 1)
    bool needs_scan = false;
    gs::ScanSpec scan{};
    std::vector<uint32_t> const_triples;   // patterns with two constant ends: s, p, o
    // The two frontier forms of a plan with a triple scan. Bitmap form (the
    // default): every level tests its candidates against its variable's
    // candidate vector. List form: only the levels listed from a candidate
    // vector (roots) get one; the others keep their predicate-presence
    // probes (lookups in label-sorted rows). list_ok: the list form exists
    // (no level has more probes than kMaxProbes).
    bool list_ok = false;
    bool list_form = false;                // levels / scan hold the list form
    // binding-tree paths of Sec. 7.1: variables from a root; step j > 0 is
    // reached from step j - 1 through pattern path_pat[.][j] (-1 at j = 0).
    // A variable no path reaches (its edges all go to constants) is a path
    // of its own.
    std::vector<std::vector<int>> paths, path_pat;
    gs::ScanSpec path_scan{};   // with GS_PLAN_PATHS: one candidate vector per variable
    gs::LevelSpec levels_alt[gs::kMaxLevels];   // the other form's levels
    gs::ScanSpec scan_alt{};                    // the other form's scan
};

namespace gs {
// The plan in the other frontier form (bitmap <-> list); false when the
// plan has no list form.
bool switch_frontier_form(gs_plan* P);
}  // namespace gs

namespace gs {

// store.cu
gs_status build_store(gs_graph* g, const uint32_t* s, const uint32_t* p, const uint32_t* o,
                      uint64_t n, bool on_device, cudaStream_t st);
void free_store(gs_graph* g, cudaStream_t st);
// The triple scan's work items and row-start bitmap of an orientation whose
// ptr / idx / lab (M entries) are built; allocated through g's allocator.
gs_status store_items(const gs_graph* g, Store& S, uint64_t M, cudaStream_t st);
// radix sort of 64-bit keys on bits [lo_bit, hi_bit); keys end up in *keys
// (the buffers may be swapped). tmp must hold n keys.
gs_status radix_sort_u64(const gs_graph* g, uint64_t** keys, uint64_t** tmp, uint64_t n,
                         int lo_bit, int hi_bit, cudaStream_t st);

// scan.cu: candidate vectors (Eq. 17 / Eq. 21) of the variables in spec.
// bits: spec.n_bvars vectors of ceil(N/32) words. work: scan_work_bytes().
// status: a device word into which kStStall is ORed if a bounded wait for
// the bulk copies runs out (never cleared here).
// wide: 32-bit masks (up to kMaxSlotsWide predicates per direction).
size_t scan_work_bytes(const gs_graph* g, bool wide = false);
long long scan_stall_cycles();
// so / si: the orientations to scan (NULL: the graph's own; a per-query
// LSpM otherwise).
gs_status run_scan(const gs_graph* g, const ScanSpec& spec, uint32_t* bits, void* work,
                   cudaStream_t st, uint32_t* status, const Store* so = nullptr,
                   const Store* si = nullptr);

// One candidate vector to write: vertex x is set when its row mask holds
// every slot of need_out and its column mask every slot of need_in.
struct EvalVec {
    uint32_t need_out, need_in;
    uint32_t* dst;    // ceil(N/32) words
};
// The vectors of one k_scan_eval launch: list (device memory, n entries)
// or, when list is NULL, the first n entries of inl.
struct EvalArgs {
    uint32_t n;
    const EvalVec* list;
    EvalVec inl[kMaxVars];
};
// The two halves of run_scan, for scans shared by several queries:
// scan_masks streams both orientations once and leaves per-vertex masks of
// the given predicate slots in work (32-bit masks when either direction has
// more than kMaxSlots predicates, so work must hold scan_work_bytes(g,
// true) then); scan_eval turns them into the vectors of ea.
gs_status scan_masks(const gs_graph* g, const uint32_t* out_pred, uint32_t n_out,
                     const uint32_t* in_pred, uint32_t n_in, void* work, uint32_t* status,
                     cudaStream_t st, const Store* so = nullptr, const Store* si = nullptr);
gs_status scan_eval(const gs_graph* g, const void* work, bool wide, const EvalArgs& ea,
                    cudaStream_t st);
// The ScanSpec of one grouped selection (one candidate vector) from the
// (predicate, direction) list of gs_scan_candidates; `who` names the entry
// point in error messages.
gs_status scan_spec_from(const gs_graph* g, const uint32_t* preds, const uint8_t* dirs,
                         uint32_t n, ScanSpec* out, const char* who);

// plan.cpp
gs_status make_plan(const gs_graph* g, const int64_t* patterns, uint32_t n, uint32_t flags,
                    gs_plan** out);

}  // namespace gs
