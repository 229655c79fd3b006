// Batched evaluation: many queries in one persistent launch (k_batch in
// gs_small.cu). The host packs the schedules of all queries that fit the
// single-block record into one staging buffer (one copy to the device),
// launches one CTA per resident slot; every CTA pulls queries from a device
// counter and evaluates them in its own workspace, writing answers into a
// shared pool. Queries that need the full triple scan or do not fit a
// record run on the grid path from the start, and queries that outgrow the
// per-CTA budgets after the batch kernel; grid-path queries run side by
// side on the graph's side streams, each as an ordinary result.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gs_device.cuh"
#include "gs_exec.h"
#include "gs_qrec.h"

using namespace gs;

struct gs_batch {
    gs_graph* g = nullptr;
    cudaStream_t st = nullptr;
    uint32_t n = 0;
    std::vector<const gs_plan*> plans;
    std::vector<int32_t> n_vars;
    std::vector<uint8_t> in_kernel;        // 1: evaluated by k_batch
    std::vector<uint32_t> kidx;            // kernel index -> query
    uint8_t* dev = nullptr;                // records | offsets | results | counters
    uint8_t* slots = nullptr;
    uint8_t* pool = nullptr;
    uint64_t pool_bytes = 0;
    BatchResult* res_dev = nullptr;
    std::vector<BatchResult> res;
    std::vector<gs_result*> sub;           // grid-path results
    std::vector<uint8_t> staging;          // packed records and offsets (host)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    uint32_t launches = 0, escalated = 0;
    int blocks = 0;
    cudaEvent_t ev_enq = nullptr;          // after everything gs_eval_batch enqueued
    bool ready = false;
    gs_batch_config cfg{};                 // with every default filled in
    uint32_t next_side = 0;                // round robin over the side streams
    uint64_t slot_bytes = 0;
    int stage = 0;                         // 0: batch kernel enqueued, 1: its results read
    std::vector<uint32_t> todo;            // queries waiting for the grid path
    std::vector<uint32_t> active;          // queries on the grid path now
    size_t todo_next = 0;
    // shared triple scans: the pass of each query (-1: none), the candidate
    // vectors a pass wrote for it (owned here until its grid-path result
    // takes them), one completion event and status word per pass
    std::vector<int32_t> pass_of;
    std::vector<uint32_t*> scan_bits;
    std::vector<cudaEvent_t> ev_pass;
    uint32_t* pass_status = nullptr;       // in dev
    void* scan_work = nullptr;
    std::vector<gs_plan> form;             // plans switched to the configured frontier form
    std::vector<int32_t> form_of;          // index into form (-1: the caller's plan)
    uint32_t n_scans = 0, n_scan_plans = 0;
};

namespace {

constexpr uint64_t kBatchCand = 1ull << 16;
constexpr uint64_t kBatchRows = 1ull << 16;
constexpr uint64_t kSlotMax = 24ull << 20;

// Workspace of one CTA: the control block and up to 12 levels of
// cand_budget nodes with their scratch; a query that needs more is handed
// to the grid path.
uint64_t slot_bytes_for(uint64_t cand_budget) {
    return std::min<uint64_t>(kSlotMax, (256ull << 10) + cand_budget * 160);
}
constexpr uint64_t kPoolDefault = 4ull << 30;
constexpr uint32_t kGridStreams = 4;

// Side stream i of the graph, created on first use.
gs_status side_stream(gs_graph* g, uint32_t i, cudaStream_t* out) {
    i %= 16;
    while (g->n_side <= (int)i) {
        GS_CUDA(cudaStreamCreateWithFlags(&g->side[g->n_side], cudaStreamNonBlocking));
        g->n_side++;
    }
    *out = g->side[i];
    return GS_OK;
}

const gs_plan* plan_of(const gs_batch* b, uint32_t q) {
    return b->form_of.empty() || b->form_of[q] < 0 ? b->plans[q] : &b->form[b->form_of[q]];
}

// The grid path for query q on the batch's next side stream (from the
// vectors of its shared scan when it had one).
gs_status grid_query(gs_batch* b, uint32_t q, gs_result** r) {
    cudaStream_t st = nullptr;
    gs_status rc = side_stream(b->g, b->next_side++ % b->cfg.grid_streams, &st);
    if (rc != GS_OK) return rc;
    const gs_plan* plan = plan_of(b, q);
    if (!b->pass_of.empty() && b->pass_of[q] >= 0) {
        uint32_t* bits = b->scan_bits[q];
        b->scan_bits[q] = nullptr;   // the result owns them from here on
        const int ps = b->pass_of[q];
        return eval_query_prescanned(b->g, plan, (void*)st, bits, b->ev_pass[ps], b->pass_status + ps, r);
    }
    return eval_query_path(b->g, plan, (void*)st, 1, r);
}

gs_batch_config resolve(const gs_graph* g, const gs_batch_config* c) {
    gs_batch_config r = c ? *c : gs_batch_config{};
    const int fit = batch_blocks_per_sm();
    if (r.blocks_per_sm == 0) {
        r.blocks_per_sm = (uint32_t)fit;
        if (const char* e = getenv("GS_BATCH_BLOCKS_PER_SM")) r.blocks_per_sm = (uint32_t)std::max(1, atoi(e));
    }
    r.blocks_per_sm = std::max(1u, std::min(r.blocks_per_sm, (uint32_t)fit));
    if (r.grid_streams == 0) r.grid_streams = kGridStreams;
    r.grid_streams = std::min(r.grid_streams, 16u);
    if (r.cand_budget == 0) r.cand_budget = kBatchCand;
    if (r.row_budget == 0) r.row_budget = kBatchRows;
    if (r.scan_share == 0) r.scan_share = 1;
    if (r.frontier == 0) r.frontier = 1;
    if (r.pool_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        r.pool_bytes = std::min<uint64_t>(kPoolDefault, free_b / 4);
        if (const char* e = getenv("GS_BATCH_POOL_BYTES")) r.pool_bytes = strtoull(e, nullptr, 10);
    }
    (void)g;
    return r;
}

// Start grid-path queries from the to-do list while fewer than
// grid_streams run (bounds the workspaces held at once).
gs_status launch_todo(gs_batch* b) {
    while (b->active.size() < b->cfg.grid_streams && b->todo_next < b->todo.size()) {
        const uint32_t q = b->todo[b->todo_next++];
        gs_result* r = nullptr;
        gs_status rc = grid_query(b, q, &r);
        if (rc != GS_OK) return rc;
        b->sub[q] = r;
        b->active.push_back(q);
    }
    return GS_OK;
}

// A grid-path query finished: its count, then its answers compacted.
gs_status retire(gs_batch* b, uint32_t q) {
    uint64_t rows = 0;
    gs_status rc = gs_result_info(b->sub[q], &rows, nullptr);
    if (rc != GS_OK) return rc;
    uint32_t nl = 0;
    gs_result_stats(b->sub[q], nullptr, &nl);
    b->launches += nl;
    b->res[q].rows = rows;
    return result_compact(b->sub[q]);
}

// The batch kernel has finished: read its results and queue the queries it
// handed back.
gs_status collect_kernel(gs_batch* b) {
    const uint32_t nk = (uint32_t)b->kidx.size();
    if (b->res_dev && nk) {
        std::vector<BatchResult> kr(nk);
        GS_CUDA(cudaMemcpy(kr.data(), b->res_dev, sizeof(BatchResult) * nk, cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < nk; ++i) b->res[b->kidx[i]] = kr[i];
    }
    for (uint32_t q = 0; q < b->n; ++q) {
        if (!b->in_kernel[q] || b->res[q].status == 0) continue;
        b->escalated++;
        b->todo.push_back(q);
    }
    b->g->alloc.put(b->slots, b->st);   // the CTA workspaces are done
    b->slots = nullptr;
    b->stage = 1;
    return launch_todo(b);
}

gs_status all_done(gs_batch* b) {
    GS_CUDA(cudaEventRecord(b->ev1, b->st));
    GS_CUDA(cudaEventSynchronize(b->ev1));
    b->ready = true;
    return GS_OK;
}

gs_status finish(gs_batch* b) {
    if (b->ready) return GS_OK;
    if (b->stage == 0) {
        GS_CUDA(cudaStreamSynchronize(b->st));
        gs_status rc = collect_kernel(b);
        if (rc != GS_OK) return rc;
    }
    while (!b->active.empty()) {
        const uint32_t q = b->active.front();
        b->active.erase(b->active.begin());
        gs_status rc = retire(b, q);
        if (rc == GS_OK) rc = launch_todo(b);
        if (rc != GS_OK) return rc;
    }
    return all_done(b);
}

void release(gs_batch* b) {
    if (!b) return;
    if (b->st || b->g) cudaStreamSynchronize(b->st);
    for (gs_result* r : b->sub) gs_free_result(r);
    if (b->g) {
        b->g->alloc.put(b->dev, b->st);
        b->g->alloc.put(b->slots, b->st);
        b->g->alloc.put(b->pool, b->st);
        b->g->alloc.put(b->scan_work, b->st);
        for (uint32_t* bits : b->scan_bits) b->g->alloc.put(bits, b->st);
    }
    for (cudaEvent_t e : b->ev_pass) cudaEventDestroy(e);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->ev_enq) cudaEventDestroy(b->ev_enq);
    delete b;
}

// One shared triple scan: the union of its plans' predicates per direction
// and, per plan, its vectors with their slot masks renumbered into the union.
struct Pass {
    std::vector<uint32_t> out_pred, in_pred;
    std::vector<uint32_t> queries;
};

// Slot of predicate p in list (appended when absent and room is left).
int union_slot(std::vector<uint32_t>& list, uint32_t p, bool add) {
    for (size_t j = 0; j < list.size(); ++j)
        if (list[j] == p) return (int)j;
    if (!add || list.size() >= (size_t)kMaxSlotsWide) return -1;
    list.push_back(p);
    return (int)list.size() - 1;
}

// Does plan P fit into pass x (adding its predicates when it does)?
// Slots the plan would add to pass x (SIZE_MAX when it does not fit).
size_t pass_cost(Pass& x, const ScanSpec& S) {
    size_t new_out = 0, new_in = 0;
    for (int i = 0; i < S.n_out; ++i) new_out += union_slot(x.out_pred, S.out_pred[i], false) < 0;
    for (int i = 0; i < S.n_in; ++i) new_in += union_slot(x.in_pred, S.in_pred[i], false) < 0;
    if (x.out_pred.size() + new_out > (size_t)kMaxSlotsWide ||
        x.in_pred.size() + new_in > (size_t)kMaxSlotsWide)
        return SIZE_MAX;
    return new_out + new_in;
}

void pass_take(Pass& x, const ScanSpec& S) {
    for (int i = 0; i < S.n_out; ++i) union_slot(x.out_pred, S.out_pred[i], true);
    for (int i = 0; i < S.n_in; ++i) union_slot(x.in_pred, S.in_pred[i], true);
}

// A plan's slot mask renumbered from its own slots into the pass's.
uint32_t remap(uint32_t need, const uint32_t* own, std::vector<uint32_t>& uni) {
    uint32_t m = 0;
    for (int i = 0; need >> i; ++i)
        if ((need >> i) & 1u) m |= 1u << union_slot(uni, own[i], false);
    return m;
}

}  // namespace

extern "C" {

gs_status gs_eval_batch(gs_graph* g, const gs_plan* const* plans, uint32_t n, void* cuda_stream,
                        gs_batch** out) {
    return eval_batch_ex(g, plans, n, cuda_stream, nullptr, 0, out);
}

gs_status gs_eval_batch_cfg(gs_graph* g, const gs_plan* const* plans, uint32_t n,
                            const gs_batch_config* cfg, void* cuda_stream, gs_batch** out) {
    return eval_batch_ex(g, plans, n, cuda_stream, cfg, 0, out);
}

}  // extern "C"

gs_status gs::eval_batch_ex(gs_graph* g, const gs_plan* const* plans, uint32_t n, void* cuda_stream,
                            const gs_batch_config* cfg, int max_blocks, gs_batch** out) {
    if (!g || !out || (n && !plans)) { set_error("gs_eval_batch: NULL argument"); return GS_EINVAL; }
    *out = nullptr;
    NvtxRange nv("gs_eval_batch: pack and launch");
    for (uint32_t q = 0; q < n; ++q) {
        if (!plans[q]) { set_error("gs_eval_batch: plan %u is NULL", q); return GS_EINVAL; }
        if (plans[q]->N != 0 && (plans[q]->N != g->N || plans[q]->P != g->P)) {
            set_error("gs_eval_batch: plan %u was made for another graph", q);
            return GS_EINVAL;
        }
    }
    gs_batch* b = new (std::nothrow) gs_batch();
    if (!b) { set_error("gs_eval_batch: host out of memory"); return GS_ENOMEM; }
    b->g = g;
    b->st = (cudaStream_t)cuda_stream;
    b->n = n;
    b->cfg = resolve(g, cfg);
    // batches that run at once (a server's) spread over the side streams
    b->next_side = g->side_rr.fetch_add(b->cfg.grid_streams);
    b->plans.assign(plans, plans + n);
    b->n_vars.resize(n);
    b->in_kernel.assign(n, 0);
    b->res.assign(n, BatchResult{0, 0, 0, 0});
    b->sub.assign(n, nullptr);
    // plans in the configured frontier form (a copy when it differs)
    b->form_of.assign(n, -1);
    for (uint32_t q = 0; q < n; ++q) {
        const gs_plan* P = plans[q];
        if (P->needs_scan && P->list_ok && P->list_form != (b->cfg.frontier == 2)) {
            b->form_of[q] = (int32_t)b->form.size();
            b->form.push_back(*P);
        }
    }
    for (gs_plan& P : b->form) switch_frontier_form(&P);
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_enq, cudaEventDisableTiming) != cudaSuccess) {
        gs_status rc = cuda_fail(cudaGetLastError(), "cudaEventCreate");
        release(b);
        return rc;
    }
    // pack records
    std::vector<uint64_t> off(n, 0);
    uint64_t total = 0;
    uint32_t n_in = 0;
    for (uint32_t q = 0; q < n; ++q) {
        b->n_vars[q] = plans[q]->n_vars;
        // a first level certainly past the candidate budget goes to the grid path
        if (batch_in_kernel(g, plans[q], &b->cfg)) {
            b->in_kernel[q] = 1;
            off[n_in] = total;
            b->kidx.push_back(q);
            total += sizeof(QHdr) + plans[q]->n_levels * sizeof(LevelSpec) +
                     plans[q]->n_leaves * sizeof(LeafSpec) + 16;
            total = (total + 15) & ~15ull;
            ++n_in;
        }
    }
    // plans that need a triple scan: packed into shared passes, each plan
    // into the pass it adds the fewest new predicates to (the earliest on a
    // tie; a plan whose predicates a pass already tests costs nothing), a
    // new pass when none has room (kMaxSlotsWide per direction)
    std::vector<Pass> passes;
    std::vector<EvalVec> vecs;           // every pass's vectors, pass by pass
    std::vector<uint32_t> vec_off;       // first vector of each pass
    if (b->cfg.scan_share == 1) {
        b->pass_of.assign(n, -1);
        b->scan_bits.assign(n, nullptr);
        for (uint32_t q = 0; q < n; ++q) {
            const gs_plan* P = plan_of(b, q);
            if (b->in_kernel[q] || !P->needs_scan) continue;
            size_t best = SIZE_MAX, at = passes.size();
            for (size_t k = 0; k < passes.size() && best > 0; ++k) {
                const size_t c = pass_cost(passes[k], P->scan);
                if (c < best) { best = c; at = k; }
            }
            if (at == passes.size()) passes.emplace_back();
            pass_take(passes[at], P->scan);
            passes[at].queries.push_back(q);
            b->pass_of[q] = (int32_t)at;
        }
        const uint64_t words = (g->N + 31) / 32;
        for (Pass& x : passes) {
            vec_off.push_back((uint32_t)vecs.size());
            for (uint32_t q : x.queries) {
                const gs_plan* P = plan_of(b, q);
                uint32_t* bits = (uint32_t*)g->alloc.get(4 * words * std::max(1, P->n_levels), b->st);
                if (!bits) { set_error("gs_eval_batch: out of device memory for candidate vectors"); release(b); return GS_ENOMEM; }
                b->scan_bits[q] = bits;
                const ScanSpec& S = P->scan;
                for (int u = 0; u < S.n_bvars; ++u)
                    vecs.push_back(EvalVec{remap(S.need_out[u], S.out_pred, x.out_pred),
                                           remap(S.need_in[u], S.in_pred, x.in_pred),
                                           bits + (uint64_t)S.blevel[u] * words});
            }
        }
        b->n_scans = (uint32_t)passes.size();
        for (const Pass& x : passes) b->n_scan_plans += (uint32_t)x.queries.size();
    }
    const uint64_t n_pass = passes.size();
    const uint64_t off_bytes = 8ull * n_in, res_bytes = sizeof(BatchResult) * (uint64_t)n_in;
    const uint64_t ctr_bytes = 64 + ((4 * n_pass + 63) & ~63ull);   // counters | pass status words
    const uint64_t vec_at = total + off_bytes + res_bytes + ctr_bytes;
    const uint64_t dev_bytes = vec_at + sizeof(EvalVec) * vecs.size() + 256;
    b->staging.assign(total + off_bytes + 16, 0);
    for (uint32_t i = 0; i < n_in; ++i) pack_record(plans[b->kidx[i]], b->staging.data() + off[i]);
    std::memcpy(b->staging.data() + total, off.data(), off_bytes);
    b->dev = (uint8_t*)g->alloc.get(dev_bytes, b->st);
    int blocks = g->sm_count * (int)b->cfg.blocks_per_sm;
    if (max_blocks > 0) blocks = std::min(blocks, max_blocks);
    blocks = std::max(1, std::min<int>(blocks, (int)std::max<uint32_t>(1, n_in)));
    b->blocks = blocks;
    b->slot_bytes = slot_bytes_for(b->cfg.cand_budget);
    b->slots = (uint8_t*)g->alloc.get(b->slot_bytes * blocks, b->st);
    b->pool_bytes = b->cfg.pool_bytes;
    b->pool = (uint8_t*)g->alloc.get(std::max<uint64_t>(b->pool_bytes, 256), b->st);
    if (!b->dev || !b->slots || !b->pool) {
        set_error("gs_eval_batch: out of device memory");
        release(b);
        return GS_ENOMEM;
    }
    gs_status rc = GS_OK;
    cudaError_t e = cudaEventRecord(b->ev0, b->st);
    if (e == cudaSuccess)
        // from pageable memory: the call returns once the bytes are staged
        e = cudaMemcpyAsync(b->dev, b->staging.data(), total + off_bytes, cudaMemcpyHostToDevice, b->st);
    b->res_dev = (BatchResult*)(b->dev + total + off_bytes);
    uint32_t* counters = (uint32_t*)(b->dev + total + off_bytes + res_bytes);
    b->pass_status = counters + 16;
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, ctr_bytes, b->st);
    if (e == cudaSuccess && !vecs.empty())
        e = cudaMemcpyAsync(b->dev + vec_at, vecs.data(), sizeof(EvalVec) * vecs.size(),
                            cudaMemcpyHostToDevice, b->st);
    if (e != cudaSuccess) rc = cuda_fail(e, "gs_eval_batch");
    if (rc == GS_OK && n_in) {
        BatchDev B{};
        B.out = dview(g->out);
        B.in = dview(g->in);
        B.recs = b->dev;
        B.rec_off = (const uint64_t*)(b->dev + total);
        B.n = n_in;
        B.slots = b->slots;
        B.slot_bytes = b->slot_bytes;
        (void)0;
        B.pool = b->pool;
        B.pool_bytes = b->pool_bytes;
        B.pool_top = (unsigned long long*)(counters + 2);
        B.next = counters;
        B.res = b->res_dev;
        B.cand_budget = b->cfg.cand_budget;
        B.row_budget = b->cfg.row_budget;
        rc = enqueue_batch(B, blocks, b->st);
        b->launches = 1;
    }
    // the shared scans, one after another on the batch's stream; the
    // queries of a pass start on the side streams once its event is reached
    bool wide_any = false;
    for (const Pass& x : passes)
        wide_any |= x.out_pred.size() > (size_t)kMaxSlots || x.in_pred.size() > (size_t)kMaxSlots;
    if (rc == GS_OK && n_pass) {
        b->scan_work = g->alloc.get(scan_work_bytes(g, wide_any), b->st);
        if (!b->scan_work) { set_error("gs_eval_batch: out of device memory for the triple scan"); rc = GS_ENOMEM; }
    }
    for (size_t i = 0; i < passes.size() && rc == GS_OK; ++i) {
        const Pass& x = passes[i];
        const bool wide = x.out_pred.size() > (size_t)kMaxSlots || x.in_pred.size() > (size_t)kMaxSlots;
        rc = scan_masks(g, x.out_pred.data(), (uint32_t)x.out_pred.size(), x.in_pred.data(),
                        (uint32_t)x.in_pred.size(), b->scan_work, b->pass_status + i, b->st);
        if (rc != GS_OK) break;
        EvalArgs ea{};
        ea.n = (i + 1 < passes.size() ? vec_off[i + 1] : (uint32_t)vecs.size()) - vec_off[i];
        ea.list = (const EvalVec*)(b->dev + vec_at) + vec_off[i];
        rc = scan_eval(g, b->scan_work, wide, ea, b->st);
        if (rc != GS_OK) break;
        cudaEvent_t ev = nullptr;
        cudaError_t e3 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e3 == cudaSuccess) e3 = cudaEventRecord(ev, b->st);
        if (ev) b->ev_pass.push_back(ev);
        if (e3 != cudaSuccess) rc = cuda_fail(e3, "gs_eval_batch");
        b->launches += 3;
    }
    // plans outside the record format go straight to the grid path, beside
    // the batch kernel
    for (uint32_t q = 0; q < n; ++q)
        if (!b->in_kernel[q]) b->todo.push_back(q);
    if (rc == GS_OK) rc = launch_todo(b);
    if (rc == GS_OK) {
        cudaError_t e2 = cudaEventRecord(b->ev_enq, b->st);
        if (e2 != cudaSuccess) rc = cuda_fail(e2, "gs_eval_batch");
    }
    if (rc != GS_OK) { release(b); return rc; }
    *out = b;
    return GS_OK;
}

uint64_t gs::batch_device_bytes(const gs_batch* b) {
    return b->slot_bytes * (uint64_t)b->blocks + b->pool_bytes;
}

bool gs::batch_in_kernel(const gs_graph* g, const gs_plan* P, const gs_batch_config* cfg) {
    const uint64_t cand = cfg && cfg->cand_budget ? cfg->cand_budget : kBatchCand;
    // a first level certainly past the candidate budget goes to the grid path
    return rec_fits(P) && first_level_bound(g, P) <= 8 * cand;
}

uint64_t gs::batch_fixed_bytes(const gs_graph* g, const gs_batch_config* cfg, uint32_t n_kernel,
                               bool has_scan) {
    const uint32_t fit = (uint32_t)batch_blocks_per_sm();
    const uint32_t bps = cfg && cfg->blocks_per_sm ? std::min(cfg->blocks_per_sm, fit) : fit;
    const uint64_t cand = cfg && cfg->cand_budget ? cfg->cand_budget : kBatchCand;
    const uint64_t blocks = std::min<uint64_t>(n_kernel, (uint64_t)g->sm_count * std::max(1u, bps));
    return blocks * slot_bytes_for(cand) + (has_scan ? scan_work_bytes(g, true) : 0);
}

gs_status gs::batch_advance(gs_batch* b, int* done) {
    *done = 0;
    if (b->ready) { *done = 1; return GS_OK; }
    if (b->stage == 0) {
        cudaError_t e = cudaEventQuery(b->ev_enq);
        if (e == cudaErrorNotReady) return GS_OK;
        if (e != cudaSuccess) return cuda_fail(e, "gs_eval_batch");
        gs_status rc = collect_kernel(b);
        if (rc != GS_OK) return rc;
    }
    for (size_t i = 0; i < b->active.size();) {
        int d = 0;
        gs_status rc = result_ready(b->sub[b->active[i]], &d);
        if (rc != GS_OK) return rc;
        if (!d) { ++i; continue; }
        const uint32_t q = b->active[i];
        b->active.erase(b->active.begin() + i);
        rc = retire(b, q);
        if (rc == GS_OK) rc = launch_todo(b);
        if (rc != GS_OK) return rc;
    }
    if (!b->active.empty() || b->todo_next < b->todo.size()) return GS_OK;
    gs_status rc = all_done(b);
    if (rc != GS_OK) return rc;
    *done = 1;
    return GS_OK;
}

extern "C" {

gs_status gs_batch_scans(gs_batch* b, uint32_t* n_scans, uint32_t* n_scan_plans) {
    if (!b) { set_error("gs_batch_scans: batch is NULL"); return GS_EINVAL; }
    uint32_t own = 0;   // plans outside the shared passes run a scan each
    for (uint32_t q = 0; q < b->n; ++q)
        if (!b->in_kernel[q] && plan_of(b, q)->needs_scan && (b->pass_of.empty() || b->pass_of[q] < 0)) ++own;
    if (n_scans) *n_scans = b->n_scans + own;
    if (n_scan_plans) *n_scan_plans = b->n_scan_plans + own;
    return GS_OK;
}

gs_status gs_batch_poll(gs_batch* b, int* done) {
    if (!b || !done) { set_error("gs_batch_poll: NULL argument"); return GS_EINVAL; }
    if (b->ready) { *done = 1; return GS_OK; }
    cudaError_t e = cudaEventQuery(b->ev_enq);
    if (e == cudaErrorNotReady) { *done = 0; return GS_OK; }
    if (e != cudaSuccess) return cuda_fail(e, "gs_batch_poll");
    *done = 1;   // the launch finished; gs_batch_info completes any hand-backs
    return GS_OK;
}

gs_status gs_batch_info(gs_batch* b, uint64_t* rows, uint64_t* total_rows) {
    if (!b) { set_error("gs_batch_info: batch is NULL"); return GS_EINVAL; }
    gs_status rc = finish(b);
    if (rc != GS_OK) return rc;
    uint64_t t = 0;
    for (uint32_t q = 0; q < b->n; ++q) {
        if (rows) rows[q] = b->res[q].rows;
        t += b->res[q].rows;
    }
    if (total_rows) *total_rows = t;
    return GS_OK;
}

gs_status gs_batch_fetch(gs_batch* b, uint32_t q, int32_t* dst, uint64_t cap_rows, int dst_on_device,
                         int sort_rows) {
    if (!b) { set_error("gs_batch_fetch: batch is NULL"); return GS_EINVAL; }
    if (q >= b->n) { set_error("gs_batch_fetch: query %u of %u", q, b->n); return GS_EINVAL; }
    gs_status rc = finish(b);
    if (rc != GS_OK) return rc;
    if (b->sub[q]) return gs_fetch_bindings(b->sub[q], dst, cap_rows, dst_on_device, sort_rows);
    const uint64_t rows = b->res[q].rows;
    if (cap_rows < rows) {
        set_error("gs_batch_fetch: buffer holds %llu rows, the answer has %llu",
                  (unsigned long long)cap_rows, (unsigned long long)rows);
        return GS_EOVERFLOW;
    }
    if (rows == 0) return GS_OK;
    if (!dst) { set_error("gs_batch_fetch: dst is NULL"); return GS_EINVAL; }
    const uint32_t k = (uint32_t)b->n_vars[q];
    const uint64_t bytes = 4ull * rows * k;
    const int32_t* src = (const int32_t*)(b->pool + b->res[q].off);
    cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (sort_rows && rows > 1) {
        int32_t* tmp = (int32_t*)b->g->alloc.get(bytes, b->st);
        if (!tmp) { set_error("gs_batch_fetch: out of device memory for sorting"); return GS_ENOMEM; }
        rc = sort_rows_on_device(b->g, src, rows, k, tmp, b->st);
        if (rc == GS_OK) {
            cudaError_t e = cudaMemcpyAsync(dst, tmp, bytes, kind, b->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
            if (e != cudaSuccess) rc = cuda_fail(e, "gs_batch_fetch copy");
        }
        b->g->alloc.put(tmp, b->st);
        cudaStreamSynchronize(b->st);
        return rc;
    }
    GS_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, b->st));
    GS_CUDA(cudaStreamSynchronize(b->st));
    return GS_OK;
}

gs_status gs_batch_stats(gs_batch* b, float* device_ms, uint32_t* kernel_launches,
                         uint32_t* n_escalated) {
    if (!b) { set_error("gs_batch_stats: batch is NULL"); return GS_EINVAL; }
    gs_status rc = finish(b);
    if (rc != GS_OK) return rc;
    if (device_ms) GS_CUDA(cudaEventElapsedTime(device_ms, b->ev0, b->ev1));
    if (kernel_launches) *kernel_launches = b->launches;
    if (n_escalated) *n_escalated = b->escalated;
    return GS_OK;
}

void gs_free_batch(gs_batch* b) { release(b); }

}  // extern "C"

namespace {

// Wall time of one batched evaluation of the plans under cfg (enqueue to
// the last answer count), or a negative value on failure; *handed gets the
// queries handed to the grid path.
double time_batch(gs_graph* g, const gs_plan* const* plans, uint32_t n, const gs_batch_config& cfg,
                  void* stream, gs_status* rc, uint32_t* handed = nullptr) {
    cudaStreamSynchronize((cudaStream_t)stream);
    const auto t0 = std::chrono::steady_clock::now();
    gs_batch* b = nullptr;
    *rc = eval_batch_ex(g, plans, n, stream, &cfg, 0, &b);
    if (*rc != GS_OK) return -1.0;
    *rc = gs_batch_info(b, nullptr, nullptr);
    const auto t1 = std::chrono::steady_clock::now();
    if (*rc == GS_OK && handed) *rc = gs_batch_stats(b, nullptr, nullptr, handed);
    gs_free_batch(b);
    if (*rc != GS_OK) return -1.0;
    return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

}  // namespace

namespace {

// Autotuner choices kept for the life of the process, keyed by the device,
// the graph's sizes and the sample's shape classes.
std::mutex g_tune_mu;
std::map<std::string, std::pair<gs_batch_config, float>> g_tune_cache;

// Shape class of a plan: scan or seeded, frontier form available, levels,
// leaves.
std::string tune_key(const gs_graph* g, const gs_plan* const* plans, uint32_t n) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, g->device);
    cudaGetLastError();
    std::map<std::string, uint32_t> classes;
    for (uint32_t q = 0; q < n; ++q) {
        const gs_plan* P = plans[q];
        char c[64];
        snprintf(c, sizeof(c), "%c%c%d.%d", P->needs_scan ? 'S' : 'C', P->list_ok ? 'l' : '-',
                 P->n_levels, P->n_leaves);
        classes[c]++;
    }
    std::string k = std::string(prop.name) + "|N" + std::to_string(g->N) + "|M" +
                    std::to_string(g->M) + "|P" + std::to_string(g->P);
    for (auto& kv : classes) k += "|" + kv.first + "x" + std::to_string(kv.second);
    return k;
}

}  // namespace

extern "C" gs_status gs_batch_autotune(gs_graph* g, const gs_plan* const* plans, uint32_t n,
                                       void* cuda_stream, gs_batch_config* best, float* best_ms) {
    if (!g || !best || (n && !plans)) { set_error("gs_batch_autotune: NULL argument"); return GS_EINVAL; }
    const std::string key = tune_key(g, plans, n);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second.first;
            if (best_ms) *best_ms = it->second.second;
            return GS_OK;
        }
    }
    const uint32_t fit = (uint32_t)batch_blocks_per_sm();
    std::vector<uint32_t> bps = {1u, 2u, fit};
    std::sort(bps.begin(), bps.end());
    bps.erase(std::unique(bps.begin(), bps.end()), bps.end());
    bps.erase(std::remove_if(bps.begin(), bps.end(), [&](uint32_t x) { return x > fit; }), bps.end());
    const uint64_t cands[] = {1ull << 12, 1ull << 16};
    const uint64_t rows[] = {1ull << 12, 1ull << 16, 1ull << 20};
    bool scans = false, lists = false;
    for (uint32_t q = 0; q < n; ++q) {
        scans |= plans[q]->needs_scan;
        lists |= plans[q]->list_ok;
    }
    gs_batch_config cfg{};
    gs_status rc = GS_OK;
    time_batch(g, plans, n, cfg, cuda_stream, &rc);   // warm-up (allocator, streams)
    if (rc != GS_OK) return rc;
    // Among configurations within 3% of the fastest, the one that hands the
    // fewest queries to the grid path wins: each hand-back costs host work
    // (a plan copy, an estimate, a dozen launches) that one timed batch
    // barely shows but a stream of small served batches pays every time.
    double best_t = -1.0;
    uint32_t best_h = 0;
    auto consider = [&](const gs_batch_config& c) -> gs_status {
        double t = -1.0;
        uint32_t h = 0;
        for (int rep = 0; rep < 2; ++rep) {
            uint32_t hx = 0;
            const double x = time_batch(g, plans, n, c, cuda_stream, &rc, &hx);
            if (rc != GS_OK) return rc;
            if (t < 0 || x < t) { t = x; h = hx; }
        }
        const bool faster = best_t < 0 || t < 0.97 * best_t;
        const bool close = best_t >= 0 && t <= 1.03 * best_t;
        if (faster || (close && (h < best_h || (h == best_h && t < best_t)))) {
            best_t = t;
            best_h = h;
            *best = c;
        }
        return GS_OK;
    };
    // stage 1: CTAs per SM x candidate budget x row budget (single-CTA path)
    for (uint32_t bp : bps)
        for (uint64_t cb : cands)
            for (uint64_t rb : rows) {
                cfg = gs_batch_config{};
                cfg.blocks_per_sm = bp;
                cfg.cand_budget = cb;
                cfg.row_budget = rb;
                if (consider(cfg) != GS_OK) return rc;
            }
    // stage 2, for samples with triple scans: shared or per-plan scans x
    // bitmap or list frontier x grid-path queries side by side, under the
    // stage-1 choice
    if (scans) {
        const gs_batch_config base = *best;
        for (uint32_t share : {1u, 2u})
            for (uint32_t fr : {1u, 2u})
                for (uint32_t gsn : {kGridStreams, 16u}) {
                    if (fr == 2 && !lists) continue;
                    cfg = base;
                    cfg.scan_share = share;
                    cfg.frontier = fr;
                    cfg.grid_streams = gsn;
                    if (consider(cfg) != GS_OK) return rc;
                }
    }
    if (best->grid_streams == 0) best->grid_streams = kGridStreams;
    if (best->scan_share == 0) best->scan_share = 1;
    if (best->frontier == 0) best->frontier = 1;
    if (best_ms) *best_ms = (float)best_t;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {*best, (float)best_t};
    return GS_OK;
}
