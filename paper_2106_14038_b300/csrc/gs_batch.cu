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
#include <cstdlib>
#include <cstring>
#include <new>
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

// The grid path for plan on the batch's next side stream.
gs_status grid_query(gs_batch* b, const gs_plan* plan, gs_result** r) {
    cudaStream_t st = nullptr;
    gs_status rc = side_stream(b->g, b->next_side++ % b->cfg.grid_streams, &st);
    if (rc != GS_OK) return rc;
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
        gs_status rc = grid_query(b, b->plans[q], &r);
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
    }
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->ev_enq) cudaEventDestroy(b->ev_enq);
    delete b;
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
    b->plans.assign(plans, plans + n);
    b->n_vars.resize(n);
    b->in_kernel.assign(n, 0);
    b->res.assign(n, BatchResult{0, 0, 0, 0});
    b->sub.assign(n, nullptr);
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
        if (rec_fits(plans[q]) && first_level_bound(g, plans[q]) <= 8 * b->cfg.cand_budget) {
            b->in_kernel[q] = 1;
            off[n_in] = total;
            b->kidx.push_back(q);
            total += sizeof(QHdr) + plans[q]->n_levels * sizeof(LevelSpec) +
                     plans[q]->n_leaves * sizeof(LeafSpec) + 16;
            total = (total + 15) & ~15ull;
            ++n_in;
        }
    }
    const uint64_t off_bytes = 8ull * n_in, res_bytes = sizeof(BatchResult) * (uint64_t)n_in;
    const uint64_t dev_bytes = total + off_bytes + res_bytes + 256;
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
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 64, b->st);
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

uint64_t gs::batch_estimate(const gs_graph* g, const gs_batch_config* cfg, uint32_t n,
                            uint64_t pool_bytes) {
    const gs_batch_config c = resolve(g, cfg);
    const uint64_t blocks = std::min<uint64_t>(n, (uint64_t)g->sm_count * c.blocks_per_sm);
    // plus the grid-path queries it may run at once (workspace and scan masks)
    const uint64_t grid = (uint64_t)c.grid_streams * ((512ull << 20) + scan_work_bytes(g));
    return blocks * slot_bytes_for(c.cand_budget) + pool_bytes + grid;
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
// the last answer count), or a negative value on failure.
double time_batch(gs_graph* g, const gs_plan* const* plans, uint32_t n, const gs_batch_config& cfg,
                  void* stream, gs_status* rc) {
    cudaStreamSynchronize((cudaStream_t)stream);
    const auto t0 = std::chrono::steady_clock::now();
    gs_batch* b = nullptr;
    *rc = eval_batch_ex(g, plans, n, stream, &cfg, 0, &b);
    if (*rc != GS_OK) return -1.0;
    *rc = gs_batch_info(b, nullptr, nullptr);
    const auto t1 = std::chrono::steady_clock::now();
    gs_free_batch(b);
    if (*rc != GS_OK) return -1.0;
    return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

}  // namespace

extern "C" gs_status gs_batch_autotune(gs_graph* g, const gs_plan* const* plans, uint32_t n,
                                       void* cuda_stream, gs_batch_config* best, float* best_ms) {
    if (!g || !best || (n && !plans)) { set_error("gs_batch_autotune: NULL argument"); return GS_EINVAL; }
    const uint32_t fit = (uint32_t)batch_blocks_per_sm();
    std::vector<uint32_t> bps = {1u, 2u, fit};
    std::sort(bps.begin(), bps.end());
    bps.erase(std::unique(bps.begin(), bps.end()), bps.end());
    bps.erase(std::remove_if(bps.begin(), bps.end(), [&](uint32_t x) { return x > fit; }), bps.end());
    const uint64_t cands[] = {1ull << 12, 1ull << 16};
    const uint64_t rows[] = {1ull << 12, 1ull << 16, 1ull << 20};
    gs_batch_config cfg{};
    gs_status rc = GS_OK;
    time_batch(g, plans, n, cfg, cuda_stream, &rc);   // warm-up (allocator, streams)
    if (rc != GS_OK) return rc;
    double best_t = -1.0;
    for (uint32_t bp : bps)
        for (uint64_t cb : cands)
            for (uint64_t rb : rows) {
                cfg = gs_batch_config{};
                cfg.blocks_per_sm = bp;
                cfg.cand_budget = cb;
                cfg.row_budget = rb;
                double t = -1.0;
                for (int rep = 0; rep < 2; ++rep) {
                    const double x = time_batch(g, plans, n, cfg, cuda_stream, &rc);
                    if (rc != GS_OK) return rc;
                    if (t < 0 || x < t) t = x;
                }
                if (best_t < 0 || t < best_t) {
                    best_t = t;
                    *best = cfg;
                }
            }
    best->grid_streams = kGridStreams;
    if (best_ms) *best_ms = (float)best_t;
    return GS_OK;
}
