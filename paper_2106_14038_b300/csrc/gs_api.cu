// The C ABI (include/gsmart.h): argument checks, object lifetimes, the
// workspace retry loop and the device row sort used by gs_fetch_bindings.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>

#include "gs_device.cuh"
#include "gs_exec.h"

namespace gs {
const char* last_error();
}

using namespace gs;

namespace gs {

// ---- device row sort (lexicographic, LSD over columns) ----

__global__ void k_sort_keys(const int32_t* __restrict__ rows, uint32_t k, uint32_t c, uint64_t n,
                            uint64_t* __restrict__ keys, int first) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t perm = first ? i : (keys[i] & 0xffffffffull);
        uint32_t v = (uint32_t)rows[perm * k + c];
        keys[i] = ((uint64_t)v << 32) | perm;
    }
}

__global__ void k_sort_gather(const int32_t* __restrict__ rows, uint32_t k, uint64_t n,
                              const uint64_t* __restrict__ keys, int32_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t perm = keys[i] & 0xffffffffull;
        for (uint32_t j = 0; j < k; ++j) out[i * k + j] = rows[perm * k + j];
    }
}

gs_status sort_rows_on_device(const gs_graph* g, const int32_t* rows, uint64_t n, uint32_t k,
                        int32_t* out, cudaStream_t st) {
    if (n >= (1ull << 32)) { set_error("gs_fetch_bindings: sorting needs fewer than 2^32 rows"); return GS_ENOTIMPL; }
    uint64_t* k0 = (uint64_t*)g->alloc.get(8 * n, st);
    uint64_t* k1 = (uint64_t*)g->alloc.get(8 * n, st);
    if (!k0 || !k1) { g->alloc.put(k0, st); g->alloc.put(k1, st); set_error("gs_fetch_bindings: out of device memory for sorting"); return GS_ENOMEM; }
    const int nb = g->n_blocks;
    gs_status rc = GS_OK;
    for (int c = (int)k - 1; c >= 0 && rc == GS_OK; --c) {
        k_sort_keys<<<nb, kThreads, 0, st>>>(rows, k, (uint32_t)c, n, k0, c == (int)k - 1);
        rc = radix_sort_u64(g, &k0, &k1, n, 32, 64, st);
    }
    if (rc == GS_OK) k_sort_gather<<<nb, kThreads, 0, st>>>(rows, k, n, k0, out);
    cudaError_t e = cudaGetLastError();
    g->alloc.put(k0, st);
    g->alloc.put(k1, st);
    if (rc == GS_OK && e != cudaSuccess) rc = cuda_fail(e, "row sort");
    return rc;
}

}  // namespace gs

struct gs_result {
    gs_graph* g = nullptr;
    gs_plan plan;
    cudaStream_t st = nullptr;
    uint8_t* arena = nullptr;
    uint64_t arena_bytes = 0;
    uint32_t* bits = nullptr;
    void* work = nullptr;
    uint32_t* lists = nullptr;
    uint64_t list_stride = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the kernels
    cudaEvent_t ev2 = nullptr;                 // the head copy has landed
    uint8_t* head = nullptr;  // pinned copy of the control block's head
    bool ready = false;
    int mode = 0;             // 0: grid path, 1: single-block kernel
    int resume = 0;           // grid path: first level to build (the ones before are in the arena)
    // candidate vectors written by a triple scan shared with other queries:
    // its completion event and status word (NULL: the query scans itself)
    cudaEvent_t scan_ready = nullptr;
    const uint32_t* scan_status = nullptr;
    // the orientations evaluated against (a per-query LSpM; NULL: the graph's)
    const Store* so = nullptr;
    const Store* si = nullptr;
    bool bits_borrowed = false;   // bits belong to the caller (per-path evaluation)
    bool root_cut = false;        // only roots in [root_lo, root_hi) (gs_eval_query_roots)
    uint32_t root_lo = 0, root_hi = 0;
    std::vector<uint64_t> path_nodes;   // per-path mode: binding-tree nodes of each path
    std::vector<cudaEvent_t> phase_ev;  // traced grid-path evaluation: after setup + scan, each level, enumeration
    uint32_t launches = 0;
    uint64_t rows = 0;
    uint64_t out_off = 0;
};

namespace {

constexpr uint64_t kHeadSlot = (kCtlHead + 127) & ~127ull;
constexpr uint32_t kHeadSlotsPerBlock = 256;

// The events and the pinned head slot of a result, from the graph's pools.
gs_status take_host_res(gs_graph* g, cudaEvent_t* ev[3], uint8_t** head) {
    std::lock_guard<std::mutex> lk(g->res_mu);
    for (int i = 0; i < 3; ++i) {
        cudaEvent_t* e = ev[i];
        if (!g->ev_free.empty()) { *e = g->ev_free.back(); g->ev_free.pop_back(); }
        else GS_CUDA(cudaEventCreate(e));
    }
    if (g->head_free.empty()) {
        uint8_t* blk = nullptr;
        GS_CUDA(cudaMallocHost(&blk, kHeadSlot * kHeadSlotsPerBlock));
        g->head_blocks.push_back(blk);
        for (uint32_t i = 0; i < kHeadSlotsPerBlock; ++i) g->head_free.push_back(blk + i * kHeadSlot);
    }
    *head = g->head_free.back();
    g->head_free.pop_back();
    return GS_OK;
}

// Free device memory as last seen, looked up again when older than 0.2 s
// (the query needs only its order of magnitude).
uint64_t free_device_bytes(gs_graph* g) {
    std::lock_guard<std::mutex> lk(g->res_mu);
    const auto now = std::chrono::steady_clock::now();
    if (g->free_seen == 0 || now - g->free_seen_at > std::chrono::milliseconds(200)) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) cudaGetLastError();
        g->free_seen = free_b;
        g->free_seen_at = now;
    }
    return g->free_seen;
}

void give_host_res(gs_graph* g, const cudaEvent_t ev[3], uint8_t* head) {
    std::lock_guard<std::mutex> lk(g->res_mu);
    for (int i = 0; i < 3; ++i)
        if (ev[i]) g->ev_free.push_back(ev[i]);
    if (head) g->head_free.push_back(head);
}

constexpr uint64_t kArenaMin = 64ull << 20;
constexpr uint64_t kArenaDefault = 512ull << 20;
constexpr uint64_t kSmallRoute = 8192;          // first-level bound above which a query goes straight to the grid path
constexpr double kSmallNodes = 4096.0;          // estimated level nodes above which it does too (4 x the CTA's budget)
constexpr double kSmallRows = 16384.0;          // estimated answer rows above which it does too (4 x the CTA's budget)
constexpr int kMaxRetries = 16;

ExecDev exec_view(gs_result* r) {
    ExecDev E{};
    E.arena = r->arena;
    E.arena_bytes = r->arena_bytes;
    E.ctl = (Ctl*)r->arena;
    E.out = dview(r->so ? *r->so : r->g->out);
    E.in = dview(r->si ? *r->si : r->g->in);
    E.bits = r->bits;
    E.words = (r->g->N + 31) / 32;
    E.lists = r->lists;
    E.list_stride = r->list_stride;
    E.root_cut = r->root_cut ? 1u : 0u;
    E.root_lo = r->root_lo;
    E.root_hi = r->root_hi;
    return E;
}

gs_status enqueue(gs_result* r) {
    NvtxRange nv("gs_eval: enqueue");
    if (r->scan_ready) GS_CUDA(cudaStreamWaitEvent(r->st, r->scan_ready, 0));
    const cudaEvent_t* phases = nullptr;
    if (r->mode == 0 && r->g->trace.load()) {
        const size_t n = (size_t)r->plan.n_levels + 2;
        while (r->phase_ev.size() < n) {
            cudaEvent_t e = nullptr;
            GS_CUDA(cudaEventCreate(&e));
            r->phase_ev.push_back(e);
        }
        phases = r->phase_ev.data();
    }
    GS_CUDA(cudaEventRecord(r->ev0, r->st));
    gs_status rc = r->mode == 1
        ? enqueue_small(&r->plan, exec_view(r), &r->launches, r->st)
        : enqueue_eval(r->g, &r->plan, exec_view(r), r->work, &r->launches, r->st, r->resume,
                       r->scan_status, r->so, r->si, phases);
    if (rc != GS_OK) return rc;
    GS_CUDA(cudaEventRecord(r->ev1, r->st));
    // the head of the control block follows the kernels to pinned memory
    GS_CUDA(cudaMemcpyAsync(r->head, r->arena, kCtlHead, cudaMemcpyDeviceToHost, r->st));
    GS_CUDA(cudaEventRecord(r->ev2, r->st));
    r->ready = false;
    return GS_OK;
}

gs_status wait_result(gs_result* r) {
    if (r->ready) return GS_OK;
    NvtxRange nv("gs_eval: wait");
    for (int attempt = 0; attempt < kMaxRetries; ++attempt) {
        GS_CUDA(cudaEventSynchronize(r->ev2));
        Ctl head;
        std::memcpy(&head, r->head, kCtlHead);
        if (head.status & kStHuge) {
            set_error("gs_eval_query: the answer has more than 2^40 rows under one binding");
            return GS_ENOMEM;
        }
        if (head.status & kStStall) {
            set_error("gs_eval_query: a bulk copy of the triple scan did not complete");
            return GS_ETIMEOUT;
        }
        if (head.status & kStEscalate) {
            // the single-block kernel handed the query back: the grid path
            // continues from the levels it completed, in the same workspace
            r->mode = 0;
            r->resume = std::min<int>((int)head.levels_done, r->plan.n_levels);
            if (r->resume == 0 && r->arena_bytes < kArenaDefault) {
                r->g->alloc.put(r->arena, r->st);
                r->arena = (uint8_t*)r->g->alloc.get(kArenaDefault, r->st);
                if (!r->arena) { set_error("gs_eval_query: cannot allocate the workspace"); return GS_ENOMEM; }
                r->arena_bytes = kArenaDefault;
            }
            gs_status rc = enqueue(r);
            if (rc != GS_OK) return rc;
            continue;
        }
        if (!(head.status & kStOverflow)) {
            const int last = r->plan.n_levels - 1;
            r->rows = head.rows;
            r->out_off = host_level_off(head.n, last + 1);
            r->ready = true;
            return GS_OK;
        }
        // workspace too small: grow it and run again from the start
        r->resume = 0;
        uint64_t need = kCtlBytes;
        for (int l = 0; l < r->plan.n_levels; ++l) need += 8 * head.n[l] + 256;
        need += 4ull * head.rows * r->plan.n_vars;
        uint64_t nb = std::max<uint64_t>(r->arena_bytes * 4, need * 2);
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        r->g->alloc.put(r->arena, r->st);
        r->arena = nullptr;
        GS_CUDA(cudaStreamSynchronize(r->st));
        cudaMemGetInfo(&free_b, &total_b);
        if (nb > (uint64_t)free_b * 9 / 10) nb = (uint64_t)free_b * 9 / 10;
        if (nb <= r->arena_bytes) {
            set_error("gs_eval_query: the evaluation needs more device memory than is free");
            return GS_ENOMEM;
        }
        r->arena = (uint8_t*)r->g->alloc.get(nb, r->st);
        if (!r->arena) { set_error("gs_eval_query: cannot allocate a %llu-byte workspace", (unsigned long long)nb); return GS_ENOMEM; }
        r->arena_bytes = nb;
        gs_status rc = enqueue(r);
        if (rc != GS_OK) return rc;
    }
    set_error("gs_eval_query: workspace retries exhausted");
    return GS_ENOMEM;
}

void release(gs_result* r) {
    if (!r) return;
    if (r->g) {
        cudaStreamSynchronize(r->st);
        r->g->alloc.put(r->arena, r->st);
        if (!r->bits_borrowed) r->g->alloc.put(r->bits, r->st);
        r->g->alloc.put(r->work, r->st);
        r->g->alloc.put(r->lists, r->st);
    }
    const cudaEvent_t ev[3] = {r->ev0, r->ev1, r->ev2};
    if (r->g) give_host_res(r->g, ev, r->head);
    for (cudaEvent_t e : r->phase_ev) cudaEventDestroy(e);
    delete r;
}

void set_pool_threshold(int dev) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}

}  // namespace

extern "C" {

const char* gs_last_error(void) { return last_error(); }

gs_status gs_load_triples(const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n,
                          uint32_t n_vertices, uint32_t n_predicates, int inputs_on_device,
                          const gs_allocator* alloc, void* cuda_stream, gs_graph** out) {
    if (!out) { set_error("gs_load_triples: out is NULL"); return GS_EINVAL; }
    *out = nullptr;
    NvtxRange nv("gs_load_triples");
    if (n && (!s || !p || !o)) { set_error("gs_load_triples: NULL triple array"); return GS_EINVAL; }
    if (n_vertices == 0 || n_vertices > (1u << 31)) { set_error("gs_load_triples: n_vertices must be in 1..2^31"); return GS_EINVAL; }
    if (n_predicates == 0 || n_predicates > 65535) { set_error("gs_load_triples: n_predicates must be in 1..65535"); return GS_EINVAL; }
    if (alloc && (!alloc->alloc || !alloc->free)) { set_error("gs_load_triples: allocator needs alloc and free"); return GS_EINVAL; }
    int dev = 0;
    GS_CUDA(cudaGetDevice(&dev));
    gs_graph* g = new (std::nothrow) gs_graph();
    if (!g) { set_error("gs_load_triples: host out of memory"); return GS_ENOMEM; }
    g->N = n_vertices;
    g->P = n_predicates;
    g->device = dev;
    if (alloc) { g->alloc.hook = *alloc; g->alloc.has_hook = true; }
    cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev);
    g->n_blocks = std::min(kBlocks, std::max(1, g->sm_count * 4));
    level_grids(g->sm_count, &g->range_blocks, &g->expand_blocks);
    set_pool_threshold(dev);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gs_status rc = build_store(g, s, p, o, n, inputs_on_device != 0, st);
    if (rc == GS_OK) {
        g->scan_status = (uint32_t*)g->alloc.get(256, st);
        if (!g->scan_status) { set_error("gs_load_triples: out of device memory"); rc = GS_ENOMEM; }
        else if (cudaMemsetAsync(g->scan_status, 0, 4, st) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "gs_load_triples");
    }
    if (rc == GS_OK) {
        // row lengths on the host (routing estimates)
        std::vector<uint32_t> ptr((size_t)g->N + 1);
        for (int d = 0; d < 2 && rc == GS_OK; ++d) {
            const Store& S = d ? g->in : g->out;
            cudaError_t e = cudaMemcpy(ptr.data(), S.ptr, sizeof(uint32_t) * ptr.size(),
                                       cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { rc = cuda_fail(e, "gs_load_triples"); break; }
            std::vector<uint32_t>& deg = d ? g->deg_in : g->deg_out;
            deg.resize(g->N);
            for (uint32_t v = 0; v < g->N; ++v) deg[v] = ptr[v + 1] - ptr[v];
        }
    }
    if (rc != GS_OK) {
        free_store(g, st);
        g->alloc.put(g->scan_status, st);
        cudaStreamSynchronize(st);
        delete g;
        return rc;
    }
    *out = g;
    return GS_OK;
}



gs_status gs_graph_info(const gs_graph* g, uint64_t* n_triples, uint32_t* n_vertices,
                        uint32_t* n_predicates) {
    if (!g) { set_error("gs_graph_info: graph is NULL"); return GS_EINVAL; }
    if (n_triples) *n_triples = g->M;
    if (n_vertices) *n_vertices = g->N;
    if (n_predicates) *n_predicates = g->P;
    return GS_OK;
}

gs_status gs_graph_export(const gs_graph* g, int by_column, uint32_t* ptr, uint32_t* idx,
                          uint32_t* lab, int dst_on_device, void* cuda_stream) {
    if (!g || !ptr || !idx || !lab) { set_error("gs_graph_export: NULL argument"); return GS_EINVAL; }
    const Store& S = by_column ? g->in : g->out;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    GS_CUDA(cudaMemcpyAsync(ptr, S.ptr, sizeof(uint32_t) * ((uint64_t)g->N + 1), kind, st));
    if (g->M) {
        GS_CUDA(cudaMemcpyAsync(idx, S.idx, sizeof(uint32_t) * g->M, kind, st));
        GS_CUDA(cudaMemcpyAsync(lab, S.lab, sizeof(uint32_t) * g->M, kind, st));
    }
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status gs_plan_query(const gs_graph* g, const int64_t* patterns, uint32_t n_patterns,
                        uint32_t flags, gs_plan** out) {
    if (!out) { set_error("gs_plan_query: out is NULL"); return GS_EINVAL; }
    NvtxRange nv("gs_plan_query");
    return make_plan(g, patterns, n_patterns, flags, out);
}

gs_status gs_plan_paths(const gs_plan* plan, int32_t* buf, uint32_t cap, uint32_t* len) {
    if (!plan || !len) { set_error("gs_plan_paths: NULL argument"); return GS_EINVAL; }
    std::vector<int32_t> w;
    w.push_back((int32_t)plan->paths.size());
    for (auto& p : plan->paths) {
        w.push_back((int32_t)p.size());
        for (int v : p) w.push_back(v);
    }
    *len = (uint32_t)w.size();
    if (!buf || cap < w.size()) { set_error("gs_plan_paths: buffer holds %u words, need %zu", cap, w.size()); return GS_EOVERFLOW; }
    std::memcpy(buf, w.data(), sizeof(int32_t) * w.size());
    return GS_OK;
}

gs_status gs_plan_describe(const gs_plan* plan, int32_t* buf, uint32_t cap, uint32_t* len) {
    if (!plan || !len) { set_error("gs_plan_describe: NULL argument"); return GS_EINVAL; }
    std::vector<int32_t> w;
    w.push_back((int32_t)plan->groups.size());
    for (auto& gr : plan->groups) {
        w.push_back((int32_t)gr.first);
        w.push_back((int32_t)gr.second.size());
        for (int e : gr.second) w.push_back(e);
    }
    w.push_back((int32_t)plan->roots.size());
    for (int64_t r : plan->roots) w.push_back((int32_t)r);
    *len = (uint32_t)w.size();
    if (!buf || cap < w.size()) { set_error("gs_plan_describe: buffer holds %u words, need %zu", cap, w.size()); return GS_EOVERFLOW; }
    std::memcpy(buf, w.data(), sizeof(int32_t) * w.size());
    return GS_OK;
}

}  // extern "C"

gs_status gs::scan_spec_from(const gs_graph* g, const uint32_t* preds, const uint8_t* dirs,
                             uint32_t n, ScanSpec* out, const char* who) {
    if (!g || !preds || !dirs || n == 0) { set_error("%s: NULL argument or n == 0", who); return GS_EINVAL; }
    ScanSpec S{};
    S.n_bvars = 1;
    S.bvar[0] = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (preds[i] < 1 || preds[i] > g->P || dirs[i] > 1) {
            set_error("%s: entry %u: predicate outside 1..P or direction not 0/1", who, i);
            return GS_EINVAL;
        }
        uint32_t* list = dirs[i] ? S.in_pred : S.out_pred;
        int32_t& cnt = dirs[i] ? S.n_in : S.n_out;
        int slot = -1;
        for (int j = 0; j < cnt; ++j) if (list[j] == preds[i]) slot = j;
        if (slot < 0) {
            if (cnt >= kMaxSlots) { set_error("%s: more than %d predicates in one direction", who, kMaxSlots); return GS_EINVAL; }
            list[cnt] = preds[i];
            slot = cnt++;
        }
        (dirs[i] ? S.need_in[0] : S.need_out[0]) |= 1u << slot;
    }
    *out = S;
    return GS_OK;
}

void gs::plan_estimate(const gs_graph* g, const gs_plan* P, Estimate* e) {
    *e = Estimate{};
    const double N = std::max(1.0, (double)g->N), M = std::max(1.0, (double)g->M);
    auto stat = [&](const std::vector<uint64_t>& v, uint32_t p) -> double {
        return p < v.size() ? (double)v[p] : 0.0;
    };
    // mean range length of label p in a row (dir 0) / column (dir 1) holding it
    auto fanout = [&](uint32_t p, uint32_t dir) {
        const double r = stat(g->lab_rows[dir], p);
        return r > 0 ? stat(g->lab_cnt[dir], p) / r : 0.0;
    };
    // share of vertices whose row (dir 0) / column (dir 1) holds label p
    auto holds = [&](uint32_t p, uint32_t dir) { return stat(g->lab_rows[dir], p) / N; };
    const size_t np = P->patterns.size() / 3;
    double prev = 1.0, worst_scratch = 0.0;
    uint64_t levels = 0;
    for (int l = 0; l < P->n_levels; ++l) {
        const LevelSpec& L = P->levels[l];
        const int w = L.var;
        double cand, pass = 1.0;
        int src = -1;
        if (L.src == kSrcList) {
            cand = N;
        } else {
            cand = 1e300;
            for (int b = 0; b < L.n_binders; ++b) {
                const Binder& B = L.b[b];
                double f = fanout(B.label, B.dir);
                if (B.from_const) {   // the constant's row length x the label's share
                    const std::vector<uint32_t>& deg = B.dir == 0 ? g->deg_out : g->deg_in;
                    f = B.c < deg.size() ? std::max(1.0, deg[B.c] * stat(g->lab_cnt[B.dir], B.label) / M) : 0.0;
                }
                if (f < cand) { cand = f; src = b; }
            }
            for (int b = 0; b < L.n_binders; ++b)
                if (b != src) pass *= std::min(1.0, fanout(L.b[b].label, L.b[b].dir) / N);
        }
        // the variable's other patterns: its candidates must hold their predicates
        for (size_t i = 0; i < np; ++i) {
            const int64_t s = P->patterns[3 * i], o = P->patterns[3 * i + 2];
            const uint32_t p = (uint32_t)P->patterns[3 * i + 1];
            const bool subj = s == -(int64_t)w - 1, obj = o == -(int64_t)w - 1;
            if (!subj && !obj) continue;
            bool binder = false;   // edges to bound ends are the binders above
            for (int b = 0; b < L.n_binders && !binder; ++b)
                binder = L.b[b].label == p && ((L.b[b].dir == 0 && obj) || (L.b[b].dir == 1 && subj));
            if (binder) continue;
            if (subj) pass *= holds(p, 0);
            if (obj && !subj) pass *= holds(p, 1);
        }
        const double nodes = std::min(1e15, prev * cand * pass);
        e->nodes[l] = nodes;
        const uint32_t nbm = std::max(1, L.n_binders);
        worst_scratch = std::max(worst_scratch, prev * (16.0 + 8.0 * nbm));
        levels += (((uint64_t)(8.0 * nodes) + 8 + 255) & ~255ull);
        prev = nodes;
    }
    double rows = P->n_levels ? prev : 0.0;
    for (int j = 0; j < P->n_leaves; ++j) rows *= fanout(P->leaves[j].label, P->leaves[j].dir);
    rows = std::min(rows, 1e15);
    e->rows = rows;
    worst_scratch = std::max(worst_scratch, prev * (8.0 + 8.0 * std::max(1, P->n_leaves)));
    e->answer = (uint64_t)(4.0 * P->n_vars * rows);
    e->arena = kCtlBytes + levels + (uint64_t)worst_scratch + e->answer;
    const uint64_t words = (g->N + 31) / 32;
    e->vectors = P->needs_scan ? 4ull * words * (uint64_t)std::max(1, P->scan.n_bvars) : 0;
    e->total = e->arena + e->vectors;
}

// An upper bound on the candidates of the plan's first level when it is
// seeded from constants (their row or column lengths), else UINT64_MAX.
uint64_t gs::first_level_bound(const gs_graph* g, const gs_plan* plan) {
    if (plan->n_levels == 0 || g->deg_out.empty()) return ~0ull;
    const LevelSpec& L = plan->levels[0];
    if (L.src != kSrcBinders) return ~0ull;
    uint64_t best = ~0ull;
    for (int b = 0; b < L.n_binders; ++b) {
        const Binder& B = L.b[b];
        if (!B.from_const || B.c >= g->N) continue;
        best = std::min<uint64_t>(best, B.dir == 0 ? g->deg_out[B.c] : g->deg_in[B.c]);
    }
    return best;
}

gs_status gs::result_compact(gs_result* r) {
    gs_status rc = wait_result(r);
    if (rc != GS_OK) return rc;
    const uint64_t bytes = std::max<uint64_t>(16, 4ull * r->rows * (uint64_t)r->plan.n_vars);
    if (bytes >= r->arena_bytes / 2 && !r->bits && !r->work && !r->lists) return GS_OK;
    uint8_t* keep = (uint8_t*)r->g->alloc.get(bytes, r->st);
    if (!keep) return GS_OK;   // keep the arena: the answers stay where they are
    if (r->rows)
        GS_CUDA(cudaMemcpyAsync(keep, r->arena + r->out_off, 4ull * r->rows * r->plan.n_vars,
                                cudaMemcpyDeviceToDevice, r->st));
    r->g->alloc.put(r->arena, r->st);
    if (!r->bits_borrowed) r->g->alloc.put(r->bits, r->st);
    r->g->alloc.put(r->work, r->st);
    r->g->alloc.put(r->lists, r->st);
    r->bits = nullptr;
    r->work = nullptr;
    r->lists = nullptr;
    r->arena = keep;
    r->arena_bytes = bytes;
    r->out_off = 0;
    return GS_OK;
}

gs_status gs::result_ready(gs_result* r, int* done) {
    if (r->ready) { *done = 1; return GS_OK; }
    cudaError_t e = cudaEventQuery(r->ev2);
    if (e == cudaErrorNotReady) { *done = 0; return GS_OK; }
    if (e != cudaSuccess) return cuda_fail(e, "gs_eval_query");
    *done = 1;
    return GS_OK;
}

namespace {

// A root range of a partitioned evaluation (cut false: every root).
struct RootCut {
    bool cut = false;
    uint32_t lo = 0, hi = 0;
};

gs_status eval_query_impl(gs_graph* g, const gs_plan* plan, void* cuda_stream, int force_grid,
                          uint32_t* pre_bits, cudaEvent_t pre_ready, const uint32_t* pre_status,
                          gs_result** out, const Store* so = nullptr, const Store* si = nullptr,
                          RootCut roots = RootCut());

}  // namespace

gs_status gs::eval_query_path(gs_graph* g, const gs_plan* plan, void* cuda_stream, int force_grid,
                              gs_result** out) {
    return eval_query_impl(g, plan, cuda_stream, force_grid, nullptr, nullptr, nullptr, out);
}

gs_status gs::eval_query_borrowed(gs_graph* g, const gs_plan* plan, void* cuda_stream,
                                  uint32_t* bits, cudaEvent_t ready, const uint32_t* scan_status,
                                  gs_result** out) {
    gs_status rc = eval_query_impl(g, plan, cuda_stream, 1, bits, ready, scan_status, out);
    if (rc == GS_OK) (*out)->bits_borrowed = true;
    return rc;
}

gs_result* gs::result_new_table(gs_graph* g, const gs_plan* plan, cudaStream_t st) {
    gs_result* r = new (std::nothrow) gs_result();
    if (!r) return nullptr;
    r->g = g;
    r->plan = *plan;
    r->st = st;
    cudaEvent_t* ev[3] = {&r->ev0, &r->ev1, &r->ev2};
    if (take_host_res(g, ev, &r->head) != GS_OK || cudaEventRecord(r->ev0, st) != cudaSuccess) {
        release(r);
        return nullptr;
    }
    return r;
}

gs_status gs::result_set_table(gs_result* r, int32_t* rows, uint64_t bytes, uint64_t n,
                               uint32_t launches, const std::vector<uint64_t>& path_nodes) {
    r->arena = (uint8_t*)rows;
    r->arena_bytes = bytes;
    r->out_off = 0;
    r->rows = n;
    r->launches = launches;
    r->path_nodes = path_nodes;
    GS_CUDA(cudaEventRecord(r->ev1, r->st));
    GS_CUDA(cudaEventRecord(r->ev2, r->st));
    r->ready = true;
    return GS_OK;
}

void gs::result_free(gs_result* r) { release(r); }

const int32_t* gs::result_rows(gs_result* r) {
    return wait_result(r) == GS_OK ? (const int32_t*)(r->arena + r->out_off) : nullptr;
}

gs_status gs::eval_query_prescanned(gs_graph* g, const gs_plan* plan, void* cuda_stream,
                                    uint32_t* bits, cudaEvent_t ready, const uint32_t* scan_status,
                                    gs_result** out) {
    if (!bits || !ready || !scan_status || !plan) {
        set_error("internal: a prescanned query needs its vectors, event and status word");
        return GS_EINVAL;
    }
    return eval_query_impl(g, plan, cuda_stream, 1, bits, ready, scan_status, out);
}

namespace {

gs_status eval_query_impl(gs_graph* g, const gs_plan* plan, void* cuda_stream, int force_grid,
                          uint32_t* pre_bits, cudaEvent_t pre_ready, const uint32_t* pre_status,
                          gs_result** out, const Store* so, const Store* si, RootCut roots) {
    if (!g || !plan || !out) { set_error("gs_eval_query: NULL argument"); return GS_EINVAL; }
    *out = nullptr;
    if (plan->N == 0) {   // planned without a graph: check the ids now
        for (size_t i = 0; i < plan->patterns.size(); i += 3) {
            int64_t s = plan->patterns[i], p = plan->patterns[i + 1], o = plan->patterns[i + 2];
            if (p > (int64_t)g->P || s >= (int64_t)g->N || o >= (int64_t)g->N) {
                set_error("gs_eval_query: pattern %zu has an id outside this graph", i / 3);
                return GS_EINVAL;
            }
        }
    } else if (plan->N != g->N || plan->P != g->P) {
        set_error("gs_eval_query: the plan was made for another graph");
        return GS_EINVAL;
    }
    gs_result* r = new (std::nothrow) gs_result();
    if (!r) {
        if (pre_bits) g->alloc.put(pre_bits, (cudaStream_t)cuda_stream);
        set_error("gs_eval_query: host out of memory");
        return GS_ENOMEM;
    }
    r->g = g;
    r->plan = *plan;
    r->st = (cudaStream_t)cuda_stream;
    r->so = so;
    r->si = si;
    r->root_cut = roots.cut;
    r->root_lo = roots.lo;
    r->root_hi = roots.hi;
    const uint64_t words = (g->N + 31) / 32;
    gs_status rc = GS_OK;
    cudaEvent_t* ev[3] = {&r->ev0, &r->ev1, &r->ev2};
    if (take_host_res(g, ev, &r->head) != GS_OK) {
        rc = GS_ECUDA;
    }
    if (pre_bits) {   // the result owns the shared scan's vectors from here on
        r->bits = pre_bits;
        r->scan_ready = pre_ready;
        r->scan_status = pre_status;
    } else if (rc == GS_OK && plan->needs_scan) {
        r->bits = (uint32_t*)g->alloc.get(4 * words * std::max(1, plan->n_levels), r->st);
        r->work = g->alloc.get(scan_work_bytes(g), r->st);
        if (!r->bits || !r->work) { set_error("gs_eval_query: out of device memory"); rc = GS_ENOMEM; }
    }
    bool lists = false;
    for (int l = 1; l < plan->n_levels; ++l) lists |= plan->levels[l].src == kSrcList;
    if (rc == GS_OK && lists) {
        r->list_stride = g->N;
        r->lists = (uint32_t*)g->alloc.get(4ull * g->N * plan->n_levels, r->st);
        if (!r->lists) { set_error("gs_eval_query: out of device memory"); rc = GS_ENOMEM; }
    }
    // the single-CTA evaluator unless the first level is certainly past its
    // budget, or the plan's estimate puts a level or the answer well past
    // it (then it would most likely hand the query back, a host round trip)
    Estimate est{};
    plan_estimate(g, plan, &est);
    bool big = est.rows > kSmallRows;
    for (int l = 0; l < plan->n_levels; ++l) big |= est.nodes[l] > kSmallNodes;
    // (a root range is applied by the grid path's level-0 kernels only)
    r->mode = (small_eligible(plan) && !force_grid && !roots.cut && !big &&
               first_level_bound(g, plan) <= kSmallRoute) ? 1 : 0;
    if (rc == GS_OK) {
        // the grid path's size for both: a query the single-CTA kernel hands
        // back continues in this workspace
        const uint64_t want = first_arena_bytes(g, est);
        r->arena = (uint8_t*)g->alloc.get(want, r->st);
        r->arena_bytes = want;
        if (!r->arena) { set_error("gs_eval_query: cannot allocate the workspace"); rc = GS_ENOMEM; }
    }
    if (rc == GS_OK) rc = enqueue(r);
    if (rc != GS_OK) { release(r); return rc; }
    *out = r;
    return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_eval_query(gs_graph* g, const gs_plan* plan, void* cuda_stream, gs_result** out) {
    if (plan && (plan->flags & GS_PLAN_PATHS)) return eval_paths(g, plan, cuda_stream, out);
    const char* how = getenv("GS_EXEC");   // "grid" forces the grid path
    return eval_query_path(g, plan, cuda_stream, how && !strcmp(how, "grid"), out);
}

gs_status gs_eval_query_roots(gs_graph* g, const gs_plan* plan, uint32_t root_lo, uint32_t root_hi,
                              void* cuda_stream, gs_result** out) {
    if (out) *out = nullptr;
    if (!g || !plan || !out) { set_error("gs_eval_query_roots: NULL argument"); return GS_EINVAL; }
    if (plan->flags & GS_PLAN_PATHS) {
        set_error("gs_eval_query_roots: a per-path plan has one root per path; plan without GS_PLAN_PATHS");
        return GS_EINVAL;
    }
    if (root_lo > root_hi) {
        set_error("gs_eval_query_roots: root_lo %u > root_hi %u", root_lo, root_hi);
        return GS_EINVAL;
    }
    RootCut c;
    c.cut = true;
    c.lo = root_lo;
    c.hi = root_hi;
    return eval_query_impl(g, plan, cuda_stream, 1, nullptr, nullptr, nullptr, out, nullptr, nullptr, c);
}

gs_status gs_plan_root(const gs_plan* plan, uint32_t* var) {
    if (!plan || !var) { set_error("gs_plan_root: NULL argument"); return GS_EINVAL; }
    if (plan->flags & GS_PLAN_PATHS) {
        set_error("gs_plan_root: a per-path plan has one root per path");
        return GS_EINVAL;
    }
    if (plan->n_levels < 1) { set_error("gs_plan_root: the plan has no level"); return GS_EINVAL; }
    *var = (uint32_t)plan->levels[0].var;
    return GS_OK;
}

}  // extern "C"

uint64_t gs::first_arena_bytes(gs_graph* g, const Estimate& est) {
    if (const char* env = getenv("GS_ARENA_BYTES")) {   // initial workspace size
        unsigned long long v = strtoull(env, nullptr, 10);
        if (v >= 4096) return v;
    }
    const uint64_t free_b = free_device_bytes(g);
    uint64_t want = std::max<uint64_t>(kArenaMin, std::min<uint64_t>(kArenaDefault, free_b / 8));
    if (est.arena > want)   // a larger first workspace saves re-runs
        want = std::max(want, std::min<uint64_t>(est.arena + est.arena / 4, free_b / 4));
    return want;
}

extern "C" {

gs_status gs_plan_estimate(const gs_graph* g, const gs_plan* plan, uint64_t* bytes, double* rows) {
    if (!g || !plan) { set_error("gs_plan_estimate: NULL argument"); return GS_EINVAL; }
    if (plan->N != 0 && (plan->N != g->N || plan->P != g->P)) {
        set_error("gs_plan_estimate: the plan was made for another graph");
        return GS_EINVAL;
    }
    Estimate e;
    plan_estimate(g, plan, &e);
    if (bytes) *bytes = e.total + (plan->needs_scan ? scan_work_bytes(g) : 0);
    if (rows) *rows = e.rows;
    return GS_OK;
}

gs_status gs_eval_query_lspm(gs_graph* g, const gs_lspm* l, const gs_plan* plan, void* cuda_stream,
                             gs_result** out) {
    if (!g || !l || !plan || !out) { set_error("gs_eval_query_lspm: NULL argument"); return GS_EINVAL; }
    *out = nullptr;
    if (lspm_graph(l) != g) { set_error("gs_eval_query_lspm: the LSpM was built for another graph"); return GS_EINVAL; }
    if (!lspm_covers(l, plan)) {
        set_error("gs_eval_query_lspm: the LSpM lacks a (predicate, orientation) the plan reads");
        return GS_EINVAL;
    }
    const char* how = getenv("GS_EXEC");   // "grid" forces the grid path
    return eval_query_impl(g, plan, cuda_stream, how && !strcmp(how, "grid"), nullptr, nullptr,
                           nullptr, out, lspm_side(l, 0), lspm_side(l, 1));
}

gs_status gs_result_info(gs_result* r, uint64_t* n_rows, uint32_t* n_vars) {
    if (!r) { set_error("gs_result_info: result is NULL"); return GS_EINVAL; }
    gs_status rc = wait_result(r);
    if (rc != GS_OK) return rc;
    if (n_rows) *n_rows = r->rows;
    if (n_vars) *n_vars = (uint32_t)r->plan.n_vars;
    return GS_OK;
}

gs_status gs_result_tree(gs_result* r, uint64_t* nodes, uint32_t cap, uint32_t* n_levels) {
    if (!r || !n_levels) { set_error("gs_result_tree: NULL argument"); return GS_EINVAL; }
    gs_status rc = wait_result(r);
    if (rc != GS_OK) return rc;
    if (!r->path_nodes.empty()) {   // per-path mode: the tree of each path
        *n_levels = (uint32_t)r->path_nodes.size();
        if (!nodes || cap < *n_levels) { set_error("gs_result_tree: room for %u paths, need %u", cap, *n_levels); return GS_EOVERFLOW; }
        for (uint32_t i = 0; i < *n_levels; ++i) nodes[i] = r->path_nodes[i];
        return GS_OK;
    }
    const int nl = r->plan.n_levels;
    *n_levels = (uint32_t)nl;
    if (r->mode == 1) {   // the single-CTA kernel kept its levels in its own workspace
        set_error("gs_result_tree: the query ran in one CTA; its level sizes are not kept");
        return GS_ENOTIMPL;
    }
    if (!nodes || cap < (uint32_t)nl) { set_error("gs_result_tree: room for %u levels, need %d", cap, nl); return GS_EOVERFLOW; }
    Ctl head;
    std::memcpy(&head, r->head, kCtlHead);
    for (int l = 0; l < nl; ++l) nodes[l] = head.n[l];
    return GS_OK;
}

gs_status gs_graph_set_trace(gs_graph* g, int on) {
    if (!g) { set_error("gs_graph_set_trace: graph is NULL"); return GS_EINVAL; }
    g->trace.store(on ? 1 : 0);
    return GS_OK;
}

gs_status gs_result_phases(gs_result* r, float* ms, uint32_t cap, uint32_t* n_phases) {
    if (!r || !n_phases) { set_error("gs_result_phases: NULL argument"); return GS_EINVAL; }
    gs_status rc = wait_result(r);
    if (rc != GS_OK) return rc;
    const uint32_t n = (uint32_t)r->plan.n_levels + 2;
    if (r->mode != 0 || r->phase_ev.size() < n) {
        set_error("gs_result_phases: no phase events (tracing was off, or the query ran in the single-CTA kernel)");
        return GS_ENOTIMPL;
    }
    *n_phases = n;
    if (cap < n) {
        set_error("gs_result_phases: room for %u phases, the evaluation has %u", cap, n);
        return GS_EOVERFLOW;
    }
    if (!ms) { set_error("gs_result_phases: ms is NULL"); return GS_EINVAL; }
    cudaEvent_t prev = r->ev0;
    for (uint32_t i = 0; i < n; ++i) {
        GS_CUDA(cudaEventElapsedTime(ms + i, prev, r->phase_ev[i]));
        prev = r->phase_ev[i];
    }
    return GS_OK;
}

gs_status gs_result_stats(gs_result* r, float* device_ms, uint32_t* kernel_launches) {
    if (!r) { set_error("gs_result_stats: result is NULL"); return GS_EINVAL; }
    gs_status rc = wait_result(r);
    if (rc != GS_OK) return rc;
    if (device_ms) GS_CUDA(cudaEventElapsedTime(device_ms, r->ev0, r->ev1));
    if (kernel_launches) *kernel_launches = r->launches;
    return GS_OK;
}

gs_status gs_fetch_bindings(gs_result* r, int32_t* dst, uint64_t cap_rows, int dst_on_device,
                            int sort_rows) {
    if (!r) { set_error("gs_fetch_bindings: result is NULL"); return GS_EINVAL; }
    NvtxRange nv("gs_fetch_bindings");
    gs_status rc = wait_result(r);
    if (rc != GS_OK) return rc;
    if (cap_rows < r->rows) {
        set_error("gs_fetch_bindings: buffer holds %llu rows, the answer has %llu",
                  (unsigned long long)cap_rows, (unsigned long long)r->rows);
        return GS_EOVERFLOW;
    }
    if (r->rows == 0) return GS_OK;
    if (!dst) { set_error("gs_fetch_bindings: dst is NULL"); return GS_EINVAL; }
    const uint32_t k = (uint32_t)r->plan.n_vars;
    const uint64_t bytes = 4ull * r->rows * k;
    const int32_t* src = (const int32_t*)(r->arena + r->out_off);
    cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (sort_rows && r->rows > 1) {
        int32_t* tmp = (int32_t*)r->g->alloc.get(bytes, r->st);
        if (!tmp) { set_error("gs_fetch_bindings: out of device memory for sorting"); return GS_ENOMEM; }
        rc = sort_rows_on_device(r->g, src, r->rows, k, tmp, r->st);
        if (rc == GS_OK) {
            cudaError_t e = cudaMemcpyAsync(dst, tmp, bytes, kind, r->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(r->st);
            if (e != cudaSuccess) rc = cuda_fail(e, "gs_fetch_bindings copy");
        }
        r->g->alloc.put(tmp, r->st);
        cudaStreamSynchronize(r->st);
        return rc;
    }
    GS_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, r->st));
    GS_CUDA(cudaStreamSynchronize(r->st));
    return GS_OK;
}

gs_status gs_scan_candidates(gs_graph* g, const uint32_t* preds, const uint8_t* dirs, uint32_t n,
                             uint32_t* out_bits, void* cuda_stream) {
    if (!out_bits) { set_error("gs_scan_candidates: out_bits is NULL"); return GS_EINVAL; }
    ScanSpec S{};
    gs_status rc = scan_spec_from(g, preds, dirs, n, &S, "gs_scan_candidates");
    if (rc != GS_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void* work = g->alloc.get(scan_work_bytes(g), st);
    if (!work) { set_error("gs_scan_candidates: out of device memory"); return GS_ENOMEM; }
    rc = run_scan(g, S, out_bits, work, st, g->scan_status);
    g->alloc.put(work, st);
    return rc;
}

gs_status gs_scan_status(gs_graph* g, void* cuda_stream) {
    if (!g) { set_error("gs_scan_status: graph is NULL"); return GS_EINVAL; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t word = 0;
    GS_CUDA(cudaMemcpyAsync(&word, g->scan_status, sizeof(word), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (!(word & kStStall)) return GS_OK;
    GS_CUDA(cudaMemsetAsync(g->scan_status, 0, sizeof(word), st));
    GS_CUDA(cudaStreamSynchronize(st));
    set_error("gs_scan_status: a bounded wait of the triple scan ran out; the candidate bits of "
              "that scan are incomplete");
    return GS_ETIMEOUT;
}

void gs_free_graph(gs_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    free_store(g, nullptr);
    g->alloc.put(g->scan_status, nullptr);
    cudaDeviceSynchronize();
    for (int i = 0; i < g->n_side; ++i) cudaStreamDestroy(g->side[i]);
    for (cudaEvent_t e : g->ev_free) cudaEventDestroy(e);
    for (uint8_t* b : g->head_blocks) cudaFreeHost(b);
    delete g;
}

void gs_free_plan(gs_plan* plan) { delete plan; }

void gs_free_result(gs_result* r) { release(r); }

}  // extern "C"
