// Serving loop: continuous batching of submitted queries over the resident
// graph. A worker thread owns the device work:
//   - admission: queued plans are taken in arrival order into a batch while
//     the batch's estimated device bytes fit under the server's budget
//     together with everything in flight, and while a stream is free. Each
//     plan's bytes come from its estimated intermediate results (binding-
//     tree levels, answers, candidate vectors; gs_plan_estimate); a plan
//     that does not fit waits and later, smaller ones pass it, until it has
//     waited long enough that nothing passes it any more;
//   - launch: the batch runs on its own stream (gs_eval_batch's persistent
//     kernel), so batches admitted while others are running overlap on the
//     device;
//   - completion: in-flight batches advance without blocking (events): once
//     the batch kernel is done, the queries it handed back are launched on
//     the graph's side streams; once those are done too, the batch
//     completes its tickets (answers stay on the device until the ticket
//     is released) and returns its memory to the budget.
// Callers submit and poll from their own threads; everything shared is
// under one mutex, and CUDA work for one batch is only issued by the worker.
#include <algorithm>
#include <chrono>
#include <functional>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gs_exec.h"

using namespace gs;

namespace {

using Clock = std::chrono::steady_clock;

struct Flight {
    gs_batch* b = nullptr;
    int stream = -1;
    Clock::time_point started;    // when the worker launched the batch
    uint64_t bytes = 0;
    std::vector<uint64_t> tickets;
    std::vector<const gs_plan*> plans;
    int refs = 0;                 // tickets not yet released
    gs_status err = GS_OK;
    std::string msg;
};

struct Ticket {
    const gs_plan* plan = nullptr;
    Clock::time_point submitted, done_at;
    int state = 0;                // 0 queued, 1 running, 2 done, 3 failed
    std::shared_ptr<Flight> flight;
    uint32_t index = 0;
    uint64_t rows = 0;
    gs_status err = GS_OK;
    std::string msg;              // why the query failed
    // estimated device bytes while its batch runs (from gs_plan_estimate's
    // model): kernel queries hold a share of the answer pool; grid-path
    // queries hold their candidate vectors and, while they run, a workspace
    bool kernel = false, scan = false;
    uint64_t share = 0;           // pool share (kernel) or first workspace (grid path)
    uint64_t vectors = 0;         // candidate vectors (plans with a triple scan)
    uint64_t batch_seq = 0;       // 1-based number of the batch that took it
};

}  // namespace

struct gs_server {
    gs_graph* g = nullptr;
    gs_server_config cfg{};
    std::vector<cudaStream_t> streams;
    std::vector<char> stream_busy;
    std::mutex mu;
    std::condition_variable cv;
    bool stopping = false;
    std::thread worker;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::vector<std::shared_ptr<Flight>> inflight;
    uint64_t next_id = 1;
    uint64_t inflight_bytes = 0, peak_bytes = 0;
    uint64_t completed = 0, batches = 0, passed = 0;
    uint64_t launches = 0, scans = 0, scan_plans = 0;   // of the completed batches
    double batch_us = 0.0;        // running mean of the batches' launch-to-completion time
    gs_status fatal = GS_OK;
};

namespace {

// A batch being assembled: the estimated device bytes of the tickets taken.
struct Admit {
    uint32_t n_kernel = 0;
    bool scan = false;
    uint64_t pool = 0, vectors = 0;
    std::vector<uint64_t> grid;        // workspaces of its grid-path queries
};

// Device bytes the batch holds while it runs: fixed CTA workspaces and scan
// masks, the answer pool, every candidate vector, and the workspaces of the
// grid_streams largest grid-path queries (they run that many at a time).
uint64_t admit_bytes(const gs_server* s, const Admit& a) {
    std::vector<uint64_t> g = a.grid;
    const size_t k = std::min<size_t>(g.size(), std::max<uint32_t>(1, s->cfg.batch.grid_streams ? s->cfg.batch.grid_streams : 4));
    std::partial_sort(g.begin(), g.begin() + k, g.end(), std::greater<uint64_t>());
    uint64_t grid = 0;
    for (size_t i = 0; i < k; ++i) grid += g[i];
    return batch_fixed_bytes(s->g, &s->cfg.batch, a.n_kernel, a.scan) + a.pool + a.vectors + grid;
}

void admit_add(Admit& a, const Ticket& t) {
    if (t.kernel) { a.n_kernel++; a.pool += t.share; }
    else a.grid.push_back(t.share);
    a.scan |= t.scan;
    a.vectors += t.vectors;
}

void complete(gs_server* s, std::shared_ptr<Flight>& f, gs_status rc) {
    std::vector<uint64_t> rows(f->tickets.size(), 0);
    if (rc == GS_OK) rc = gs_batch_info(f->b, rows.data(), nullptr);   // ready: no wait
    uint32_t launches = 0, scans = 0, scan_plans = 0;
    if (rc == GS_OK) gs_batch_stats(f->b, nullptr, &launches, nullptr);
    if (rc == GS_OK) gs_batch_scans(f->b, &scans, &scan_plans);
    std::string msg = f->msg;
    if (rc != GS_OK && msg.empty()) msg = last_error();
    std::lock_guard<std::mutex> lk(s->mu);
    const auto now = Clock::now();
    for (size_t i = 0; i < f->tickets.size(); ++i) {
        auto it = s->tickets.find(f->tickets[i]);
        if (it == s->tickets.end()) continue;
        it->second.state = rc == GS_OK ? 2 : 3;
        it->second.err = rc;
        it->second.msg = msg;
        it->second.rows = rows[i];
        it->second.done_at = now;
    }
    s->stream_busy[f->stream] = 0;
    s->completed += f->tickets.size();
    s->launches += launches;
    s->scans += scans;
    s->scan_plans += scan_plans;
}

void worker_loop(gs_server* s) {
    cudaSetDevice(s->g->device);
    for (;;) {
        std::vector<std::shared_ptr<Flight>> finished;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->queue.empty() && s->inflight.empty())
                s->cv.wait_for(lk, std::chrono::microseconds(s->cfg.max_wait_us));
            if (s->stopping && s->queue.empty() && s->inflight.empty()) break;
            // completions (a batch's hand-backs run on the side streams; the
            // worker only looks at events here and never waits)
            for (size_t i = 0; i < s->inflight.size();) {
                int done = 0;
                const gs_status rc = batch_advance(s->inflight[i]->b, &done);
                if (rc != GS_OK || done) {
                    s->inflight[i]->err = rc;
                    if (rc != GS_OK) s->inflight[i]->msg = last_error();
                    s->inflight_bytes -= s->inflight[i]->bytes;   // its workspaces are done
                    const double us = std::chrono::duration<double, std::micro>(
                        Clock::now() - s->inflight[i]->started).count();
                    s->batch_us = s->batch_us > 0.0 ? 0.8 * s->batch_us + 0.2 * us : us;
                    finished.push_back(s->inflight[i]);
                    s->inflight.erase(s->inflight.begin() + i);
                } else {
                    ++i;
                }
            }
            // admission: a new batch starts when the device is idle, when
            // max_batch / 8 queries wait, or when the oldest has waited
            // max_wait_us or half the running mean batch time, whichever is
            // longer; otherwise arrivals gather into the next batch (a wait
            // short against the batches in flight costs little latency and
            // saves the per-batch work of many small batches)
            const double wait_us = std::max<double>(s->cfg.max_wait_us, 0.5 * s->batch_us);
            const bool ripe =
                !s->queue.empty() &&
                (s->inflight.empty() || s->queue.size() >= std::max<uint32_t>(1, s->cfg.max_batch / 8) ||
                 std::chrono::duration<double, std::micro>(
                     Clock::now() - s->tickets[s->queue.front()].submitted).count() >= wait_us);
            while (ripe && !s->queue.empty()) {
                int st = -1;
                for (size_t k = 0; k < s->streams.size(); ++k)
                    if (!s->stream_busy[k]) { st = (int)k; break; }
                if (st < 0) break;
                // Tickets in arrival order while the batch's estimated bytes
                // fit the budget beside everything in flight. One that does
                // not fit waits and later ones may pass it, unless it has
                // waited 50 x max_wait_us: then nothing passes it and memory
                // drains until it fits. A ticket that cannot fit even alone
                // is admitted alone once nothing else is in flight.
                NvtxRange nv("gs_server: admit a batch");
                Admit a;
                std::vector<uint64_t> take_ids;
                uint64_t bytes = 0;
                const auto now = Clock::now();
                for (auto it = s->queue.begin(); it != s->queue.end() && take_ids.size() < s->cfg.max_batch;) {
                    Ticket& t = s->tickets[*it];
                    Admit a2 = a;
                    admit_add(a2, t);
                    const uint64_t b2 = admit_bytes(s, a2);
                    const bool alone = s->inflight.empty() && take_ids.empty();
                    if (s->inflight_bytes + b2 <= s->cfg.memory_budget || alone) {
                        a = a2;
                        bytes = b2;
                        take_ids.push_back(*it);
                        it = s->queue.erase(it);
                        if (alone && s->inflight_bytes + b2 > s->cfg.memory_budget) break;
                        continue;
                    }
                    if (now - t.submitted >= std::chrono::microseconds(50ull * s->cfg.max_wait_us)) break;
                    ++it;
                }
                if (take_ids.empty()) break;   // wait for memory to free up
                for (uint64_t id : take_ids) {   // tickets taken ahead of older waiting ones
                    for (uint64_t qid : s->queue)   // ids grow in arrival order
                        if (qid < id) { s->passed++; break; }
                }
                const uint32_t take = (uint32_t)take_ids.size();
                auto f = std::make_shared<Flight>();
                f->stream = st;
                f->bytes = bytes;
                const uint64_t seq = s->batches + 1;
                for (uint32_t i = 0; i < take; ++i) {
                    Ticket& t = s->tickets[take_ids[i]];
                    t.state = 1;
                    t.flight = f;
                    t.index = i;
                    t.batch_seq = seq;
                    f->tickets.push_back(take_ids[i]);
                    f->plans.push_back(t.plan);
                }
                f->refs = (int)take;
                gs_batch_config bc = s->cfg.batch;
                bc.pool_bytes = std::max<uint64_t>(a.pool, 1ull << 20);
                gs_status rc = eval_batch_ex(s->g, f->plans.data(), take, (void*)s->streams[st],
                                             &bc, 0, &f->b);
                if (rc != GS_OK) {
                    const std::string m = last_error();
                    for (uint64_t id : f->tickets) {
                        Ticket& t = s->tickets[id];
                        t.state = 3;
                        t.err = rc;
                        t.msg = m;
                        t.done_at = Clock::now();
                    }
                    continue;
                }
                s->stream_busy[st] = 1;
                f->started = Clock::now();
                s->inflight_bytes += bytes;
                s->peak_bytes = std::max(s->peak_bytes, s->inflight_bytes);
                s->inflight.push_back(f);
                s->batches++;
            }
        }
        for (auto& f : finished) complete(s, f, f->err);
        if (finished.empty()) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (!s->inflight.empty() && s->queue.empty())
                s->cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" {

gs_status gs_server_start(gs_graph* g, const gs_server_config* cfg, gs_server** out) {
    if (!g || !out) { set_error("gs_server_start: NULL argument"); return GS_EINVAL; }
    *out = nullptr;
    gs_server* s = new (std::nothrow) gs_server();
    if (!s) { set_error("gs_server_start: host out of memory"); return GS_ENOMEM; }
    s->g = g;
    gs_server_config c{};
    c.max_batch = 1024;
    c.n_streams = 4;
    c.memory_budget = 40ull << 30;
    c.max_wait_us = 200;
    c.pool_bytes_per_query = 16ull << 20;
    if (cfg) {
        if (cfg->max_batch) c.max_batch = cfg->max_batch;
        if (cfg->n_streams) c.n_streams = cfg->n_streams;
        if (cfg->memory_budget) c.memory_budget = cfg->memory_budget;
        if (cfg->max_wait_us) c.max_wait_us = cfg->max_wait_us;
        if (cfg->pool_bytes_per_query) c.pool_bytes_per_query = cfg->pool_bytes_per_query;
        c.batch = cfg->batch;
        c.batch.pool_bytes = 0;
    }
    s->cfg = c;
    for (uint32_t i = 0; i < c.n_streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            gs_status rc = cuda_fail(cudaGetLastError(), "gs_server_start");
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return rc;
        }
        s->streams.push_back(st);
    }
    s->stream_busy.assign(c.n_streams, 0);
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return GS_OK;
}

}  // extern "C"

namespace {

// A queued ticket for plan with its estimated device bytes (filled in
// outside the lock).
Ticket make_ticket(gs_server* s, const gs_plan* plan) {
    Ticket t;
    Estimate est;
    plan_estimate(s->g, plan, &est);
    t.plan = plan;
    t.kernel = batch_in_kernel(s->g, plan, &s->cfg.batch);
    t.scan = plan->needs_scan;
    t.share = t.kernel
        ? std::min<uint64_t>(std::max<uint64_t>(est.answer + est.answer / 4, 64ull << 10),
                             s->cfg.pool_bytes_per_query)
        : first_arena_bytes(s->g, est);
    t.vectors = est.vectors;
    return t;
}

}  // namespace

extern "C" {

gs_status gs_server_submit_many(gs_server* s, const gs_plan* const* plans, uint32_t n,
                                uint64_t* tickets) {
    if (!s || (n && (!plans || !tickets))) { set_error("gs_server_submit: NULL argument"); return GS_EINVAL; }
    std::vector<Ticket> ts;
    ts.reserve(n);
    for (uint32_t i = 0; i < n; ++i) {
        const gs_plan* plan = plans[i];
        if (!plan) { set_error("gs_server_submit: plan %u is NULL", i); return GS_EINVAL; }
        if (plan->N != 0 && (plan->N != s->g->N || plan->P != s->g->P)) {
            set_error("gs_server_submit: the plan was made for another graph");
            return GS_EINVAL;
        }
        ts.push_back(make_ticket(s, plan));
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) { set_error("gs_server_submit: the server is stopping"); return GS_EINVAL; }
        const auto now = Clock::now();
        for (uint32_t i = 0; i < n; ++i) {
            const uint64_t id = s->next_id++;
            ts[i].submitted = now;
            s->tickets[id] = ts[i];
            s->queue.push_back(id);
            tickets[i] = id;
        }
    }
    s->cv.notify_one();
    return GS_OK;
}

gs_status gs_server_submit(gs_server* s, const gs_plan* plan, uint64_t* ticket) {
    if (!s || !plan || !ticket) { set_error("gs_server_submit: NULL argument"); return GS_EINVAL; }
    return gs_server_submit_many(s, &plan, 1, ticket);
}

gs_status gs_server_poll(gs_server* s, uint64_t ticket, int* done, uint64_t* rows,
                         double* latency_us) {
    if (!s || !done) { set_error("gs_server_poll: NULL argument"); return GS_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) { set_error("gs_server_poll: unknown ticket %llu", (unsigned long long)ticket); return GS_EINVAL; }
    const Ticket& t = it->second;
    if (t.state == 3) {
        set_error("gs_server_poll: the query failed: %s", t.msg.c_str());
        *done = 1;
        return t.err;
    }
    *done = t.state == 2;
    if (*done) {
        if (rows) *rows = t.rows;
        if (latency_us)
            *latency_us = std::chrono::duration<double, std::micro>(t.done_at - t.submitted).count();
    }
    return GS_OK;
}

gs_status gs_server_fetch(gs_server* s, uint64_t ticket, int32_t* dst, uint64_t cap_rows,
                          int dst_on_device, int sort_rows) {
    if (!s) { set_error("gs_server_fetch: NULL argument"); return GS_EINVAL; }
    std::shared_ptr<Flight> f;
    uint32_t index = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end() || it->second.state != 2) {
            set_error("gs_server_fetch: ticket %llu is not finished", (unsigned long long)ticket);
            return GS_EINVAL;
        }
        f = it->second.flight;
        index = it->second.index;
    }
    return gs_batch_fetch(f->b, index, dst, cap_rows, dst_on_device, sort_rows);
}

gs_status gs_server_release(gs_server* s, uint64_t ticket) {
    if (!s) { set_error("gs_server_release: NULL argument"); return GS_EINVAL; }
    std::shared_ptr<Flight> f;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) { set_error("gs_server_release: unknown ticket"); return GS_EINVAL; }
        if (it->second.state < 2) { set_error("gs_server_release: ticket still running"); return GS_EINVAL; }
        f = it->second.flight;
        s->tickets.erase(it);
        if (f && --f->refs > 0) f.reset();
    }
    if (f) gs_free_batch(f->b);   // last ticket of its batch
    return GS_OK;
}

gs_status gs_server_ticket(gs_server* s, uint64_t ticket, uint64_t* batch_seq, uint64_t* est_bytes) {
    if (!s) { set_error("gs_server_ticket: NULL argument"); return GS_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) { set_error("gs_server_ticket: unknown ticket %llu", (unsigned long long)ticket); return GS_EINVAL; }
    if (batch_seq) *batch_seq = it->second.batch_seq;
    if (est_bytes) *est_bytes = it->second.share + it->second.vectors;
    return GS_OK;
}

gs_status gs_server_admission(gs_server* s, uint64_t* passed, uint64_t* inflight_bytes) {
    if (!s) { set_error("gs_server_admission: NULL argument"); return GS_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    if (passed) *passed = s->passed;
    if (inflight_bytes) *inflight_bytes = s->inflight_bytes;
    return GS_OK;
}

gs_status gs_server_work(gs_server* s, uint64_t* launches, uint64_t* scans, uint64_t* scan_plans) {
    if (!s) { set_error("gs_server_work: NULL argument"); return GS_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    if (launches) *launches = s->launches;
    if (scans) *scans = s->scans;
    if (scan_plans) *scan_plans = s->scan_plans;
    return GS_OK;
}

gs_status gs_server_stats(gs_server* s, uint64_t* completed, uint64_t* batches,
                          uint64_t* peak_bytes) {
    if (!s) { set_error("gs_server_stats: NULL argument"); return GS_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (batches) *batches = s->batches;
    if (peak_bytes) *peak_bytes = s->peak_bytes;
    return GS_OK;
}

void gs_server_stop(gs_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    std::vector<gs_batch*> left;
    for (auto& kv : s->tickets)
        if (kv.second.flight && kv.second.flight->b) left.push_back(kv.second.flight->b);
    std::sort(left.begin(), left.end());
    left.erase(std::unique(left.begin(), left.end()), left.end());
    for (gs_batch* b : left) gs_free_batch(b);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"

extern "C" gs_status gs_server_replay(gs_server* s, const gs_plan* const* plans, uint32_t n_plans,
                                      const double* arrival_s, uint64_t n, double timeout_s,
                                      double* latency_us, double* done_s, int32_t* fetch_buf,
                                      uint64_t fetch_cap_rows, uint64_t* fetched_bytes) {
    if (fetched_bytes) *fetched_bytes = 0;
    if (!s || (n && (!plans || !arrival_s || n_plans == 0))) {
        set_error("gs_server_replay: NULL argument");
        return GS_EINVAL;
    }
    const Clock::time_point t0 = Clock::now();
    auto since = [&](Clock::time_point t) { return std::chrono::duration<double>(t - t0).count(); };
    std::vector<uint64_t> ticket(n, 0);
    uint64_t next = 0, head = 0;   // next to submit; oldest not yet seen done
    std::vector<char> seen(n, 0);
    gs_status fail = GS_OK;
    while (head < n) {
        const double now = since(Clock::now());
        if (now > timeout_s) { set_error("gs_server_replay: not finished after %.1f s", timeout_s); return GS_ETIMEOUT; }
        while (next < n && arrival_s[next] <= now) {
            gs_status rc = gs_server_submit(s, plans[next % n_plans], &ticket[next]);
            if (rc != GS_OK) return rc;
            ++next;
        }
        // completions, oldest first; stop at the first still running
        while (head < next) {
            Clock::time_point done_at;
            int state = 0;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                auto it = s->tickets.find(ticket[head]);
                if (it == s->tickets.end()) { state = 3; }
                else { state = it->second.state; done_at = it->second.done_at; if (state == 3) fail = it->second.err; }
            }
            if (state < 2) break;
            if (fetch_buf && state == 2) {   // the answers to host memory before release
                uint64_t rows = 0;
                int d = 0;
                gs_server_poll(s, ticket[head], &d, &rows, nullptr);
                const gs_status rc = gs_server_fetch(s, ticket[head], fetch_buf, fetch_cap_rows, 0, 0);
                if (rc != GS_OK) return rc;
                if (fetched_bytes) *fetched_bytes += 4ull * rows * (uint64_t)plans[head % n_plans]->n_vars;
            }
            if (latency_us) latency_us[head] = std::chrono::duration<double, std::micro>(done_at - t0).count() - arrival_s[head] * 1e6;
            if (done_s) done_s[head] = since(done_at);
            gs_server_release(s, ticket[head]);
            ++head;
        }
        if (head < n && (next == n || arrival_s[next] > since(Clock::now()) + 20e-6))
            std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
    if (fail != GS_OK) { set_error("gs_server_replay: a query failed"); return fail; }
    return GS_OK;
}
