// Per-path binding trees (Sec. 7.1) reconciled by tree-pruning (Sec. 8.1,
// Sec. 8.2): the evaluation of a plan made with GS_PLAN_PATHS.
//
// 1. One triple scan writes a candidate vector per variable (Eq. 17 /
//    Eq. 21 over all its incident edges).
// 2. Each path of the traversal (root, v1, .., vk; Ex. 7.1) is evaluated as
//    its own chain: level 0 holds the root's bindings, level j the bindings
//    of vj reached from a level j-1 node through the path's j-th edge, every
//    candidate tested against its variable's vector (the pre-pruning of
//    Sec. 7.2.2) and its constant edges. The path's binding tree is those
//    levels; its root-to-end walks are written out as a table with one
//    column per path step (the grid path's enumeration).
// 3. Local tree-pruning (Sec. 8.1): the trees of one root keep, per root
//    binding, only the bindings of each common variable that every tree
//    holding it has; global tree-pruning (Sec. 8.2) does the same for the
//    variables shared by the trees of different roots. On the tables both
//    are semi-joins on the shared variables (the root is among them for
//    trees of one root); they repeat until no table shrinks. Dropping a
//    walk drops its target node's subtree and the parents left without
//    children, as steps 3-4 of Sec. 8.1 do on the trees.
// 4. The answers are the join of the pruned tables on their shared
//    variables (exact: a binding of every variable that all trees agree
//    on), columns in variable order.
// Semi-joins and joins hash the shared columns of one side, sort those keys
// (radix sort), and probe them from the other side, comparing the shared
// columns exactly.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gs_device.cuh"
#include "gs_exec.h"

namespace gs {

namespace {

struct ColMap {
    int32_t J, E;                  // shared columns, extra columns of B
    int32_t ca[kMaxVars], cb[kMaxVars], eb[kMaxVars];
};

__device__ __forceinline__ uint32_t key_hash(const int32_t* row, const int32_t* cols, int J) {
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the 32-bit values
    for (int j = 0; j < J; ++j) {
        h ^= (uint32_t)row[cols[j]];
        h *= 1099511628211ull;
    }
    return (uint32_t)(h ^ (h >> 32));
}

// keys[i] = (hash of B row i's shared columns) << 32 | i
__global__ void k_table_keys(const int32_t* __restrict__ B, uint64_t n, int kB, ColMap m,
                             uint64_t* __restrict__ keys) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        keys[i] = ((uint64_t)key_hash(B + i * kB, m.cb, m.J) << 32) | i;
}

// For each A row, the B rows whose shared columns equal its own (found by
// their hash among the sorted keys, then compared exactly). Count pass
// (off == NULL): cnt[a] = matches (semi: 0 or 1). Write pass: at off[a],
// the A row (semi) or, per match, the A row followed by B's extra columns.
__global__ void k_probe(const int32_t* __restrict__ A, uint64_t nA, int kA,
                        const int32_t* __restrict__ B, int kB, const uint64_t* __restrict__ keys,
                        uint64_t nB, ColMap m, int semi, uint64_t* __restrict__ cnt,
                        const uint64_t* __restrict__ off, int32_t* __restrict__ out) {
    const int kOut = semi ? kA : kA + m.E;
    for (uint64_t a = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; a < nA;
         a += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t* ra = A + a * kA;
        const uint64_t h = (uint64_t)key_hash(ra, m.ca, m.J) << 32;
        uint64_t lo = 0, hi = nB;   // first key >= h
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (keys[mid] < h) lo = mid + 1; else hi = mid;
        }
        uint64_t c = 0;
        uint64_t at = off ? off[a] : 0;
        for (uint64_t t = lo; t < nB && (keys[t] & 0xffffffff00000000ull) == h; ++t) {
            const int32_t* rb = B + (keys[t] & 0xffffffffull) * kB;
            bool eq = true;
            for (int j = 0; j < m.J && eq; ++j) eq = ra[m.ca[j]] == rb[m.cb[j]];
            if (!eq) continue;
            ++c;
            if (off) {
                int32_t* o = out + at * kOut;
                for (int j = 0; j < kA; ++j) o[j] = ra[j];
                if (!semi)
                    for (int e = 0; e < m.E; ++e) o[kA + e] = rb[m.eb[e]];
                ++at;
            }
            if (semi) break;
        }
        if (!off) cnt[a] = c;
    }
}

// out row i, column v = T row i, column perm[v]
__global__ void k_permute(const int32_t* __restrict__ T, uint64_t n, int k, ColMap perm,
                          int32_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        for (int v = 0; v < k; ++v) out[i * k + v] = T[i * k + perm.ca[v]];
}

// A table of bindings on the device: n rows of vars.size() int32 columns.
struct Table {
    int32_t* d = nullptr;
    uint64_t n = 0;
    std::vector<int> vars;
    int32_t* own = nullptr;        // allocation to free (NULL: a sub-result's arena)
};

// The chain schedule of path pi of plan M; false when a step has more
// binders (its path edge and its constant edges) than a level holds.
bool path_plan(const gs_plan* M, size_t pi, gs_plan* out) {
    std::vector<int> vars = M->paths[pi];
    const std::vector<int>& pats = M->path_pat[pi];
    // a path that closes onto one of its own earlier steps (only its last
    // step can) checks that edge at its previous step instead of binding
    // the variable again
    int close_at = -1;
    for (size_t i = 0; vars.size() > 1 && i + 1 < vars.size(); ++i)
        if (vars[i] == vars.back()) close_at = (int)i;
    if (close_at >= 0) vars.pop_back();
    out->N = M->N;
    out->P = M->P;
    out->flags = 0;
    out->n_vars = (int)vars.size();
    out->n_levels = (int)vars.size();
    out->n_leaves = 0;
    out->needs_scan = false;
    out->const_triples = M->const_triples;
    const int64_t* pat = M->patterns.data();
    const size_t np = M->patterns.size() / 3;
    for (size_t j = 0; j < vars.size(); ++j) {
        LevelSpec& L = out->levels[j];
        std::memset(&L, 0, sizeof(L));
        const int w = vars[j];
        const int64_t wv = -(int64_t)w - 1;
        L.var = (int32_t)j;
        L.vec = w;
        L.use_bitmap = 1;
        if (j > 0) {   // the path's edge from step j - 1
            const int e = pats[j];
            Binder& B = L.b[L.n_binders++];
            B.label = (uint32_t)pat[3 * e + 1];
            B.from_const = 0;
            B.level = (int16_t)(j - 1);
            B.dir = pat[3 * e + 2] == wv ? 0 : 1;   // w the object: the row of step j - 1
        }
        for (size_t i = 0; i < np; ++i) {
            const int64_t s = pat[3 * i], o = pat[3 * i + 2];
            const uint32_t p = (uint32_t)pat[3 * i + 1];
            if (s == wv && o == wv) {
                bool dup = false;
                for (int q = 0; q < L.n_self; ++q) dup |= L.self_label[q] == p;
                if (!dup && L.n_self < kMaxSelf) L.self_label[L.n_self++] = p;
            } else if ((s == wv && o >= 0) || (o == wv && s >= 0)) {
                if (L.n_binders >= kMaxBinders) return false;
                Binder& B = L.b[L.n_binders++];
                B.label = p;
                B.from_const = 1;
                B.c = (uint32_t)(s == wv ? o : s);
                B.level = -1;
                B.dir = o == wv ? 0 : 1;
            }
        }
        if (close_at >= 0 && j + 1 == vars.size()) {   // the closing edge, to step close_at
            if (L.n_binders >= kMaxBinders) return false;
            const int e = pats[vars.size()];
            Binder& B = L.b[L.n_binders++];
            B.label = (uint32_t)pat[3 * e + 1];
            B.from_const = 0;
            B.level = (int16_t)close_at;
            B.dir = pat[3 * e + 2] == wv ? 0 : 1;    // w the object: the row of step close_at
        }
        L.src = L.n_binders > 0 ? kSrcBinders : kSrcList;
        out->var_src[j] = (int32_t)j;
    }
    return true;
}

}  // namespace

namespace {

// Semi-join (semi) or join of tables A and B on their shared variables.
gs_status match(gs_graph* g, const Table& A, const Table& B, bool semi, cudaStream_t st, Table* out,
                uint32_t* launches) {
    ColMap m{};
    std::vector<int> ov = A.vars;
    for (size_t j = 0; j < B.vars.size(); ++j) {
        auto it = std::find(A.vars.begin(), A.vars.end(), B.vars[j]);
        if (it != A.vars.end()) {
            m.ca[m.J] = (int32_t)(it - A.vars.begin());
            m.cb[m.J] = (int32_t)j;
            m.J++;
        } else {
            m.eb[m.E++] = (int32_t)j;
            ov.push_back(B.vars[j]);
        }
    }
    if (semi) ov = A.vars;
    const int kA = (int)A.vars.size(), kB = (int)B.vars.size(), kO = (int)ov.size();
    out->vars = ov;
    if (B.n >= (1ull << 32)) { set_error("gs_eval_query: a path table has 2^32 rows or more"); return GS_ENOTIMPL; }
    const int nb = g->n_blocks;
    const uint64_t nBk = std::max<uint64_t>(1, B.n), nAk = std::max<uint64_t>(1, A.n);
    uint64_t* keys = (uint64_t*)g->alloc.get(8 * nBk, st);
    uint64_t* tmp = (uint64_t*)g->alloc.get(8 * nBk, st);
    uint64_t* cnt = (uint64_t*)g->alloc.get(8 * (nAk + 1), st);
    uint64_t* misc = (uint64_t*)g->alloc.get(sizeof(uint64_t) * (2 * kBlocks + 8), st);
    auto done = [&](gs_status r) {
        g->alloc.put(keys, st); g->alloc.put(tmp, st); g->alloc.put(cnt, st); g->alloc.put(misc, st);
        return r;
    };
    if (!keys || !tmp || !cnt || !misc) { set_error("gs_eval_query: out of device memory (path join)"); return done(GS_ENOMEM); }
    if (B.n) k_table_keys<<<nb, kThreads, 0, st>>>(B.d, B.n, kB, m, keys);
    gs_status rc = B.n > 1 ? radix_sort_u64(g, &keys, &tmp, B.n, 32, 64, st) : GS_OK;
    if (rc != GS_OK) return done(rc);
    GS_CUDA(cudaMemsetAsync(cnt + A.n, 0, 8, st));
    if (A.n) k_probe<<<nb, kThreads, 0, st>>>(A.d, A.n, kA, B.d, kB, keys, B.n, m, semi, cnt, nullptr, nullptr);
    uint64_t* bsum = misc;
    uint64_t* boff = misc + kBlocks;
    uint64_t* total = misc + 2 * kBlocks;
    uint64_t* n_dev = total + 1;
    const uint64_t n1 = A.n + 1;
    GS_CUDA(cudaMemcpyAsync(n_dev, &n1, 8, cudaMemcpyHostToDevice, st));
    k_block_sums_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, bsum, nullptr);
    k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, boff, (uint32_t)nb, total, nullptr);
    k_scan_apply_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, boff, nullptr);
    uint64_t rows = 0;
    GS_CUDA(cudaMemcpyAsync(&rows, total, 8, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    out->n = rows;
    out->own = (int32_t*)g->alloc.get(std::max<uint64_t>(16, 4ull * rows * kO), st);
    out->d = out->own;
    if (!out->own) { set_error("gs_eval_query: out of device memory (%llu joined rows)", (unsigned long long)rows); return done(GS_ENOMEM); }
    if (A.n && rows)
        k_probe<<<nb, kThreads, 0, st>>>(A.d, A.n, kA, B.d, kB, keys, B.n, m, semi, cnt, cnt, out->d);
    GS_CUDA(cudaGetLastError());
    if (launches) *launches += 7 + (B.n > 1 ? 8 : 0);
    return done(GS_OK);
}

bool shares(const Table& a, const Table& b) {
    for (int v : a.vars)
        if (std::find(b.vars.begin(), b.vars.end(), v) != b.vars.end()) return true;
    return false;
}

}  // namespace

gs_status eval_paths(gs_graph* g, const gs_plan* M, void* cuda_stream, gs_result** out) {
    if (!g || !M || !out) { set_error("gs_eval_query: NULL argument"); return GS_EINVAL; }
    *out = nullptr;
    if (M->N != 0 && (M->N != g->N || M->P != g->P)) { set_error("gs_eval_query: the plan was made for another graph"); return GS_EINVAL; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint64_t words = (g->N + 31) / 32;
    const int k = M->n_vars;
    gs_result* R = result_new_table(g, M, st);
    if (!R) { set_error("gs_eval_query: cannot set up the result"); return GS_ECUDA; }
    uint32_t* bits = (uint32_t*)g->alloc.get(4 * words * std::max(1, k), st);
    void* work = g->alloc.get(scan_work_bytes(g), st);
    uint32_t* status = (uint32_t*)g->alloc.get(256, st);
    cudaEvent_t ev = nullptr;
    std::vector<gs_result*> sub;
    std::vector<Table> T;
    uint32_t launches = 3;
    auto cleanup = [&](gs_status r) {
        for (gs_result* s : sub) result_free(s);
        for (Table& t : T) g->alloc.put(t.own, st);
        cudaStreamSynchronize(st);
        g->alloc.put(bits, st);
        g->alloc.put(work, st);
        g->alloc.put(status, st);
        if (ev) cudaEventDestroy(ev);
        if (r != GS_OK) result_free(R);
        return r;
    };
    if (!bits || !work || !status) { set_error("gs_eval_query: out of device memory"); return cleanup(GS_ENOMEM); }
    GS_CUDA(cudaMemsetAsync(status, 0, 4, st));
    gs_status rc = run_scan(g, M->path_scan, bits, work, st, status);
    if (rc != GS_OK) return cleanup(rc);
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ev, st) != cudaSuccess)
        return cleanup(cuda_fail(cudaGetLastError(), "gs_eval_query"));
    // one binding tree per path, written out as its table of walks
    std::vector<uint64_t> nodes(M->paths.size(), 0);
    for (size_t pi = 0; pi < M->paths.size(); ++pi) {
        gs_plan* PP = new (std::nothrow) gs_plan();
        if (!PP) { set_error("gs_eval_query: host out of memory"); return cleanup(GS_ENOMEM); }
        if (!path_plan(M, pi, PP)) {
            delete PP;
            set_error("gs_eval_query: a path step has more than %d edges to bound ends", kMaxBinders);
            return cleanup(GS_ENOTIMPL);
        }
        gs_result* r = nullptr;
        rc = eval_query_borrowed(g, PP, (void*)st, bits, ev, status, &r);
        delete PP;   // the result keeps its own copy
        if (rc != GS_OK) return cleanup(rc);
        sub.push_back(r);
    }
    for (size_t pi = 0; pi < sub.size(); ++pi) {
        uint64_t n = 0;
        rc = gs_result_info(sub[pi], &n, nullptr);
        if (rc != GS_OK) return cleanup(rc);
        uint64_t lv[kMaxLevels];
        uint32_t nl = 0;
        if (gs_result_tree(sub[pi], lv, kMaxLevels, &nl) == GS_OK)
            for (uint32_t l = 0; l < nl; ++l) nodes[pi] += lv[l];
        uint32_t sl = 0;
        gs_result_stats(sub[pi], nullptr, &sl);
        launches += sl;
        Table t;
        t.d = const_cast<int32_t*>(result_rows(sub[pi]));
        t.n = n;
        t.vars = M->paths[pi];
        if (t.vars.size() > 1 &&
            std::find(t.vars.begin(), t.vars.end() - 1, t.vars.back()) != t.vars.end() - 1)
            t.vars.pop_back();   // closed onto itself: checked inside the path
        T.push_back(t);
    }
    // tree-pruning: semi-joins on shared variables until no table shrinks
    for (size_t round = 0; round < 2 * T.size() + 2; ++round) {
        bool shrunk = false;
        for (size_t i = 0; i < T.size(); ++i)
            for (size_t j = 0; j < T.size(); ++j) {
                if (i == j || !shares(T[i], T[j])) continue;
                Table s;
                rc = match(g, T[i], T[j], true, st, &s, &launches);
                if (rc != GS_OK) { g->alloc.put(s.own, st); return cleanup(rc); }
                if (s.n < T[i].n) shrunk = true;
                g->alloc.put(T[i].own, st);
                T[i] = s;
            }
        if (!shrunk) break;
    }
    // the join of the pruned trees: next, a table sharing variables with the
    // joined part when there is one
    Table J = T[0];
    T[0].own = nullptr;
    std::vector<char> used(T.size(), 0);
    used[0] = 1;
    for (size_t step = 1; step < T.size(); ++step) {
        size_t pick = T.size();
        for (size_t i = 0; i < T.size() && pick == T.size(); ++i)
            if (!used[i] && shares(J, T[i])) pick = i;
        for (size_t i = 0; i < T.size() && pick == T.size(); ++i)
            if (!used[i]) pick = i;
        used[pick] = 1;
        Table nj;
        rc = match(g, J, T[pick], false, st, &nj, &launches);
        g->alloc.put(J.own, st);
        J.own = nullptr;
        if (rc != GS_OK) { g->alloc.put(nj.own, st); return cleanup(rc); }
        J = nj;
    }
    // columns in variable order
    ColMap perm{};
    for (int v = 0; v < k; ++v)
        perm.ca[v] = (int32_t)(std::find(J.vars.begin(), J.vars.end(), v) - J.vars.begin());
    int32_t* fin = (int32_t*)g->alloc.get(std::max<uint64_t>(16, 4ull * J.n * k), st);
    if (!fin) { g->alloc.put(J.own, st); set_error("gs_eval_query: out of device memory (answers)"); return cleanup(GS_ENOMEM); }
    if (J.n) k_permute<<<g->n_blocks, kThreads, 0, st>>>(J.d, J.n, k, perm, fin);
    launches += 1;
    cudaError_t e = cudaGetLastError();
    g->alloc.put(J.own, st);
    if (e != cudaSuccess) { g->alloc.put(fin, st); return cleanup(cuda_fail(e, "gs_eval_query")); }
    rc = result_set_table(R, fin, std::max<uint64_t>(16, 4ull * J.n * k), J.n, launches, nodes);
    if (rc != GS_OK) return cleanup(rc);
    rc = cleanup(GS_OK);
    *out = R;
    return rc;
}

}  // namespace gs
