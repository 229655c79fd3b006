// Per-query light-weight sparse matrix (LSpM, Sec. 6.2): the RDF matrix
// reduced to the predicates one query uses, built on the device from the
// resident store.
//
// Sec. 6.2.1 keeps, row-wise, only the triples whose predicate appears in
// the query and drops the empty rows, recording with Mr which rows remain
// (Mr[i + 1] - Mr[i] = 1 when row i is kept, and it is then row Mr[i] of
// the reduced matrix); Sec. 6.2.2 does the same column-wise (Mc) for the
// edges evaluated against their direction, each orientation with its own
// predicate set. Here, per orientation:
//   1. k_lspm_count: per row, the entries of the set's predicates (one
//      pass over a short row's labels, or over a long row's label runs,
//      each tested against the set's bitmap), packed as
//      (count << 32) | (count > 0);
//   2. one device-wide exclusive scan of the packed words gives, per row,
//      the first entry of the reduced row (high half) and Mr (low half);
//   3. k_lspm_write: a warp per 32 rows copies their kept entries in
//      order (a stream compaction over runs of short rows, run by run
//      through the label directory for long rows), so the reduced rows keep
//      the (label, other end) order, and writes the compacted row pointers
//      Pr of the kept rows.
// The reduced orientation is also kept with one row pointer per vertex id
// (empty rows included) and the triple scan's work items, so the
// evaluation kernels run on it unchanged.
#include <algorithm>
#include <new>
#include <vector>

#include "gs_device.cuh"
#include "gs_exec.h"

struct gs_lspm {
    gs_graph* g = nullptr;
    gs::Store side[2];                 // 0: row-wise (CSR), 1: column-wise (CSC)
    uint32_t* mr[2] = {};              // N + 1 words
    uint32_t* pr[2] = {};              // kept + 1 words
    uint64_t kept[2] = {}, nnz[2] = {};
    std::vector<uint32_t> preds[2];    // sorted, distinct
};

namespace gs {

// The set's predicates as a bitmap in shared memory (P <= 65535), filled
// by each block from the set's list.
constexpr uint32_t kKeepWords = 65536 / 32;

__device__ __forceinline__ void load_keep(uint32_t* keep, const uint32_t* __restrict__ set,
                                          uint32_t n_set) {
    for (uint32_t w = threadIdx.x; w < kKeepWords; w += blockDim.x) keep[w] = 0;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n_set; j += blockDim.x)
        atomicOr(&keep[set[j] >> 5], 1u << (set[j] & 31u));
    __syncthreads();
}

__device__ __forceinline__ bool kept_label(const uint32_t* keep, uint32_t l) {
    return (keep[(l >> 5) & (kKeepWords - 1)] >> (l & 31u)) & 1u;
}

// Entries of the set's predicates in each row, packed for the scan. A row
// of at most kDirMin entries is read once, each label tested against the
// set's bitmap; a longer row is walked run by run through its label
// directory (one test per run of equal labels).
__global__ void k_lspm_count(DStore S, uint32_t N, const uint32_t* __restrict__ set, uint32_t n_set,
                             uint64_t* __restrict__ packed) {
    __shared__ uint32_t keep[kKeepWords];
    load_keep(keep, set, n_set);
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = ld(S.ptr + r), e = ld(S.ptr + r + 1);
        uint64_t c = 0;
        if (e - b <= kDirMin || !S.dir_off) {
            for (uint32_t i = b; i < e; i += 4) {   // four loads in flight (label 0 is never kept)
                const uint32_t l0 = ld(S.lab + i);
                const uint32_t l1 = i + 1 < e ? ld(S.lab + i + 1) : 0u;
                const uint32_t l2 = i + 2 < e ? ld(S.lab + i + 2) : 0u;
                const uint32_t l3 = i + 3 < e ? ld(S.lab + i + 3) : 0u;
                c += kept_label(keep, l0) + kept_label(keep, l1) + kept_label(keep, l2) +
                     kept_label(keep, l3);
            }
        } else {
            const uint32_t d0 = ld(S.dir_off + r), d1 = ld(S.dir_off + r + 1);
            for (uint32_t j = d0; j < d1; ++j)
                if (kept_label(keep, ld(S.dir_lab + j)))
                    c += (j + 1 < d1 ? ld(S.dir_pos + j + 1) : e) - ld(S.dir_pos + j);
        }
        packed[r] = (c << 32) | (c ? 1u : 0u);
    }
}

// Each warp takes 32 consecutive rows. Their kept entries are contiguous in
// the output and in the same order as in the store, so the warp copies
// them as a stream compaction: runs of consecutive rows of at most kDirMin
// entries are one contiguous entry range, read 32 entries at a time (a
// ballot and a population count place each kept entry), and a longer row
// is copied run by run from its label directory (runs of predicates
// outside the set are skipped). Row pointers per vertex id, Mr and, for
// kept rows, the compacted pointers Pr are written on the way.
__global__ void k_lspm_write(DStore S, uint32_t N, const uint32_t* __restrict__ set, uint32_t n_set,
                             const uint64_t* __restrict__ packed, uint32_t nnz,
                             uint32_t* __restrict__ ptr, uint32_t* __restrict__ mr,
                             uint32_t* __restrict__ pr, uint32_t* __restrict__ idx,
                             uint32_t* __restrict__ lab) {
    __shared__ uint32_t keep[kKeepWords];
    load_keep(keep, set, n_set);
    const uint32_t lane = lane_id();
    const uint32_t below = (1u << lane) - 1u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t r0 = (blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < N;
         r0 += warps * 32) {
        const uint32_t nr = N - r0 < 32 ? (uint32_t)(N - r0) : 32u;   // rows of this block
        const uint64_t r = r0 + lane;
        const bool valid = lane < nr;
        uint32_t b = 0, e = 0, base = 0, m = 0;
        if (valid) {
            const uint64_t pk = packed[r];
            base = (uint32_t)(pk >> 32);
            m = (uint32_t)pk;
            b = ld(S.ptr + r);
            e = ld(S.ptr + r + 1);
            ptr[r] = base;
            mr[r] = m;
        }
        // the next row's first output position: the row's kept entries end there
        uint32_t next = __shfl_down_sync(0xffffffffu, base, 1);
        if (lane == nr - 1) next = r0 + nr < N ? (uint32_t)(packed[r0 + nr] >> 32) : nnz;
        if (valid && next > base) pr[m] = base;
        const uint32_t longs = __ballot_sync(0xffffffffu, valid && e - b > kDirMin && S.dir_off);
        uint32_t at = __shfl_sync(0xffffffffu, base, 0);
        uint32_t k = 0;
        while (k < nr) {
            // rows k .. kl - 1 are short: one contiguous entry range
            const uint32_t rest = longs & ~((1u << k) - 1u);
            const uint32_t kl = rest ? (uint32_t)(__ffs(rest) - 1) : nr;
            if (kl > k) {
                const uint32_t x0 = __shfl_sync(0xffffffffu, b, k);
                const uint32_t x1 = __shfl_sync(0xffffffffu, e, kl - 1);
                for (uint32_t i0 = x0; i0 < x1; i0 += 128) {   // four loads in flight per lane
                    uint32_t l[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t i = i0 + 32u * (uint32_t)u + lane;
                        l[u] = i < x1 ? ld(S.lab + i) : 0u;   // label 0 is never kept
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t i = i0 + 32u * (uint32_t)u + lane;
                        const bool kp = kept_label(keep, l[u]);
                        const uint32_t mask = __ballot_sync(0xffffffffu, kp);
                        if (kp) {
                            const uint32_t o = at + __popc(mask & below);
                            idx[o] = ld(S.idx + i);
                            lab[o] = l[u];
                        }
                        at += __popc(mask);
                    }
                }
            }
            if (kl >= nr) break;
            // row kl is long: its kept runs, one after the other
            const uint32_t rr = (uint32_t)(r0 + kl);
            const uint32_t ek = __shfl_sync(0xffffffffu, e, kl);
            const uint32_t d0 = ld(S.dir_off + rr), d1 = ld(S.dir_off + rr + 1);
            for (uint32_t j = d0; j < d1; ++j) {
                const uint32_t l = ld(S.dir_lab + j);
                if (!kept_label(keep, l)) continue;
                const uint32_t lo = ld(S.dir_pos + j), hi = j + 1 < d1 ? ld(S.dir_pos + j + 1) : ek;
                for (uint32_t t = lane; t < hi - lo; t += 32) {
                    idx[at + t] = ld(S.idx + lo + t);
                    lab[at + t] = l;
                }
                at += hi - lo;
            }
            k = kl + 1;
        }
    }
}

namespace {

// One orientation of the reduced matrix under predicate set `preds`.
gs_status build_side(gs_lspm* L, int dir, cudaStream_t st) {
    gs_graph* g = L->g;
    const Store& F = dir ? g->in : g->out;
    Store& R = L->side[dir];
    const std::vector<uint32_t>& preds = L->preds[dir];
    const uint32_t N = g->N;
    const int nb = g->n_blocks;
    uint64_t* packed = (uint64_t*)g->alloc.get(sizeof(uint64_t) * (uint64_t)N, st);
    uint64_t* misc = (uint64_t*)g->alloc.get(sizeof(uint64_t) * (2 * kBlocks + 8), st);
    uint32_t* set = (uint32_t*)g->alloc.get(sizeof(uint32_t) * std::max<size_t>(1, preds.size()), st);
    gs_status rc = GS_OK;
    auto done = [&](gs_status r) {
        g->alloc.put(packed, st);
        g->alloc.put(misc, st);
        g->alloc.put(set, st);
        return r;
    };
    if (!packed || !misc || !set) { set_error("gs_lspm_build: out of device memory"); return done(GS_ENOMEM); }
    uint64_t* bsum = misc;
    uint64_t* boff = misc + kBlocks;
    uint64_t* total = misc + 2 * kBlocks;
    uint64_t* n_dev = total + 1;
    const uint64_t n_host = N;
    cudaError_t e = cudaMemcpyAsync(n_dev, &n_host, sizeof(uint64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !preds.empty())
        e = cudaMemcpyAsync(set, preds.data(), sizeof(uint32_t) * preds.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return done(cuda_fail(e, "gs_lspm_build"));
    k_lspm_count<<<g->sm_count * 6, kThreads, 0, st>>>(dview(F), N, set, (uint32_t)preds.size(), packed);
    k_block_sums_u64<<<nb, kThreads, 0, st>>>(packed, n_dev, bsum, nullptr);
    k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, boff, (uint32_t)nb, total, nullptr);
    k_scan_apply_u64<<<nb, kThreads, 0, st>>>(packed, n_dev, boff, nullptr);
    uint64_t tot = 0;
    e = cudaMemcpyAsync(&tot, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(cuda_fail(e, "gs_lspm_build"));
    const uint64_t nnz = tot >> 32, kept = tot & 0xffffffffull;
    L->nnz[dir] = nnz;
    L->kept[dir] = kept;
    // padded like the resident store: aligned 16-byte loads and bulk copies
    // that start inside an array stay inside its allocation
    R.ptr = (uint32_t*)g->alloc.get(sizeof(uint32_t) * ((uint64_t)N + 1 + 4), st);
    R.idx = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (nnz + 4), st);
    R.lab = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (nnz + 4), st);
    L->mr[dir] = (uint32_t*)g->alloc.get(sizeof(uint32_t) * ((uint64_t)N + 1), st);
    L->pr[dir] = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (kept + 1), st);
    if (!R.ptr || !R.idx || !R.lab || !L->mr[dir] || !L->pr[dir]) {
        set_error("gs_lspm_build: out of device memory");
        return done(GS_ENOMEM);
    }
    const uint32_t tail[2] = {(uint32_t)nnz, (uint32_t)kept};
    if (e == cudaSuccess) e = cudaMemsetAsync(R.ptr + N + 1, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.idx + nnz, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.lab + nnz, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.ptr + N, &tail[0], 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->mr[dir] + N, &tail[1], 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->pr[dir] + kept, &tail[0], 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return done(cuda_fail(e, "gs_lspm_build"));
    k_lspm_write<<<g->sm_count * 6, kThreads, 0, st>>>(dview(F), N, set, (uint32_t)preds.size(), packed,
                                          (uint32_t)nnz, R.ptr, L->mr[dir], L->pr[dir], R.idx, R.lab);
    e = cudaGetLastError();
    if (e != cudaSuccess) return done(cuda_fail(e, "gs_lspm_build"));
    rc = store_items(g, R, nnz, st);   // synchronizes st
    return done(rc);
}

void release(gs_lspm* L, cudaStream_t st) {
    if (!L) return;
    if (L->g) {
        cudaStreamSynchronize(st);
        for (int d = 0; d < 2; ++d) {
            Store& R = L->side[d];
            L->g->alloc.put(R.ptr, st); L->g->alloc.put(R.idx, st); L->g->alloc.put(R.lab, st);
            L->g->alloc.put(R.items, st); L->g->alloc.put(R.heads, st);
            L->g->alloc.put(L->mr[d], st); L->g->alloc.put(L->pr[d], st);
        }
    }
    delete L;
}

gs_status sorted_set(const gs_graph* g, const uint32_t* preds, uint32_t n, std::vector<uint32_t>* out) {
    if (n && !preds) { set_error("gs_lspm_build: NULL predicate list"); return GS_EINVAL; }
    out->assign(preds, preds + n);
    for (uint32_t p : *out)
        if (p < 1 || p > g->P) { set_error("gs_lspm_build: predicate %u outside 1..%u", p, g->P); return GS_EINVAL; }
    std::sort(out->begin(), out->end());
    out->erase(std::unique(out->begin(), out->end()), out->end());
    return GS_OK;
}

}  // namespace

// The (predicate, orientation) pairs the evaluation of P reads: edges
// expanded from a row or checked as membership in it, pre-pruning probes,
// leaves, self-loops, fully constant patterns, and the triple scan's slots.
void plan_store_preds(const gs_plan* P, std::vector<uint32_t>* rows, std::vector<uint32_t>* cols) {
    auto add = [&](uint32_t dir, uint32_t p) { (dir ? cols : rows)->push_back(p); };
    for (int l = 0; l < P->n_levels; ++l) {
        const LevelSpec& L = P->levels[l];
        for (int b = 0; b < L.n_binders; ++b) add(L.b[b].dir, L.b[b].label);
        for (int j = 0; j < L.n_probes; ++j) add(L.pr[j].dir, L.pr[j].label);
        for (int j = 0; j < L.n_self; ++j) add(0, L.self_label[j]);
    }
    for (int j = 0; j < P->n_leaves; ++j) add(P->leaves[j].dir, P->leaves[j].label);
    for (size_t i = 0; i + 2 < P->const_triples.size(); i += 3) add(0, P->const_triples[i + 1]);
    if (P->needs_scan) {
        for (int i = 0; i < P->scan.n_out; ++i) add(0, P->scan.out_pred[i]);
        for (int i = 0; i < P->scan.n_in; ++i) add(1, P->scan.in_pred[i]);
    }
    for (auto* v : {rows, cols}) {
        std::sort(v->begin(), v->end());
        v->erase(std::unique(v->begin(), v->end()), v->end());
    }
}

const Store* lspm_side(const gs_lspm* L, int dir) { return &L->side[dir]; }

bool lspm_covers(const gs_lspm* L, const gs_plan* P) {
    std::vector<uint32_t> r, c;
    plan_store_preds(P, &r, &c);
    return std::includes(L->preds[0].begin(), L->preds[0].end(), r.begin(), r.end()) &&
           std::includes(L->preds[1].begin(), L->preds[1].end(), c.begin(), c.end());
}

const gs_graph* lspm_graph(const gs_lspm* L) { return L->g; }

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_lspm_build(gs_graph* g, const uint32_t* row_preds, uint32_t n_row,
                        const uint32_t* col_preds, uint32_t n_col, void* cuda_stream, gs_lspm** out) {
    if (!g || !out) { set_error("gs_lspm_build: NULL argument"); return GS_EINVAL; }
    *out = nullptr;
    gs_lspm* L = new (std::nothrow) gs_lspm();
    if (!L) { set_error("gs_lspm_build: host out of memory"); return GS_ENOMEM; }
    L->g = g;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gs_status rc = sorted_set(g, row_preds, n_row, &L->preds[0]);
    if (rc == GS_OK) rc = sorted_set(g, col_preds, n_col, &L->preds[1]);
    for (int d = 0; d < 2 && rc == GS_OK; ++d) rc = build_side(L, d, st);
    if (rc != GS_OK) { release(L, st); return rc; }
    *out = L;
    return GS_OK;
}

gs_status gs_lspm_for_plan(gs_graph* g, const gs_plan* plan, void* cuda_stream, gs_lspm** out) {
    if (!g || !plan || !out) { set_error("gs_lspm_for_plan: NULL argument"); return GS_EINVAL; }
    std::vector<uint32_t> r, c;
    plan_store_preds(plan, &r, &c);
    return gs_lspm_build(g, r.data(), (uint32_t)r.size(), c.data(), (uint32_t)c.size(), cuda_stream, out);
}

gs_status gs_lspm_info(const gs_lspm* L, int by_column, uint64_t* kept, uint64_t* nnz) {
    if (!L) { set_error("gs_lspm_info: NULL argument"); return GS_EINVAL; }
    const int d = by_column ? 1 : 0;
    if (kept) *kept = L->kept[d];
    if (nnz) *nnz = L->nnz[d];
    return GS_OK;
}

gs_status gs_lspm_export(const gs_lspm* L, int by_column, uint32_t* m, uint32_t* ptr, uint32_t* val,
                         uint32_t* idx, int dst_on_device, void* cuda_stream) {
    if (!L || !m || !ptr || ((!val || !idx) && L->nnz[by_column ? 1 : 0])) {
        set_error("gs_lspm_export: NULL argument");
        return GS_EINVAL;
    }
    const int d = by_column ? 1 : 0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    GS_CUDA(cudaMemcpyAsync(m, L->mr[d], sizeof(uint32_t) * ((uint64_t)L->g->N + 1), kind, st));
    GS_CUDA(cudaMemcpyAsync(ptr, L->pr[d], sizeof(uint32_t) * (L->kept[d] + 1), kind, st));
    if (L->nnz[d]) {
        GS_CUDA(cudaMemcpyAsync(val, L->side[d].lab, sizeof(uint32_t) * L->nnz[d], kind, st));
        GS_CUDA(cudaMemcpyAsync(idx, L->side[d].idx, sizeof(uint32_t) * L->nnz[d], kind, st));
    }
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

void gs_free_lspm(gs_lspm* L) { release(L, nullptr); }

}  // extern "C"
