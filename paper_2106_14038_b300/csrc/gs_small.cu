// Single-block evaluation of whole queries: light-query seeds, every level
// of the binding tree and the enumeration run inside one CTA, the phases
// separated by __syncthreads. Same arena layout and candidate tests as the
// grid path (gs_exec.cu). Used for plans that need no full triple scan
// (queries with constants, whose frontiers start from the constants' rows).
//
//   k_query_block   one query, one launch (the plain form);
//   k_batch         a persistent launch over many queries: every CTA takes
//                   the next query from a device counter and evaluates it in
//                   its own workspace slot, writing the answer rows into a
//                   shared pool reserved by atomic bump allocation.
//
// When a level has more than the candidate budget or the answer more than
// the row budget (or the pool is full), the query stops with kStEscalate and
// the host re-runs it on the grid path.
#include <mutex>

#include "gs_exec_dev.cuh"
#include "gs_qrec.h"

namespace gs {

__device__ __forceinline__ void flag(Ctl* ctl, uint32_t bit) {
    if (threadIdx.x == 0) atomicOr(&ctl->status, bit);
}

// Block-wide in-place exclusive scan of a[0..n); returns the total.
__device__ __forceinline__ uint64_t block_scan_inplace(uint64_t* a, uint64_t n) {
    uint64_t carry = 0;
    for (uint64_t base = 0; base < n; base += kThreads) {
        uint64_t i = base + threadIdx.x;
        uint64_t v = i < n ? a[i] : 0, t;
        uint64_t ex = block_excl_scan_u64(v, &t);
        if (i < n) a[i] = carry + ex;
        carry += t;
    }
    __syncthreads();
    return carry;
}

// Where the answer rows go: the workspace (pool == nullptr) or a pool.
struct PoolOut {
    uint8_t* pool;
    uint64_t pool_bytes;
    unsigned long long* top;
};

// Evaluates the query of record Q in workspace E with the calling block.
// Returns 0, kStEscalate or kStOverflow; on success *off / *rows give the
// answer's byte offset (in the pool, or in the workspace) and row count;
// *done gets the number of complete levels (all of them when it returns 0
// or escalates at the enumeration).
__device__ uint32_t run_query_block(const ExecDev& E, const QRec& Q, uint64_t cand_budget,
                                    uint64_t row_budget, const PoolOut* po, uint64_t* off,
                                    uint64_t* rows, int* done_out) {
    Ctl* ctl = E.ctl;
    __shared__ const uint2* lv[kMaxLevels];
    __shared__ uint64_t sh_off;
    for (uint32_t i = threadIdx.x; i < kCtlHead / 8; i += kThreads) ((uint64_t*)ctl)[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < Q.h->n_cc; i += kThreads) {
        uint32_t lo, len;
        label_range(E.out, Q.h->cc[3 * i], Q.h->cc[3 * i + 1], lo, len);
        if (!in_range(E.out, lo, len, Q.h->cc[3 * i + 2])) atomicOr(&ctl->dead, 1u);
    }
    __syncthreads();
    const bool dead = ctl->dead != 0;
    const int n_levels = Q.h->n_levels;
    int& done = *done_out;
    done = 0;
    for (int l = 0; l < n_levels && !dead; ++l) {
        const LevelSpec& L = Q.lv[l];
        const uint64_t np = l == 0 ? 1 : ctl->n[l - 1];
        if (np == 0) break;
        load_levels(E, l - 1, lv);
        const uint32_t nbm = L.n_binders > 0 ? L.n_binders : 1;
        Scratch S = scratch_at(E, np, nbm);
        const uint64_t base_l = level_off(ctl, l);
        if (S.base < base_l + 256 || E.arena_bytes < scratch_bytes(np, nbm)) return kStEscalate;
        // ranges of the binders of every parent node; the shortest is the source
        for (uint64_t i = threadIdx.x; i < np; i += kThreads) {
            uint32_t vid[kMaxLevels];
            if (l > 0) walk(lv, l - 1, (uint32_t)i, vid);
            uint32_t best = 0xffffffffu, sel = 0;
            for (int b = 0; b < L.n_binders; ++b) {
                const Binder& B = L.b[b];
                uint32_t row = B.from_const ? B.c : vid[B.level];
                uint32_t lo, len;
                label_range(store_of(E, B.dir), row, B.label, lo, len);
                S.rng[i * nbm + b] = make_uint2(lo, len);
                if (len < best) { best = len; sel = (uint32_t)b; }
            }
            S.roff[i] = best;
            S.sel[i] = (uint8_t)sel;
        }
        __syncthreads();
        const uint64_t T = block_scan_inplace(S.roff, np);
        if (T > cand_budget) return kStEscalate;
        const uint64_t cap = (S.base - base_l) / 8;
        uint2* dst = (uint2*)(E.arena + base_l);
        for (uint64_t q0 = 0; q0 < T; q0 += kThreads) {
            uint64_t q = q0 + threadIdx.x;
            bool keep = false;
            uint32_t x = 0, node = 0;
            if (q < T) {
                uint64_t i = upper_bound_u64(S.roff, 0, np, q) - 1;
                node = (uint32_t)i;
                uint32_t sel = S.sel[i];
                const uint2* rng = S.rng + i * nbm;
                uint2 r = rng[sel];
                x = __ldg(store_of(E, L.b[sel].dir).idx + r.x + (q - S.roff[i]));
                keep = keep_candidate(E, L, l, x, rng, sel);
            }
            append(ctl, l, dst, cap, keep, x, node);
        }
        __syncthreads();
        if (ctl->status & kStOverflow) return kStEscalate;
        done = l + 1;
    }
    if (dead || done < n_levels) {
        *off = 0;
        *rows = 0;
        return 0;
    }
    // enumeration
    const int last = n_levels - 1;
    const uint64_t n = ctl->n[last];
    const int n_leaves = Q.h->n_leaves, n_vars = Q.h->n_vars;
    const uint32_t nl = n_leaves > 0 ? n_leaves : 1;
    load_levels(E, last, lv);
    Scratch S = scratch_at(E, n, nl);
    const uint64_t out_off = level_off(ctl, last + 1);
    if (S.base < out_off || E.arena_bytes < scratch_bytes(n, nl)) return kStEscalate;
    for (uint64_t i = threadIdx.x; i < n; i += kThreads) {
        uint64_t cnt = 1;
        if (n_leaves > 0) {
            uint32_t vid[kMaxLevels];
            walk(lv, last, (uint32_t)i, vid);
            for (int j = 0; j < n_leaves; ++j) {
                const LeafSpec& Lf = Q.lf[j];
                uint32_t lo, len;
                label_range(store_of(E, Lf.dir), vid[Lf.level], Lf.label, lo, len);
                S.rng[i * nl + j] = make_uint2(lo, len);
                cnt *= len;
                if (cnt > row_budget) cnt = row_budget + 1;   // saturate: escalates below
            }
        }
        S.roff[i] = cnt;
    }
    __syncthreads();
    const uint64_t R = block_scan_inplace(S.roff, n);
    if (R > row_budget) return kStEscalate;
    const uint64_t rowb = 4ull * n_vars;
    int32_t* out;
    if (po) {
        if (threadIdx.x == 0) {
            uint64_t want = (R * rowb + 15) & ~15ull;
            uint64_t o = want ? atomicAdd(po->top, (unsigned long long)want) : 0;
            sh_off = (o + want <= po->pool_bytes) ? o : ~0ull;
        }
        __syncthreads();
        if (sh_off == ~0ull) return kStEscalate;      // pool full
        *off = sh_off;
        out = (int32_t*)(po->pool + sh_off);
    } else {
        if (R > (S.base - out_off) / rowb) return kStEscalate;
        *off = out_off;
        out = (int32_t*)(E.arena + out_off);
    }
    for (uint64_t q = threadIdx.x; q < R; q += kThreads) {
        uint64_t i = upper_bound_u64(S.roff, 0, n, q) - 1;
        uint64_t loc = q - S.roff[i];
        uint32_t vid[kMaxLevels];
        walk(lv, last, (uint32_t)i, vid);
        uint32_t leafv[kMaxVars];
        for (int j = n_leaves - 1; j >= 0; --j) {
            uint2 r = S.rng[i * nl + j];
            uint64_t d = loc % r.y;
            loc /= r.y;
            leafv[j] = __ldg(store_of(E, Q.lf[j].dir).idx + r.x + d);
        }
        int32_t* row = out + q * n_vars;
        for (int v = 0; v < n_vars; ++v) {
            int32_t src = Q.h->var_src[v];
            row[v] = (int32_t)(src >= 0 ? vid[src] : leafv[-src - 1]);
        }
    }
    *rows = R;
    return 0;
}

constexpr uint64_t kPlainCand = 1ull << 10;
constexpr uint64_t kPlainRows = 1ull << 12;

__global__ void __launch_bounds__(kThreads) k_query_block(ExecDev E, RecParam P) {
    __shared__ uint4 rec[kRecMax / 16];
    const uint32_t words = ((const QHdr*)&P)->bytes / 16;
    for (uint32_t i = threadIdx.x; i < words; i += kThreads) rec[i] = P.w[i];
    __syncthreads();
    const QRec Q = rec_view(rec);
    uint64_t off = 0, rows = 0;
    int done = 0;
    uint32_t st = run_query_block(E, Q, kPlainCand, kPlainRows, nullptr, &off, &rows, &done);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (st) {
            E.ctl->levels_done = (uint32_t)done;   // the grid path resumes here
            atomicOr(&E.ctl->status, kStEscalate);
        } else {
            E.ctl->rows = rows;
        }
    }
}

// Batch: per query result.
__global__ void __launch_bounds__(kThreads) k_batch(BatchDev B) {
    __shared__ uint4 rec[kRecMax / 16];
    __shared__ uint32_t q_sh;
    ExecDev E{};
    E.arena = B.slots + (uint64_t)blockIdx.x * B.slot_bytes;
    E.arena_bytes = B.slot_bytes;
    E.ctl = (Ctl*)E.arena;
    E.out = B.out;
    E.in = B.in;
    const PoolOut po{B.pool, B.pool_bytes, B.pool_top};
    for (;;) {
        if (threadIdx.x == 0) q_sh = atomicAdd(B.next, 1u);
        __syncthreads();
        const uint32_t q = q_sh;
        if (q >= B.n) break;
        const uint4* src = (const uint4*)(B.recs + B.rec_off[q]);
        const uint32_t words = ((const QHdr*)src)->bytes / 16;
        for (uint32_t i = threadIdx.x; i < words; i += kThreads) rec[i] = src[i];
        __syncthreads();
        const QRec Q = rec_view(rec);
        uint64_t off = 0, rows = 0;
        int done = 0;
        uint32_t st = run_query_block(E, Q, B.cand_budget, B.row_budget, &po, &off, &rows, &done);
        __syncthreads();
        if (threadIdx.x == 0) {
            BatchResult r;
            r.off = off;
            r.rows = st ? 0 : rows;
            r.status = st ? kStEscalate : 0u;
            r.pad = 0;
            B.res[q] = r;
        }
        __syncthreads();
    }
}

bool small_eligible(const gs_plan* P) { return rec_fits(P); }

gs_status enqueue_small(const gs_plan* P, const ExecDev& E, uint32_t* launches, cudaStream_t st) {
    RecParam R;
    if (!pack_record(P, &R)) { set_error("internal: query does not fit the single-block record"); return GS_EINVAL; }
    k_query_block<<<1, kThreads, 0, st>>>(E, R);
    if (launches) *launches = 1;
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

// Resident k_batch CTAs per SM of the current device, looked up once per
// device.
int batch_blocks_per_sm() {
    constexpr int kDevs = 64;
    static std::mutex mu;
    static int per_sm[kDevs] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) {
        cudaGetLastError();
        dev = -1;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && per_sm[dev] > 0) return per_sm[dev];
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch, kThreads, 0);
    cudaGetLastError();
    a = a > 0 ? a : 1;
    if (dev >= 0) per_sm[dev] = a;
    return a;
}

gs_status enqueue_batch(const BatchDev& B, int blocks, cudaStream_t st) {
    k_batch<<<blocks, kThreads, 0, st>>>(B);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
