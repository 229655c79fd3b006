// Executor: grouped incident-edge evaluation of one plan (Sec. 5, Sec. 7).
//
// Bindings are kept as a tree in device memory (Sec. 7.1): level l holds
// one (vertex, parent index) pair per binding of the l-th materialized
// variable, each node extending the partial binding of its parent. A level
// is produced from the previous one in four steps, all sized on the device
// (no host round trip):
//   k_range       per parent node: the entry range of every binder edge in
//                 the row / column of the bound end (a predicate-filtered
//                 row selection, Eq. 15 / Eq. 19 / Eq. 23 for one node), and
//                 the shortest of them;
//                 Its blocks also scan their counts into block-local
//                 offsets, and the last block to finish turns the block
//                 sums into block offsets and the level's candidate total;
//   k_expand      load-balanced over all candidates: take the candidate from
//                 the shortest range, keep it when it is in every other
//                 binder range, passes the pre-pruning tests of Sec. 7.2.2
//                 (candidate vector or predicate presence) and its
//                 self-loops; survivors are appended with warp-aggregated
//                 atomics.
// Consecutive kernels are chained with programmatic dependent launch: each
// is scheduled while the one before it finishes and waits for it on entry.
// A parent without candidates has no children, so dead bindings never
// reach later levels (pre-pruning). Leaves (variables with one pattern)
// are not materialized: k_enum_range stores their range per last-level
// node and k_enum_write writes the cross product as int32 tuples.
//
// Workspace ("arena"): [control block | level 0 | level 1 | ... | output]
// growing up, per-level scratch at the top growing down. Offsets are
// functions of the level sizes, so every kernel recomputes them. A level or
// an output that does not fit sets kStOverflow; the host then re-runs with
// a larger arena.
#include <algorithm>

#include "gs_exec_dev.cuh"

namespace gs {

// ------------------------------------------------------------------ //

// inherit: NULL, or the status word of a triple scan shared with other
// queries, whose kStStall the query takes over.
__global__ void k_init(ExecDev E, ConstChecks cc, const uint32_t* inherit) {
    Ctl* c = E.ctl;
    for (uint32_t i = threadIdx.x; i < kCtlHead / 8; i += blockDim.x) ((uint64_t*)c)[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        c->one = 1;
        if (inherit) c->status = *inherit & kStStall;
    }
    for (uint32_t i = threadIdx.x; i < cc.n; i += blockDim.x) {
        uint32_t s = cc.t[3 * i], p = cc.t[3 * i + 1], o = cc.t[3 * i + 2];
        uint32_t lo, len;
        label_range(E.out, s, p, lo, len);
        if (!in_range(E.out, lo, len, o)) atomicOr(&c->dead, 1u);
    }
    chain_done();
}

// Resuming from the single-block kernel at level `from`: the counts of the
// levels from `from` on, the totals and the status start again at zero;
// the complete levels, `dead` and the level-0 parent count stay.
__global__ void k_resume(ExecDev E, int from) {
    Ctl* c = E.ctl;
    for (int l = from + threadIdx.x; l < kMaxLevels; l += blockDim.x) {
        c->n[l] = 0;
        c->list_n[l] = 0;
    }
    if (threadIdx.x == 0) {
        c->cand = 0;
        c->rows = 0;
        c->status = 0;
        c->arrive = 0;
        c->one = 1;
    }
    chain_done();
}

// Candidate counts of the parent nodes of level l, as block-local
// exclusive offsets; the last block writes the block offsets and the total.
__global__ void __launch_bounds__(kThreads) k_range(ExecDev E, int l, LevelSpec L) {
    chain_enter();
    Ctl* ctl = E.ctl;
    if (overflowed(ctl)) return;
    __shared__ const uint2* lv[kMaxLevels];
    load_levels(E, l - 1, lv);
    const uint64_t np = l == 0 ? 1 : ctl->n[l - 1];
    const uint32_t nbm = L.n_binders > 0 ? L.n_binders : 1;
    Scratch S = scratch_at(E, np, nbm);
    if (S.base < level_off(ctl, l) + 256 || E.arena_bytes < scratch_bytes(np, nbm)) {
        // the scratch would overlap the tree: report, write nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr((uint32_t*)&E.ctl->status, kStOverflow);
        return;
    }
    const bool dead = ctl->dead != 0;
    const uint32_t ch = even_chunk(np, gridDim.x);
    const uint64_t beg = min((uint64_t)blockIdx.x * ch, np), end = min(beg + ch, np);
    uint64_t carry = 0;
    for (uint64_t base = beg; base < end; base += kThreads) {
        const uint64_t i = base + threadIdx.x;
        uint64_t cnt = 0;
        uint32_t sel = 0;
        if (i < end && !dead) {
            if (L.src == kSrcList) {
                cnt = ctl->list_n[l];
            } else {
                uint32_t vid[kMaxLevels];
                if (l > 0) walk(lv, l - 1, (uint32_t)i, vid);
                uint32_t best = 0xffffffffu;
                for (int b = 0; b < L.n_binders; ++b) {
                    const Binder& B = L.b[b];
                    uint32_t row = B.from_const ? B.c : vid[B.level];
                    uint32_t lo, len;
                    label_range(store_of(E, B.dir), row, B.label, lo, len);
                    S.rng[i * nbm + b] = make_uint2(lo, len);
                    if (len < best) { best = len; sel = (uint32_t)b; }
                }
                cnt = best;
            }
        }
        uint64_t t;
        const uint64_t ex = block_excl_scan_u64(cnt, &t);
        if (i < end) {
            S.roff[i] = carry + ex;
            S.sel[i] = (uint8_t)sel;
        }
        carry += t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->roff_chunk = ch;
    arrive_and_scan(ctl, carry, &ctl->cand);
}

__global__ void __launch_bounds__(kThreads) k_expand(ExecDev E, int l, LevelSpec L) {
    chain_enter();
    Ctl* ctl = E.ctl;
    if (overflowed(ctl)) return;
    __shared__ uint64_t roff_s[kExpTileNodes];
    __shared__ uint32_t owner[kExpTile];
    const uint64_t np = l == 0 ? 1 : ctl->n[l - 1];
    const uint32_t nbm = L.n_binders > 0 ? L.n_binders : 1;
    Scratch S = scratch_at(E, np, nbm);
    const uint64_t T = ctl->cand;
    const uint32_t ch = ctl->roff_chunk;
    uint64_t base_l = kCtlBytes;
    for (int j = 0; j < l; ++j) base_l += align256(8ull * ctl->n[j]);
    const uint64_t cap = S.base > base_l ? (S.base - base_l) / 8 : 0;
    uint2* dst = (uint2*)(E.arena + base_l);
    const uint32_t* list = E.lists ? E.lists + (uint64_t)l * E.list_stride : nullptr;
    for (uint64_t t0 = (uint64_t)blockIdx.x * kExpTile; t0 < T; t0 += (uint64_t)gridDim.x * kExpTile) {
        uint64_t t1 = min(t0 + kExpTile, T);
        const uint64_t i0 = block_upper_bound_roff(S.roff, ctl, ch, 0, np, t0) - 1;
        const uint64_t i1 = block_upper_bound_roff(S.roff, ctl, ch, i0, np, t1 - 1);
        // When the tile's nodes fit in shared memory, its candidates find
        // their nodes there without a search: owner[u] is marked with the
        // last node k whose first candidate is t0 + u (nodes without
        // candidates share the next node's offset, and the last of them is
        // the one that has some), and a max-scan over the tile carries each
        // mark forward to the candidates that follow it.
        const bool local = i1 - i0 <= kExpTileNodes;
        if (local) {
            for (uint32_t u = threadIdx.x; u < kExpTile; u += kThreads) owner[u] = 0;
            __syncthreads();
            for (uint64_t k = threadIdx.x; k < i1 - i0; k += kThreads) {
                const uint64_t o = roff_at(S.roff, ctl, ch, i0 + k);
                roff_s[k] = o;
                if (o >= t0 && o < t1) atomicMax(&owner[o - t0], (uint32_t)k);
            }
            __syncthreads();
            uint32_t run = 0, m[kExpItems];
#pragma unroll
            for (int e = 0; e < kExpItems; ++e) {
                run = max(run, owner[threadIdx.x * kExpItems + e]);
                m[e] = run;
            }
            const uint32_t before = block_excl_max_u32(run);
#pragma unroll
            for (int e = 0; e < kExpItems; ++e) owner[threadIdx.x * kExpItems + e] = max(m[e], before);
        }
        __syncthreads();
        for (int k = 0; k < kExpItems; ++k) {
            uint64_t q = t0 + (uint64_t)k * kThreads + threadIdx.x;
            bool keep = false;
            uint32_t x = 0, node = 0;
            if (q < t1) {
                uint64_t i, j;
                if (local) {
                    const uint32_t k = owner[q - t0];
                    i = i0 + k;
                    j = q - roff_s[k];
                } else {
                    i = upper_bound_roff(S.roff, ctl, ch, i0, i1, q) - 1;
                    j = q - roff_at(S.roff, ctl, ch, i);
                }
                node = (uint32_t)i;
                uint32_t sel = S.sel[i];
                const uint2* rng = S.rng + i * nbm;
                if (L.src == kSrcList) {
                    x = list[j];
                } else {
                    uint2 r = rng[sel];
                    x = __ldg(store_of(E, L.b[sel].dir).idx + r.x + j);
                }
                keep = (l != 0 || root_ok(E, x)) &&
                       keep_candidate(E, L, l, x, rng, L.src == kSrcList ? 0xffffffffu : sel);
            }
            append(ctl, l, dst, cap, keep, x, node);
        }
        __syncthreads();
    }
    chain_done();
}

// ------------------------------------------------------------------ //
// Candidate vector -> ordered vertex list (warp ballot / popc + block scan).

// Per-block counts of the candidate vector's vertices; the last block writes
// the block offsets and the total (level 0's size, or the list length).
__global__ void __launch_bounds__(kThreads) k_bits_count(ExecDev E, int l, LevelSpec L) {
    chain_enter();
    if (overflowed(E.ctl)) return;
    const uint32_t* bm = E.bits + (uint64_t)L.vec * E.words;
    uint64_t beg, end;
    block_chunk(E.words, blockIdx.x, gridDim.x, beg, end);
    uint64_t c = 0;
    if (!E.ctl->dead)
        for (uint64_t w = beg + threadIdx.x; w < end; w += kThreads) {
            const uint32_t word = l == 0 ? bm[w] & root_word_mask(E, (uint32_t)w) : bm[w];
            c += __popc(word_keep(E, L, (uint32_t)w, word));
        }
    c = block_sum_u64(c);
    arrive_and_scan(E.ctl, c, l == 0 ? &E.ctl->n[0] : &E.ctl->list_n[l]);
}

// to_level: write (vertex, 0) pairs as level l (a root); else the list of level l
__global__ void __launch_bounds__(kThreads) k_bits_write(ExecDev E, int l, LevelSpec L, int to_level) {
    chain_enter();
    Ctl* ctl = E.ctl;
    if (overflowed(ctl) || ctl->dead) return;
    const uint32_t* bm = E.bits + (uint64_t)L.vec * E.words;
    uint64_t base_l = kCtlBytes;
    for (int j = 0; j < l; ++j) base_l += align256(8ull * ctl->n[j]);
    const uint64_t cap = E.arena_bytes > base_l ? (E.arena_bytes - base_l) / 8 : 0;
    uint2* dst = (uint2*)(E.arena + base_l);
    uint32_t* list = E.lists ? E.lists + (uint64_t)l * E.list_stride : nullptr;
    uint64_t beg, end;
    block_chunk(E.words, blockIdx.x, gridDim.x, beg, end);
    uint64_t carry = ctl->boff[blockIdx.x];
    for (uint64_t base = beg; base < end; base += kThreads) {
        uint64_t w = base + threadIdx.x;
        uint32_t word = 0u;
        if (w < end)
            word = word_keep(E, L, (uint32_t)w, to_level ? bm[w] & root_word_mask(E, (uint32_t)w) : bm[w]);
        uint64_t t;
        uint64_t pos = carry + block_excl_scan_u64(__popc(word), &t);
        for (uint32_t m = word; m; m &= m - 1) {
            uint32_t x = (uint32_t)w * 32 + (__ffs(m) - 1);
            if (to_level) {
                if (pos < cap) dst[pos] = make_uint2(x, 0u);
                else atomicOr(&ctl->status, kStOverflow);
            } else {
                list[pos] = x;
            }
            ++pos;
        }
        carry += t;
    }
    chain_done();
}

// ------------------------------------------------------------------ //
// Enumeration.

constexpr uint64_t kCountCap = 1ull << 40;

// Answer rows per last-level node (the product of its leaf ranges), as
// block-local exclusive offsets; the last block writes the block offsets and
// the row total.
__global__ void __launch_bounds__(kThreads) k_enum_range(ExecDev E, int last, EnumSpec F) {
    chain_enter();
    Ctl* ctl = E.ctl;
    if (overflowed(ctl)) return;
    __shared__ const uint2* lv[kMaxLevels];
    load_levels(E, last, lv);
    const uint64_t n = ctl->n[last];
    const uint32_t nl = F.n_leaves > 0 ? F.n_leaves : 1;
    Scratch S = scratch_at(E, n, nl);
    if (S.base < level_off(ctl, last + 1) || E.arena_bytes < scratch_bytes(n, nl)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->status, kStOverflow);
        return;
    }
    const uint32_t ch = even_chunk(n, gridDim.x);
    const uint64_t beg = min((uint64_t)blockIdx.x * ch, n), end = min(beg + ch, n);
    uint64_t carry = 0;
    for (uint64_t base = beg; base < end; base += kThreads) {
        const uint64_t i = base + threadIdx.x;
        uint64_t cnt = i < end ? 1 : 0;
        if (i < end && F.n_leaves > 0) {
            uint32_t vid[kMaxLevels];
            walk(lv, last, (uint32_t)i, vid);
            for (int j = 0; j < F.n_leaves; ++j) {
                const LeafSpec& Lf = F.leaf[j];
                uint32_t lo, len;
                label_range(store_of(E, Lf.dir), vid[Lf.level], Lf.label, lo, len);
                S.rng[i * nl + j] = make_uint2(lo, len);
                cnt = cnt * len;
                if (cnt > kCountCap) { cnt = kCountCap; atomicOr(&ctl->status, kStHuge); }
            }
        }
        uint64_t t;
        const uint64_t ex = block_excl_scan_u64(cnt, &t);
        if (i < end) S.roff[i] = carry + ex;
        carry += t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->roff_chunk = ch;
    arrive_and_scan(ctl, carry, &ctl->rows);
}

// Tiles of answer rows: consecutive threads take consecutive rows (their
// node data and leaf entries are then shared or adjacent), decode the leaf
// digits (32-bit division when the offset fits), and stage the rows in
// shared memory; the tile is written out with 16-byte stores.
constexpr uint32_t kEnumStageWords = 7168;    // 28 KB of staged rows
constexpr uint32_t kEnumTileNodes = 2048;     // row offsets of a tile's nodes kept in shared memory

__global__ void __launch_bounds__(kThreads) k_enum_write(ExecDev E, int last, EnumSpec F) {
    chain_enter();
    Ctl* ctl = E.ctl;
    if (overflowed(ctl) || (ctl->status & kStHuge)) return;
    __shared__ const uint2* lv[kMaxLevels];
    __shared__ __align__(16) uint32_t stage[kEnumStageWords];
    __shared__ uint64_t roff_s[kEnumTileNodes + 1];
    load_levels(E, last, lv);
    const uint64_t n = ctl->n[last];
    const uint32_t nl = F.n_leaves > 0 ? F.n_leaves : 1;
    Scratch S = scratch_at(E, n, nl);
    const uint64_t T = ctl->rows;
    const uint32_t ch = ctl->roff_chunk;
    uint64_t out_off = kCtlBytes;
    for (int j = 0; j <= last; ++j) out_off += align256(8ull * ctl->n[j]);
    const uint32_t nv = (uint32_t)F.n_vars;
    const uint64_t rowb = 4ull * nv;
    const uint64_t cap = S.base > out_off ? (S.base - out_off) / rowb : 0;
    if (T > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->status, kStOverflow);
        return;
    }
    uint8_t* out = E.arena + out_off;   // 256-byte aligned
    // rows per tile: a multiple of 4 (so every tile starts on 16 bytes)
    const uint32_t tile_rows = min(kThreads * 8u, (kEnumStageWords / nv) & ~3u);
    for (uint64_t t0 = (uint64_t)blockIdx.x * tile_rows; t0 < T; t0 += (uint64_t)gridDim.x * tile_rows) {
        const uint64_t t1 = min(t0 + tile_rows, T);
        const uint64_t i0 = block_upper_bound_roff(S.roff, ctl, ch, 0, n, t0) - 1;
        const uint64_t i1 = block_upper_bound_roff(S.roff, ctl, ch, i0, n, t1 - 1);
        // the tile's node offsets in shared memory (when they fit): the row ->
        // node search then runs there
        const bool local = i1 - i0 <= kEnumTileNodes;
        if (local)
            for (uint64_t k = threadIdx.x; k < i1 - i0; k += kThreads)
                roff_s[k] = roff_at(S.roff, ctl, ch, i0 + k);
        __syncthreads();
        for (uint64_t q = t0 + threadIdx.x; q < t1; q += kThreads) {
            uint64_t i, base;
            if (local) {
                uint32_t lo = 0, hi = (uint32_t)(i1 - i0);   // last k with roff_s[k] <= q
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (roff_s[mid] <= q) lo = mid; else hi = mid;
                }
                i = i0 + lo;
                base = roff_s[lo];
            } else {
                i = upper_bound_roff(S.roff, ctl, ch, i0, i1, q) - 1;
                base = roff_at(S.roff, ctl, ch, i);
            }
            uint64_t loc = q - base;
            // straight into the staged row: each level's and leaf's column
            uint32_t* row = stage + (q - t0) * nv;
            uint32_t node = (uint32_t)i;
            for (int j = last; j >= 0; --j) {
                const uint2 e = lv[j][node];
                row[F.col_of_level[j]] = e.x;
                node = e.y;
            }
            if (loc < (1ull << 32)) {
                uint32_t l32 = (uint32_t)loc;
                for (int j = F.n_leaves - 1; j >= 0; --j) {
                    const uint2 r = S.rng[i * nl + j];
                    const uint32_t d = l32 % r.y;
                    l32 /= r.y;
                    row[F.col_of_leaf[j]] = __ldg(store_of(E, F.leaf[j].dir).idx + r.x + d);
                }
            } else {
                for (int j = F.n_leaves - 1; j >= 0; --j) {
                    const uint2 r = S.rng[i * nl + j];
                    const uint64_t d = loc % r.y;
                    loc /= r.y;
                    row[F.col_of_leaf[j]] = __ldg(store_of(E, F.leaf[j].dir).idx + r.x + d);
                }
            }
        }
        __syncthreads();
        // the tile's rows are contiguous in the output: 16-byte stores, then the tail
        const uint64_t bytes = (t1 - t0) * rowb;
        uint8_t* dst = out + t0 * rowb;
        const uint64_t n16 = bytes / 16;
        for (uint64_t k = threadIdx.x; k < n16; k += kThreads)
            reinterpret_cast<uint4*>(dst)[k] = reinterpret_cast<const uint4*>(stage)[k];
        for (uint64_t k = n16 * 4 + threadIdx.x; k < bytes / 4; k += kThreads)
            reinterpret_cast<uint32_t*>(dst)[k] = stage[k];
        __syncthreads();
    }
    chain_done();
}

// ------------------------------------------------------------------ //

void level_grids(int sm_count, int* range_blocks, int* expand_blocks) {
    int fr = 0, fe = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fr, k_range, kThreads, 0) != cudaSuccess || fr < 1) fr = 4;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fe, k_expand, kThreads, 0) != cudaSuccess || fe < 1) fe = 4;
    cudaGetLastError();
    *range_blocks = std::max(1, std::min(kBlocks, sm_count * fr));
    *expand_blocks = std::max(1, sm_count * fe);
}

uint64_t host_level_off(const uint64_t* n, int l) {
    uint64_t o = kCtlBytes;
    for (int j = 0; j < l; ++j) o += align256(8ull * n[j]);
    return o;
}

gs_status enqueue_eval(const gs_graph* g, const gs_plan* P, const ExecDev& E, void* scan_work, uint32_t* launches,
                       cudaStream_t st, int start_level, const uint32_t* scanned, const Store* so,
                       const Store* si, const cudaEvent_t* phase_ev) {
    const dim3 nb(g->n_blocks), th(kThreads);
    Ctl* ctl = E.ctl;
    uint32_t nl_launch = 1;
    if (start_level > 0) {
        if (P->needs_scan || start_level > P->n_levels) {
            set_error("internal: a resumed query must be a scan-free plan");
            return GS_EINVAL;
        }
        k_resume<<<1, kThreads, 0, st>>>(E, start_level);
    } else {
        ConstChecks cc{};
        cc.n = (uint32_t)(P->const_triples.size() / 3);
        if (cc.n > kMaxPatterns) cc.n = kMaxPatterns;
        for (uint32_t i = 0; i < 3 * cc.n; ++i) cc.t[i] = P->const_triples[i];
        k_init<<<1, kThreads, 0, st>>>(E, cc, scanned);   // zeroes the control block's head
        if (P->needs_scan && !scanned) {
            gs_status rc = run_scan(g, P->scan, E.bits, scan_work, st, &ctl->status, so, si);
            if (rc != GS_OK) return rc;
            nl_launch += 3;
        }
    }
    if (phase_ev) {
        for (int l = 0; l <= start_level && l <= P->n_levels; ++l)   // setup and scan; levels resumed past
            GS_CUDA(cudaEventRecord(phase_ev[l], st));
    }
    for (int l = start_level; l < P->n_levels; ++l) {
        const LevelSpec& L = P->levels[l];
        if (L.src == kSrcList) {
            GS_CUDA(launch_chained(k_bits_count, nb, th, 0, st, E, l, L));
            GS_CUDA(launch_chained(k_bits_write, nb, th, 0, st, E, l, L, l == 0 ? 1 : 0));
            nl_launch += 2;
            if (l == 0) {
                if (phase_ev) GS_CUDA(cudaEventRecord(phase_ev[1], st));
                continue;
            }
        }
        GS_CUDA(launch_chained(k_range, dim3(g->range_blocks), th, 0, st, E, l, L));
        GS_CUDA(launch_chained(k_expand, dim3(g->expand_blocks), th, 0, st, E, l, L));
        nl_launch += 2;
        if (phase_ev) GS_CUDA(cudaEventRecord(phase_ev[l + 1], st));
    }
    const int last = P->n_levels - 1;
    EnumSpec F{};
    F.n_leaves = P->n_leaves;
    F.n_vars = P->n_vars;
    for (int j = 0; j < P->n_leaves; ++j) F.leaf[j] = P->leaves[j];
    for (int v = 0; v < P->n_vars; ++v) F.var_src[v] = P->var_src[v];
    for (int l = 0; l < P->n_levels; ++l) F.col_of_level[l] = P->levels[l].var;
    for (int j = 0; j < P->n_leaves; ++j) F.col_of_leaf[j] = P->leaves[j].var;
    GS_CUDA(launch_chained(k_enum_range, nb, th, 0, st, E, last, F));
    GS_CUDA(launch_chained(k_enum_write, nb, th, 0, st, E, last, F));
    nl_launch += 2;
    if (phase_ev) GS_CUDA(cudaEventRecord(phase_ev[P->n_levels + 1], st));
    if (launches) *launches = nl_launch;
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
