// Store build (Sec. 6.2): triples -> deduplicated CSR and CSC RDF matrices
// whose entries carry uint32 predicate labels, each row sorted by
// (label, other end). Off the per-query path: runs once per graph.
//
// Steps, all on the device: pack each triple into a 64-bit key
// (row | label | col), LSD radix sort, drop equal neighbours, split the
// keys into idx / lab arrays and derive the row pointers; then cut the
// orientation into the triple scan's equal-cost work items.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gs_device.cuh"

namespace gs {

__global__ void k_u64_to_u32(const uint64_t* __restrict__ a, uint64_t n, uint32_t* __restrict__ b);

constexpr int kRsWarps = kThreads / 32;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsWarps * 32 * kRsRounds;   // 4096 keys per block tile

static inline int bits_for(uint64_t maxval) {          // bits to hold 0..maxval
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b < 1 ? 1 : b;
}

__device__ __forceinline__ void rs_segment(uint64_t n, uint32_t b, uint32_t nb, uint64_t& beg,
                                           uint64_t& end) {
    uint64_t tiles = (n + kRsTile - 1) / kRsTile;
    uint64_t per = (tiles + nb - 1) / nb;
    beg = (uint64_t)b * per * kRsTile;
    end = beg + per * kRsTile;
    if (beg > n) beg = n;
    if (end > n) end = n;
}

// hist[d * nb + b] = number of keys of block b's segment with digit d.
__global__ void __launch_bounds__(kThreads) k_rs_hist(const uint64_t* __restrict__ keys, uint64_t n,
                                                      int shift, uint64_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t beg, end;
    rs_segment(n, blockIdx.x, gridDim.x, beg, end);
    for (uint64_t i = beg + threadIdx.x; i < end; i += kThreads)
        atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of block b's segment by digit. hoff holds the exclusive
// scan of hist in digit-major order. Within a tile the key order is
// (warp, round, lane), which is the input order, so the sort is stable.
__global__ void __launch_bounds__(kThreads) k_rs_scatter(const uint64_t* __restrict__ in,
                                                         uint64_t* __restrict__ out, uint64_t n,
                                                         int shift,
                                                         const uint64_t* __restrict__ hoff) {
    __shared__ uint32_t whist[kRsWarps][256];
    __shared__ uint32_t wpre[kRsWarps][256];
    __shared__ uint64_t run[256];
    __shared__ uint32_t tcount[256];
    const uint32_t t = threadIdx.x, lane = t & 31, w = t >> 5;
    run[t] = hoff[(uint64_t)t * gridDim.x + blockIdx.x];
    for (int k = 0; k < kRsWarps; ++k) whist[k][t] = 0;
    __syncthreads();
    uint64_t beg, end;
    rs_segment(n, blockIdx.x, gridDim.x, beg, end);
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (uint64_t tile = beg; tile < end; tile += kRsTile) {
        uint64_t key[kRsRounds];
        uint32_t dig[kRsRounds], rank[kRsRounds];
        const uint64_t wbase = tile + (uint64_t)w * 32 * kRsRounds;
#pragma unroll
        for (int r = 0; r < kRsRounds; ++r) {
            uint64_t i = wbase + (uint64_t)r * 32 + lane;
            bool v = i < end;
            key[r] = v ? in[i] : 0ull;
            dig[r] = v ? (uint32_t)((key[r] >> shift) & 255u) : 256u;
        }
#pragma unroll
        for (int r = 0; r < kRsRounds; ++r) {
            uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
            uint32_t leader = __ffs(peers) - 1;
            uint32_t c0 = dig[r] < 256u ? whist[w][dig[r]] : 0u;
            __syncwarp();
            if (lane == leader && dig[r] < 256u) whist[w][dig[r]] = c0 + __popc(peers);
            __syncwarp();
            rank[r] = c0 + __popc(peers & lt_mask);
        }
        __syncthreads();
        {
            uint32_t s = 0;
            for (int k = 0; k < kRsWarps; ++k) {
                uint32_t c = whist[k][t];
                wpre[k][t] = s;
                s += c;
            }
            tcount[t] = s;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRsRounds; ++r)
            if (dig[r] < 256u) out[run[dig[r]] + wpre[w][dig[r]] + rank[r]] = key[r];
        __syncthreads();
        run[t] += tcount[t];
        for (int k = 0; k < kRsWarps; ++k) whist[k][t] = 0;
        __syncthreads();
    }
}

gs_status radix_sort_u64(const gs_graph* g, uint64_t** keys, uint64_t** tmp, uint64_t n,
                         int lo_bit, int hi_bit, cudaStream_t st) {
    if (n <= 1 || hi_bit <= lo_bit) return GS_OK;
    uint64_t tiles = (n + kRsTile - 1) / kRsTile;
    uint32_t nb = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)g->n_blocks);
    size_t hbytes = sizeof(uint64_t) * 256 * nb;
    uint64_t* hist = (uint64_t*)g->alloc.get(hbytes, st);
    uint64_t* bsum = (uint64_t*)g->alloc.get(sizeof(uint64_t) * (kBlocks + 2), st);
    if (!hist || !bsum) {
        g->alloc.put(hist, st); g->alloc.put(bsum, st);
        set_error("radix sort: out of device memory");
        return GS_ENOMEM;
    }
    uint64_t* aux = (uint64_t*)g->alloc.get(sizeof(uint64_t) * (kBlocks + 2), st);
    if (!aux) { g->alloc.put(hist, st); g->alloc.put(bsum, st); set_error("radix sort: oom"); return GS_ENOMEM; }
    uint64_t hn = 256ull * nb;
    uint64_t* hn_dev = aux + kBlocks;      // device copy of the histogram length
    GS_CUDA(cudaMemcpyAsync(hn_dev, &hn, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    int sb = g->n_blocks;
    for (int shift = lo_bit; shift < hi_bit; shift += 8) {
        k_rs_hist<<<nb, kThreads, 0, st>>>(*keys, n, shift, hist);
        k_block_sums_u64<<<sb, kThreads, 0, st>>>(hist, hn_dev, bsum, nullptr);
        k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, aux, sb, aux + kBlocks + 1, nullptr);
        k_scan_apply_u64<<<sb, kThreads, 0, st>>>(hist, hn_dev, aux, nullptr);
        k_rs_scatter<<<nb, kThreads, 0, st>>>(*keys, *tmp, n, shift, hist);
        std::swap(*keys, *tmp);
    }
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamSynchronize(st));   // hn lives on the host stack
    g->alloc.put(hist, st);
    g->alloc.put(bsum, st);
    g->alloc.put(aux, st);
    return GS_OK;
}

// ------------------------------------------------------------------ //

// key = row << (lb + vb) | label << vb | col, with row/col = (s, o) or (o, s)
__global__ void k_pack(const uint32_t* __restrict__ s, const uint32_t* __restrict__ p,
                       const uint32_t* __restrict__ o, uint64_t n, uint32_t N, uint32_t P,
                       int by_col, int vb, int lb, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ bad) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t a = s[i], l = p[i], b = o[i];
        if (a >= N || b >= N || l < 1 || l > P) {
            atomicOr(bad, 1u);
            keys[i] = 0;
            continue;
        }
        uint64_t row = by_col ? b : a, col = by_col ? a : b;
        keys[i] = (row << (lb + vb)) | ((uint64_t)l << vb) | col;
    }
}

__global__ void k_uniq_count(const uint64_t* __restrict__ keys, const uint64_t* n_ptr,
                             uint64_t* __restrict__ bsum) {
    uint64_t beg, end;
    block_chunk(*n_ptr, blockIdx.x, gridDim.x, beg, end);
    uint64_t c = 0;
    for (uint64_t i = beg + threadIdx.x; i < end; i += kThreads)
        c += (i == 0 || keys[i] != keys[i - 1]);
    c = block_sum_u64(c);
    if (threadIdx.x == 0) bsum[blockIdx.x] = c;
}

// Writes the unique entries in order and the row pointers of their rows.
__global__ void k_uniq_write(const uint64_t* __restrict__ keys, const uint64_t* n_ptr,
                             const uint64_t* __restrict__ boff, int vb, int lb,
                             uint32_t* __restrict__ idx, uint32_t* __restrict__ lab,
                             uint32_t* __restrict__ ptr) {
    const uint64_t n = *n_ptr;
    uint64_t beg, end;
    block_chunk(n, blockIdx.x, gridDim.x, beg, end);
    const uint64_t vmask = (1ull << vb) - 1, lmask = (1ull << lb) - 1;
    uint64_t carry = boff[blockIdx.x];
    for (uint64_t base = beg; base < end; base += kThreads) {
        uint64_t i = base + threadIdx.x;
        bool in = i < end;
        uint64_t k = in ? keys[i] : 0;
        bool u = in && (i == 0 || k != keys[i - 1]);
        uint64_t t;
        uint64_t j = carry + block_excl_scan_u64(u ? 1 : 0, &t);
        if (u) {
            idx[j] = (uint32_t)(k & vmask);
            lab[j] = (uint32_t)((k >> vb) & lmask);
            int64_t r = (int64_t)(k >> (vb + lb));
            int64_t rp = i == 0 ? -1 : (int64_t)(keys[i - 1] >> (vb + lb));
            for (int64_t rr = rp + 1; rr <= r; ++rr) ptr[rr] = (uint32_t)j;
        }
        carry += t;
    }
}

// Rows after the last stored row point at the end.
__global__ void k_ptr_tail(const uint64_t* __restrict__ keys, uint64_t n, int vb, int lb,
                           uint32_t N, uint64_t M, uint32_t* __restrict__ ptr) {
    int64_t last = n ? (int64_t)(keys[n - 1] >> (vb + lb)) : -1;
    for (int64_t r = last + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= (int64_t)N;
         r += (int64_t)gridDim.x * blockDim.x)
        ptr[r] = (uint32_t)M;
}

// Row-start bits: bit ptr[r] for every non-empty row r.
__global__ void k_heads(const uint32_t* __restrict__ ptr, uint32_t N, uint32_t* __restrict__ heads) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
        const uint32_t b = ptr[r];
        if (b < ptr[r + 1]) atomicOr(heads + (b >> 5), 1u << (b & 31));
    }
}

// Scan items (merge path over row ends and labels): boundary c sits at cost
// d = min(c * kScanItemCost, w N + M); the rows completed before it are the
// largest r with w r + ptr[r] <= d, the labels consumed min(d - w r, ptr[r+1]).
__global__ void k_items(const uint32_t* __restrict__ ptr, uint32_t N, uint64_t M, uint32_t w,
                        uint32_t n_items, uint2* __restrict__ items) {
    const uint64_t total = (uint64_t)w * N + M;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= n_items;
         c += gridDim.x * blockDim.x) {
        const uint64_t d = min((uint64_t)c * kScanItemCost, total);
        uint32_t lo = 0, hi = N;                      // w * 0 + ptr[0] = 0 <= d
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo + 1) / 2;
            if ((uint64_t)w * mid + ptr[mid] <= d) lo = mid; else hi = mid - 1;
        }
        const uint64_t k = lo < N ? min(d - (uint64_t)w * lo, (uint64_t)ptr[lo + 1]) : M;
        items[c] = make_uint2(lo, (uint32_t)k);
    }
}

static gs_status build_dir(gs_graph* g, const uint32_t* s, const uint32_t* p, const uint32_t* o,
                           uint64_t n, int by_col, int vb, int lb, uint64_t* k0, uint64_t* k1,
                           uint64_t* misc, Store& S, cudaStream_t st) {
    const int nb = g->n_blocks;
    uint32_t* bad = (uint32_t*)(misc + 2 * kBlocks + 8);
    GS_CUDA(cudaMemsetAsync(bad, 0, sizeof(uint32_t), st));
    k_pack<<<nb, kThreads, 0, st>>>(s, p, o, n, g->N, g->P, by_col, vb, lb, k0, bad);
    GS_CUDA(cudaGetLastError());
    uint32_t hbad = 0;
    GS_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (hbad) {
        set_error("gs_load_triples: a triple has a vertex >= n_vertices or a predicate outside 1..n_predicates");
        return GS_EINVAL;
    }
    uint64_t* keys = k0;
    uint64_t* tmp = k1;
    gs_status rc = radix_sort_u64(g, &keys, &tmp, n, 0, 2 * vb + lb, st);
    if (rc != GS_OK) return rc;

    uint64_t* bsum = misc;
    uint64_t* boff = misc + kBlocks;
    uint64_t* n_dev = misc + 2 * kBlocks;
    uint64_t* tot = misc + 2 * kBlocks + 1;
    GS_CUDA(cudaMemcpyAsync(n_dev, &n, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    k_uniq_count<<<nb, kThreads, 0, st>>>(keys, n_dev, bsum);
    k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, boff, nb, tot, nullptr);
    uint64_t M = 0;
    GS_CUDA(cudaMemcpyAsync(&M, tot, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (M >= (1ull << 32) - 8) {
        set_error("gs_load_triples: %llu distinct triples exceed the 32-bit entry index",
                  (unsigned long long)M);
        return GS_EINVAL;
    }
    g->M = M;
    S.ptr = (uint32_t*)g->alloc.get(sizeof(uint32_t) * ((uint64_t)g->N + 1 + 4), st);
    S.idx = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (M + 4), st);
    S.lab = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (M + 4), st);
    if (!S.ptr || !S.idx || !S.lab) { set_error("gs_load_triples: out of device memory"); return GS_ENOMEM; }
    GS_CUDA(cudaMemsetAsync(S.ptr + g->N + 1, 0, 16, st));
    GS_CUDA(cudaMemsetAsync(S.idx + M, 0, 16, st));
    GS_CUDA(cudaMemsetAsync(S.lab + M, 0, 16, st));
    k_uniq_write<<<nb, kThreads, 0, st>>>(keys, n_dev, boff, vb, lb, S.idx, S.lab, S.ptr);
    k_ptr_tail<<<nb, kThreads, 0, st>>>(keys, n, vb, lb, g->N, M, S.ptr);
    GS_CUDA(cudaGetLastError());
    return store_items(g, S, M, st);
}

gs_status store_items(const gs_graph* g, Store& S, uint64_t M, cudaStream_t st) {
    const int nb = g->n_blocks;
    // scan items
    const uint32_t w = 1;   // one cost unit per row end
    const uint64_t cost = (uint64_t)w * g->N + M;
    const uint64_t ni = (cost + kScanItemCost - 1) / kScanItemCost;
    if (ni >= (1ull << 31)) {
        set_error("gs_load_triples: %llu scan items exceed the 31-bit item index",
                  (unsigned long long)ni);
        return GS_EINVAL;
    }
    S.n_items = (uint32_t)ni;
    S.items = (uint2*)g->alloc.get(sizeof(uint2) * (ni + 1), st);
    if (!S.items) { set_error("gs_load_triples: out of device memory"); return GS_ENOMEM; }
    k_items<<<(unsigned)std::min<uint64_t>((ni + kThreads) / kThreads, (uint64_t)nb), kThreads, 0, st>>>(
        S.ptr, g->N, M, w, S.n_items, S.items);
    const uint64_t hwords = M / 32 + 8;
    S.heads = (uint32_t*)g->alloc.get(sizeof(uint32_t) * hwords, st);
    if (!S.heads) { set_error("gs_load_triples: out of device memory"); return GS_ENOMEM; }
    GS_CUDA(cudaMemsetAsync(S.heads, 0, sizeof(uint32_t) * hwords, st));
    k_heads<<<nb, kThreads, 0, st>>>(S.ptr, g->N, S.heads);
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

// Label directory (see Store): a row longer than kDirMin is walked run by
// run, each step jumping past the current label with a search (at most P
// runs per row), to count its runs (write = 0) or write them.
__global__ void k_dir_rows(const uint32_t* __restrict__ ptr, const uint32_t* __restrict__ lab,
                           uint32_t N, uint64_t* __restrict__ cnt, const uint64_t* __restrict__ off,
                           uint32_t* __restrict__ dlab, uint32_t* __restrict__ dpos, int write) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = ptr[r], e = ptr[r + 1];
        uint64_t c = 0;
        if (e - b > kDirMin) {
            uint64_t at = write ? off[r] : 0;
            for (uint32_t j = b; j < e;) {
                const uint32_t l = lab[j];
                if (write) { dlab[at] = l; dpos[at] = j; ++at; }
                ++c;
                j = lower_bound_u32(lab, j, e, l + 1);
            }
        }
        if (!write) cnt[r] = c;
    }
}

// Builds S's label directory (dir_off over the N rows, u32: the runs are at
// most M < 2^32). Synchronizes st.
static gs_status build_label_dir(const gs_graph* g, Store& S, cudaStream_t st) {
    const uint32_t N = g->N;
    const int nb = g->n_blocks;
    uint64_t* cnt = (uint64_t*)g->alloc.get(sizeof(uint64_t) * ((uint64_t)N + 1), st);
    uint64_t* misc = (uint64_t*)g->alloc.get(sizeof(uint64_t) * (2 * kBlocks + 8), st);
    auto done = [&](gs_status r) { g->alloc.put(cnt, st); g->alloc.put(misc, st); return r; };
    if (!cnt || !misc) { set_error("gs_load_triples: out of device memory (label directory)"); return done(GS_ENOMEM); }
    uint64_t* bsum = misc;
    uint64_t* boff = misc + kBlocks;
    uint64_t* total = misc + 2 * kBlocks;
    uint64_t* n_dev = total + 1;
    const uint64_t n_host = (uint64_t)N + 1;
    GS_CUDA(cudaMemcpyAsync(n_dev, &n_host, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemsetAsync(cnt + N, 0, sizeof(uint64_t), st));
    k_dir_rows<<<nb, kThreads, 0, st>>>(S.ptr, S.lab, N, cnt, nullptr, nullptr, nullptr, 0);
    k_block_sums_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, bsum, nullptr);
    k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, boff, (uint32_t)nb, total, nullptr);
    k_scan_apply_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, boff, nullptr);   // cnt[r]: first run of row r
    uint64_t runs = 0;
    GS_CUDA(cudaMemcpyAsync(&runs, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    S.dir_runs = runs;
    S.dir_off = (uint32_t*)g->alloc.get(sizeof(uint32_t) * ((uint64_t)N + 1 + 4), st);
    S.dir_lab = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (runs + 4), st);
    S.dir_pos = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (runs + 4), st);
    if (!S.dir_off || !S.dir_lab || !S.dir_pos) { set_error("gs_load_triples: out of device memory (label directory)"); return done(GS_ENOMEM); }
    GS_CUDA(cudaMemsetAsync(S.dir_lab + runs, 0, 16, st));   // padding read by 16-byte loads
    GS_CUDA(cudaMemsetAsync(S.dir_pos + runs, 0, 16, st));
    GS_CUDA(cudaMemsetAsync(S.dir_off + N + 1, 0, 16, st));
    k_dir_rows<<<nb, kThreads, 0, st>>>(S.ptr, S.lab, N, nullptr, cnt, S.dir_lab, S.dir_pos, 1);
    k_u64_to_u32<<<nb, kThreads, 0, st>>>(cnt, (uint64_t)N + 1, S.dir_off);
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamSynchronize(st));
    return done(GS_OK);
}

// Per predicate label l of one orientation: cnt[l] = entries with label l,
// rows[l] = rows holding label l. Rows are sorted by (label, other end), so
// the entries of (row, l) form one run: a run starts at a row start or
// where the label changes. Labels of a warp's 32 consecutive entries are
// aggregated with __match_any_sync (one atomic per distinct label).
__global__ void k_label_stats(const uint32_t* __restrict__ lab, const uint32_t* __restrict__ heads,
                              uint64_t M, unsigned long long* __restrict__ cnt,
                              unsigned long long* __restrict__ rows) {
    const uint32_t lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; base < M;
         base += stride) {
        const uint64_t k = base + lane;
        const bool in = k < M;
        const uint32_t l = in ? lab[k] : 0xffffffffu;
        const bool run = in && (((heads[k >> 5] >> (k & 31)) & 1u) || k == 0 || lab[k - 1] != l);
        const uint32_t same = __match_any_sync(0xffffffffu, l);
        const uint32_t runs = __ballot_sync(0xffffffffu, run) & same;
        if (in && lane == (uint32_t)(__ffs(same) - 1)) {
            atomicAdd(cnt + l, (unsigned long long)__popc(same));
            if (runs) atomicAdd(rows + l, (unsigned long long)__popc(runs));
        }
    }
}

// Label statistics of both orientations into g->lab_cnt / g->lab_rows.
static gs_status label_stats(gs_graph* g, cudaStream_t st) {
    const uint64_t np = (uint64_t)g->P + 1;
    unsigned long long* d = (unsigned long long*)g->alloc.get(sizeof(unsigned long long) * 4 * np, st);
    if (!d) { set_error("gs_load_triples: out of device memory for label statistics"); return GS_ENOMEM; }
    GS_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * 4 * np, st));
    for (int dir = 0; dir < 2; ++dir) {
        const Store& S = dir ? g->in : g->out;
        if (g->M) k_label_stats<<<g->n_blocks, kThreads, 0, st>>>(S.lab, S.heads, g->M, d + 2 * dir * np,
                                                                 d + (2 * dir + 1) * np);
    }
    GS_CUDA(cudaGetLastError());
    std::vector<unsigned long long> h(4 * np);
    cudaError_t e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * 4 * np,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    g->alloc.put(d, st);
    if (e != cudaSuccess) return cuda_fail(e, "gs_load_triples (label statistics)");
    for (int dir = 0; dir < 2; ++dir) {
        g->lab_cnt[dir].assign(h.begin() + 2 * dir * np, h.begin() + (2 * dir + 1) * np);
        g->lab_rows[dir].assign(h.begin() + (2 * dir + 1) * np, h.begin() + (2 * dir + 2) * np);
    }
    return GS_OK;
}

__global__ void k_u64_to_u32(const uint64_t* __restrict__ a, uint64_t n, uint32_t* __restrict__ b) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        b[i] = (uint32_t)a[i];
}

gs_status build_store(gs_graph* g, const uint32_t* s, const uint32_t* p, const uint32_t* o,
                      uint64_t n, bool on_device, cudaStream_t st) {
    const int vb = bits_for(g->N ? g->N - 1 : 0);
    const int lb = bits_for(g->P);
    if (2 * vb + lb > 64) {
        set_error("gs_load_triples: 2*%d vertex bits + %d label bits exceed a 64-bit key", vb, lb);
        return GS_EINVAL;
    }
    const uint32_t* ds = s;
    const uint32_t* dp = p;
    const uint32_t* dpo = o;
    uint32_t* copy = nullptr;
    uint64_t nn = n ? n : 1;
    if (!on_device && n) {
        copy = (uint32_t*)g->alloc.get(sizeof(uint32_t) * 3 * nn, st);
        if (!copy) { set_error("gs_load_triples: out of device memory for the input copy"); return GS_ENOMEM; }
        GS_CUDA(cudaMemcpyAsync(copy, s, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
        GS_CUDA(cudaMemcpyAsync(copy + nn, p, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
        GS_CUDA(cudaMemcpyAsync(copy + 2 * nn, o, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
        ds = copy; dp = copy + nn; dpo = copy + 2 * nn;
    }
    uint64_t* k0 = (uint64_t*)g->alloc.get(sizeof(uint64_t) * nn, st);
    uint64_t* k1 = (uint64_t*)g->alloc.get(sizeof(uint64_t) * nn, st);
    uint64_t* misc = (uint64_t*)g->alloc.get(sizeof(uint64_t) * (2 * kBlocks + 16), st);
    gs_status rc = GS_OK;
    if (!k0 || !k1 || !misc) { set_error("gs_load_triples: out of device memory for sort keys"); rc = GS_ENOMEM; }
    if (rc == GS_OK) rc = build_dir(g, ds, dp, dpo, n, 0, vb, lb, k0, k1, misc, g->out, st);
    if (rc == GS_OK) rc = build_dir(g, ds, dp, dpo, n, 1, vb, lb, k0, k1, misc, g->in, st);
    if (rc == GS_OK) rc = build_label_dir(g, g->out, st);
    if (rc == GS_OK) rc = build_label_dir(g, g->in, st);
    if (rc == GS_OK) rc = label_stats(g, st);
    g->alloc.put(k0, st);
    g->alloc.put(k1, st);
    g->alloc.put(misc, st);
    g->alloc.put(copy, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == GS_OK && e != cudaSuccess) rc = cuda_fail(e, "gs_load_triples");
    return rc;
}

void free_store(gs_graph* g, cudaStream_t st) {
    for (Store* S : {&g->out, &g->in}) {
        g->alloc.put(S->ptr, st); g->alloc.put(S->idx, st); g->alloc.put(S->lab, st);
        g->alloc.put(S->items, st);
        g->alloc.put(S->heads, st);
        g->alloc.put(S->dir_off, st);
        g->alloc.put(S->dir_lab, st);
        g->alloc.put(S->dir_pos, st);
        *S = Store{};
    }
}

}  // namespace gs
