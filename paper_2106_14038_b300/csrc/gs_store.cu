// Store build (Sec. 6.2): triples -> deduplicated CSR and CSC RDF matrices
// whose entries carry uint32 predicate labels, each row sorted by
// (label, other end). Off the per-query path: runs once per graph.
//
// Steps, all on the device: pack each triple into a 64-bit key
// (row | label | col), LSD radix sort, drop equal neighbours, split the
// keys into idx / lab arrays and derive the row pointers; then list the
// rows longer than kHeavyDeg and cut them into chunks for the scan.
#include <algorithm>
#include <cstring>

#include "gs_device.cuh"

namespace gs {

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

// Heavy rows: per row, (1 << 36) per heavy row plus its chunk count.
constexpr int kHeavyShift = 36;

__global__ void k_heavy_counts(const uint32_t* __restrict__ ptr, uint32_t N,
                               uint64_t* __restrict__ cnt) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t d = ptr[r + 1] - ptr[r];
        cnt[r] = d > kHeavyDeg ? ((1ull << kHeavyShift) | ((d + kHeavyChunk - 1) / kHeavyChunk)) : 0ull;
    }
}

__global__ void k_heavy_write(const uint32_t* __restrict__ ptr, uint32_t N,
                              const uint64_t* __restrict__ off, uint32_t* __restrict__ hrow,
                              uint32_t* __restrict__ chunk_h, uint32_t* __restrict__ chunk_start) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t b = ptr[r], d = ptr[r + 1] - b;
        if (d <= kHeavyDeg) continue;
        uint64_t o = off[r];
        uint32_t h = (uint32_t)(o >> kHeavyShift);
        uint64_t c = o & ((1ull << kHeavyShift) - 1);
        hrow[h] = (uint32_t)r;
        uint32_t nc = (d + kHeavyChunk - 1) / kHeavyChunk;
        for (uint32_t j = 0; j < nc; ++j) {
            chunk_h[c + j] = h;
            chunk_start[c + j] = b + j * kHeavyChunk;
        }
    }
}

// Scan tiles: runs of consecutive light rows (degree <= kHeavyDeg) cut
// every kTileLabels light labels, every kTileRows rows and at every heavy
// row. With pre[r] = (heavy rows before r) << 40 | (light labels before r),
// a light row's tile key is (heavy rows before, light labels / kTileLabels,
// r / kTileRows); a tile is a maximal run of light rows with one key, so it
// holds at most kTileRows rows and kTileLabels + kHeavyDeg labels.
constexpr uint64_t kLow40 = (1ull << 40) - 1;

__device__ __forceinline__ uint64_t tile_key(uint64_t pre, uint32_t r) {
    return ((pre >> 40) << 40) | ((uint64_t)(r / kTileRows) << 20) | ((pre & kLow40) / kTileLabels);
}

__global__ void k_tile_prep(const uint32_t* __restrict__ ptr, uint32_t N, uint64_t* __restrict__ val) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t d = ptr[r + 1] - ptr[r];
        val[r] = d > kHeavyDeg ? (1ull << 40) : (uint64_t)d;
    }
}

__device__ __forceinline__ bool tile_start(const uint32_t* __restrict__ ptr,
                                           const uint64_t* __restrict__ pre, uint32_t r) {
    if (ptr[r + 1] - ptr[r] > kHeavyDeg) return false;
    if (r == 0) return true;
    if (ptr[r] - ptr[r - 1] > kHeavyDeg) return true;
    return tile_key(pre[r], r) != tile_key(pre[r - 1], r - 1);
}

__global__ void k_tile_flags(const uint32_t* __restrict__ ptr, uint32_t N,
                             const uint64_t* __restrict__ pre, uint64_t* __restrict__ flg) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x)
        flg[r] = tile_start(ptr, pre, (uint32_t)r) ? 1ull : 0ull;
}

__global__ void k_tile_write(const uint32_t* __restrict__ ptr, uint32_t N,
                             const uint64_t* __restrict__ pre, const uint64_t* __restrict__ tix,
                             uint2* __restrict__ tiles) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < N;
         r += (uint64_t)gridDim.x * blockDim.x) {
        if (!tile_start(ptr, pre, (uint32_t)r)) continue;
        const uint64_t key = tile_key(pre[r], (uint32_t)r);
        uint32_t e = (uint32_t)r + 1;
        while (e < N && ptr[e + 1] - ptr[e] <= kHeavyDeg && tile_key(pre[e], e) == key) ++e;
        tiles[tix[r]] = make_uint2((uint32_t)r, e - (uint32_t)r);
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
    S.ptr = (uint32_t*)g->alloc.get(sizeof(uint32_t) * ((uint64_t)g->N + 1), st);
    S.idx = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (M + 4), st);
    S.lab = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (M + 4), st);
    if (!S.ptr || !S.idx || !S.lab) { set_error("gs_load_triples: out of device memory"); return GS_ENOMEM; }
    GS_CUDA(cudaMemsetAsync(S.idx + M, 0, 16, st));
    GS_CUDA(cudaMemsetAsync(S.lab + M, 0, 16, st));
    k_uniq_write<<<nb, kThreads, 0, st>>>(keys, n_dev, boff, vb, lb, S.idx, S.lab, S.ptr);
    k_ptr_tail<<<nb, kThreads, 0, st>>>(keys, n, vb, lb, g->N, M, S.ptr);
    GS_CUDA(cudaGetLastError());

    // heavy rows and their chunks
    uint64_t* cnt = tmp;   // N + 1 entries fit: tmp holds n >= ... keys; use a fresh buffer if short
    bool own_cnt = false;
    if (n < (uint64_t)g->N + 1) {
        cnt = (uint64_t*)g->alloc.get(sizeof(uint64_t) * ((uint64_t)g->N + 1), st);
        if (!cnt) { set_error("gs_load_triples: out of device memory"); return GS_ENOMEM; }
        own_cnt = true;
    }
    uint64_t nrows = g->N;
    GS_CUDA(cudaMemcpyAsync(n_dev, &nrows, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    k_heavy_counts<<<nb, kThreads, 0, st>>>(S.ptr, g->N, cnt);
    k_block_sums_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, bsum, nullptr);
    k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, boff, nb, tot, nullptr);
    k_scan_apply_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, boff, nullptr);
    uint64_t ht = 0;
    GS_CUDA(cudaMemcpyAsync(&ht, tot, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    S.n_heavy = (uint32_t)(ht >> kHeavyShift);
    S.n_chunks = (uint32_t)(ht & ((1ull << kHeavyShift) - 1));
    S.hrow = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (S.n_heavy + 1), st);
    S.chunk_h = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (S.n_chunks + 1), st);
    S.chunk_start = (uint32_t*)g->alloc.get(sizeof(uint32_t) * (S.n_chunks + 1), st);
    if (!S.hrow || !S.chunk_h || !S.chunk_start) {
        if (own_cnt) g->alloc.put(cnt, st);
        set_error("gs_load_triples: out of device memory");
        return GS_ENOMEM;
    }
    k_heavy_write<<<nb, kThreads, 0, st>>>(S.ptr, g->N, cnt, S.hrow, S.chunk_h, S.chunk_start);
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamSynchronize(st));

    // scan tiles: pre = prefix of (heavy << 40 | light degree), flags, their prefix
    uint64_t* flg = keys;   // the sorted keys are no longer needed
    bool own_flg = false;
    if (n < (uint64_t)g->N + 1) {
        flg = (uint64_t*)g->alloc.get(sizeof(uint64_t) * ((uint64_t)g->N + 1), st);
        if (!flg) {
            if (own_cnt) g->alloc.put(cnt, st);
            set_error("gs_load_triples: out of device memory");
            return GS_ENOMEM;
        }
        own_flg = true;
    }
    k_tile_prep<<<nb, kThreads, 0, st>>>(S.ptr, g->N, cnt);
    k_block_sums_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, bsum, nullptr);
    k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, boff, nb, tot, nullptr);
    k_scan_apply_u64<<<nb, kThreads, 0, st>>>(cnt, n_dev, boff, nullptr);
    k_tile_flags<<<nb, kThreads, 0, st>>>(S.ptr, g->N, cnt, flg);
    k_block_sums_u64<<<nb, kThreads, 0, st>>>(flg, n_dev, bsum, nullptr);
    k_scan_block_sums<<<1, kThreads, 0, st>>>(bsum, boff, nb, tot, nullptr);
    k_scan_apply_u64<<<nb, kThreads, 0, st>>>(flg, n_dev, boff, nullptr);
    uint64_t nt = 0;
    GS_CUDA(cudaMemcpyAsync(&nt, tot, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    S.n_tiles = (uint32_t)nt;
    S.tiles = (uint2*)g->alloc.get(sizeof(uint2) * (nt + 1), st);
    if (!S.tiles) {
        if (own_cnt) g->alloc.put(cnt, st);
        if (own_flg) g->alloc.put(flg, st);
        set_error("gs_load_triples: out of device memory");
        return GS_ENOMEM;
    }
    k_tile_write<<<nb, kThreads, 0, st>>>(S.ptr, g->N, cnt, flg, S.tiles);
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamSynchronize(st));
    if (own_flg) g->alloc.put(flg, st);
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaStreamSynchronize(st));
    if (own_cnt) g->alloc.put(cnt, st);
    return GS_OK;
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
        g->alloc.put(S->hrow, st); g->alloc.put(S->chunk_h, st); g->alloc.put(S->chunk_start, st);
        g->alloc.put(S->tiles, st);
        *S = Store{};
    }
}

}  // namespace gs
