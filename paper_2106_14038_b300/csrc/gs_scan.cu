// Triple scan: candidate vectors of query variables by grouped predicate
// selection (Sec. 5, Step 1). For a variable u with out-predicates O(u)
// (u is the subject) and in-predicates I(u) (u is the object):
//
//     v_u = AND_{p in O(u)} (A (x) u_p)  AND  AND_{p in I(u)} (A^T (x) u_p)
//
// (Eq. 17 with only outgoing edges, Eq. 21 with both; Eq. 4 and Eq. 5 for
// the single selections). All predicates of the query are tested in one
// pass over the label array of each orientation:
//   1. k_scan<false> streams the CSR labels and writes, per vertex, the mask
//      of query out-predicates its row holds;
//   2. k_scan<true> streams the CSC labels, forms the in-mask per vertex,
//      combines it with the out-mask and ORs one bit per variable into the
//      candidate vectors (warp ballot -> one word per 32 vertices);
//   3. k_scan_fixup finishes the vertices whose column is heavy.
//
// Work items, taken by CTAs from a device counter: store tiles (a run of at
// most kTileRows light rows, whose labels are one contiguous span) and
// chunks of kHeavyChunk entries of the rows longer than kHeavyDeg. A tile's
// row pointers are loaded once into shared memory; its label span is then
// staged in rounds of 8192 labels (coalesced 16-byte loads, a 16-bit one-hot
// predicate bit per label in shared memory) and reduced per row by threads
// that each OR 32 consecutive labels word by word (a segmented OR). Bytes moved per
// pass: 4(N+1) row pointers + 4M labels, plus a 4N mask written and read
// once and N/8 per vector.
#include <algorithm>

#include "gs_device.cuh"

namespace gs {

struct ScanDev {
    uint32_t n_bvars;
    uint32_t need_out[kMaxVars];
    uint32_t need_in[kMaxVars];
    uint32_t out_pred[kMaxSlots];
    uint32_t in_pred[kMaxSlots];
    uint32_t n_out, n_in;
};

constexpr int kScanWarps = kThreads / 32;
constexpr uint32_t kSpWords = (kTileRows + 1 + 3) & ~3u;   // row pointers, 16-byte padded
constexpr int kScanUnroll = 4;   // 16-byte words per thread in flight

// label -> slot bit lookup in shared memory (P + 1 bytes: slot + 1, 0 = none)
__device__ __forceinline__ void fill_lut(uint8_t* lut, uint32_t P, const uint32_t* preds,
                                         uint32_t n) {
    for (uint32_t i = threadIdx.x; i <= P + 1; i += blockDim.x) lut[i] = 0;
    __syncthreads();
    if (threadIdx.x < n) lut[preds[threadIdx.x]] = (uint8_t)(threadIdx.x + 1);
    __syncthreads();
}

__device__ __forceinline__ uint32_t lut_bit(const uint8_t* lut, uint32_t P, uint32_t l) {
    uint32_t s = l <= P ? lut[l] : 0u;
    return s ? (1u << (s - 1)) : 0u;
}

// Largest j in [lo, hi] with sp[j] <= pos (requires sp[lo] <= pos).
__device__ __forceinline__ uint32_t search_row(const uint32_t* sp, uint32_t lo, uint32_t hi,
                                               uint32_t pos) {
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (sp[mid] <= pos) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// OR the query-predicate bits of one tile's labels into rm[0..nr).
// sp[0..nr] are the tile's row pointers (all rows light; at most
// kTileLabels + kHeavyDeg labels). The span is processed in rounds of
// kRound labels: the CTA loads them with coalesced 16-byte loads and stores
// each label's predicate bit (16-bit one-hot, 0 when not a query predicate)
// in shared memory; then every thread ORs its kPerThread consecutive bits
// word by word (two labels per 32-bit word) into the current row,
// splitting a word only where a row boundary falls inside it, and ORs each
// finished row into rm with one shared-memory atomic.
constexpr uint32_t kPerThread = 32;
constexpr uint32_t kRound = kThreads * kPerThread;        // 8192 labels per round

// lut holds slot + 1 (0: not a query predicate); (1 << s) >> 1 is the one-hot bit.
__device__ __forceinline__ uint32_t onehot(const uint8_t* lut, uint32_t P, uint32_t l) {
    const uint32_t s = lut[min(l, P + 1)];
    return (1u << s) >> 1;
}

__device__ __forceinline__ uint32_t fold16(uint32_t x) { return (x | (x >> 16)) & 0xffffu; }

__device__ __forceinline__ void tile_masks(const uint32_t* __restrict__ lab, const uint32_t* sp,
                                           uint32_t nr, uint32_t* rm, const uint8_t* lut,
                                           uint32_t P, uint16_t* bits) {
    const uint32_t ks = sp[0], ke = sp[nr];
    const uint4* v = reinterpret_cast<const uint4*>(lab);
    uint32_t rhint = 0;   // row of this thread's previous segment (rows only grow)
    for (uint32_t c0 = ks & ~3u; c0 < ke; c0 += kRound) {
        const uint32_t c1 = min(c0 + kRound, ke);
        // stage: bits of positions [c0, c1) (0 outside [ks, c1)), zero up to the round's end
        const uint32_t qa = c0 >> 2;
        const uint32_t nw = (c1 - c0 + 3) >> 2;
        constexpr uint32_t kBurst = 8;
        for (uint32_t base = threadIdx.x; base < kRound / 4; base += kBurst * kThreads) {
            uint4 x[kBurst];
#pragma unroll
            for (uint32_t u = 0; u < kBurst; ++u) {
                const uint32_t wi = base + u * kThreads;
                x[u] = wi < nw ? __ldcs(v + qa + wi) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (uint32_t u = 0; u < kBurst; ++u) {
                const uint32_t wi = base + u * kThreads;
                if (wi >= kRound / 4) break;
                const uint32_t k = c0 + 4 * wi;
                uint2 c = make_uint2(0, 0);
                if (wi < nw) {
                    uint32_t b0 = onehot(lut, P, x[u].x), b1 = onehot(lut, P, x[u].y);
                    uint32_t b2 = onehot(lut, P, x[u].z), b3 = onehot(lut, P, x[u].w);
                    if (k < ks || k + 3 >= c1) {           // an edge word of the span
                        if (k < ks || k >= c1) b0 = 0;
                        if (k + 1 < ks || k + 1 >= c1) b1 = 0;
                        if (k + 2 < ks || k + 2 >= c1) b2 = 0;
                        if (k + 3 < ks || k + 3 >= c1) b3 = 0;
                    }
                    c = make_uint2(b0 | (b1 << 16), b2 | (b3 << 16));
                }
                reinterpret_cast<uint2*>(bits)[wi] = c;
            }
        }
        __syncthreads();
        // consume: this thread's kPerThread consecutive positions, two per word
        const uint32_t p0 = c0 + threadIdx.x * kPerThread;
        const uint32_t first = max(p0, ks);
        const uint32_t stop = min(p0 + kPerThread, c1);
        if (first < stop) {
            uint32_t r = search_row(sp, rhint, nr - 1, first);
            uint32_t nxt = sp[r + 1];                 // start of the next row
            uint32_t acc = 0;
            const uint4* cw = reinterpret_cast<const uint4*>(bits + threadIdx.x * kPerThread);
#pragma unroll
            for (uint32_t i = 0; i < kPerThread / 8; ++i) {
                const uint4 q = cw[i];
                if (p0 + i * 8 + 8 <= nxt) {                   // all eight labels in row r
                    acc |= q.x | q.y | q.z | q.w;
                    continue;
                }
                const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (uint32_t t = 0; t < 4; ++t) {
                    const uint32_t pos = p0 + i * 8 + t * 2;   // first of the word's two labels
                    const uint32_t w = wv[t];
                    if (pos + 2 <= nxt) {                      // both labels in row r
                        acc |= w;
                    } else if (w) {
                        // a row boundary inside the word: place each half
                        for (uint32_t h = 0; h < 2; ++h) {
                            const uint32_t b = (w >> (16 * h)) & 0xffffu;
                            if (!b) continue;
                            const uint32_t pp = pos + h;
                            if (pp >= nxt) {
                                if (acc) atomicOr(rm + r, fold16(acc));
                                acc = 0;
                                while (sp[r + 1] <= pp) ++r;
                                nxt = sp[r + 1];
                            }
                            acc |= b;
                        }
                    }
                }
            }
            if (acc) atomicOr(rm + r, fold16(acc));
            rhint = r;
        }
        __syncthreads();
    }
}

// Block-cooperative OR over lab[b..e) (a heavy-row chunk).
__device__ __forceinline__ uint32_t chunk_mask(const uint32_t* __restrict__ lab, uint32_t b,
                                               uint32_t e, const uint8_t* lut, uint32_t P,
                                               uint32_t* red) {
    const uint4* v = reinterpret_cast<const uint4*>(lab);
    const uint32_t q0 = b >> 2, q1 = (e + 3) >> 2;
    constexpr uint32_t kStep = kThreads * kScanUnroll;
    uint32_t m = 0;
    for (uint32_t qb = q0; qb < q1; qb += kStep) {
        uint4 x[kScanUnroll];
#pragma unroll
        for (int u = 0; u < kScanUnroll; ++u) {
            uint32_t q = qb + (uint32_t)u * kThreads + threadIdx.x;
            x[u] = q < q1 ? __ldcs(v + q) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kScanUnroll; ++u) {
            uint32_t k = (qb + (uint32_t)u * kThreads + threadIdx.x) << 2;
            if (k >= b && k < e) m |= lut_bit(lut, P, x[u].x);
            if (k + 1 >= b && k + 1 < e) m |= lut_bit(lut, P, x[u].y);
            if (k + 2 >= b && k + 2 < e) m |= lut_bit(lut, P, x[u].z);
            if (k + 3 >= b && k + 3 < e) m |= lut_bit(lut, P, x[u].w);
        }
    }
    m = __reduce_or_sync(0xffffffffu, m);
    if (lane_id() == 0) atomicOr(red, m);
    __syncthreads();
    return *red;
}

// Heavy rows' mask slots, the candidate vectors and the work counters start
// at zero; the chunks and tiles OR into them.
__global__ void k_scan_zero(const uint32_t* __restrict__ hrow_out, uint32_t n_out_heavy,
                            uint32_t* __restrict__ mask_out, uint32_t* __restrict__ hmask_in,
                            uint32_t n_in_heavy, uint32_t* __restrict__ bits, uint64_t n_words,
                            uint32_t* __restrict__ counters) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t i = t; i < n_out_heavy; i += stride) mask_out[hrow_out[i]] = 0;
    for (uint32_t i = t; i < n_in_heavy; i += stride) hmask_in[i] = 0;
    for (uint64_t i = t; i < n_words; i += stride) bits[i] = 0;
    if (t < 2) counters[t] = 0;
}

__device__ __forceinline__ uint32_t eval_bits(const ScanDev& sd, uint32_t mo, uint32_t mi,
                                              uint32_t u) {
    return ((mo & sd.need_out[u]) == sd.need_out[u]) && ((mi & sd.need_in[u]) == sd.need_in[u]);
}

// Pass 1 (EVAL = false): out-masks of all rows into mask_out.
// Pass 2 (EVAL = true): in-masks of the light columns, combined with
// mask_out into the candidate vectors; heavy columns go to hmask_in.
template <bool EVAL>
__global__ void __launch_bounds__(kThreads) k_scan(DStore S, uint32_t P, const uint2* __restrict__ tiles,
                                                   uint32_t n_tiles,
                                                   const uint32_t* __restrict__ chunk_h,
                                                   const uint32_t* __restrict__ chunk_start,
                                                   const uint32_t* __restrict__ hrow,
                                                   uint32_t n_chunks, ScanDev sd,
                                                   uint32_t* __restrict__ mask_out,
                                                   uint32_t* __restrict__ hmask_in,
                                                   uint32_t* __restrict__ bits, uint32_t words,
                                                   uint32_t* counter) {
    // dynamic shared memory: bits[kRound] (u16) | sp[kTileRows + 1] | rm[kTileRows] | lut[P + 2]
    extern __shared__ __align__(16) uint8_t dsm[];
    uint16_t* codes = (uint16_t*)dsm;
    uint32_t* sp = (uint32_t*)(dsm + 2 * kRound);
    uint32_t* rm = sp + kSpWords;
    uint8_t* lut = (uint8_t*)(rm + kTileRows);
    __shared__ uint32_t item_sh, red;
    if (EVAL) fill_lut(lut, P, sd.in_pred, sd.n_in);
    else fill_lut(lut, P, sd.out_pred, sd.n_out);
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    const uint32_t items = n_chunks + n_tiles;   // heavy chunks first
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t it = item_sh;
        __syncthreads();
        if (it >= items) break;
        if (it < n_chunks) {
            const uint32_t h = ld(chunk_h + it);
            const uint32_t r = ld(hrow + h);
            const uint32_t b = ld(chunk_start + it);
            const uint32_t e = min(b + kHeavyChunk, ld(S.ptr + r + 1));
            if (threadIdx.x == 0) red = 0;
            __syncthreads();
            const uint32_t m = chunk_mask(S.lab, b, e, lut, P, &red);
            if (threadIdx.x == 0 && m) atomicOr(EVAL ? hmask_in + h : mask_out + r, m);
            __syncthreads();
            continue;
        }
        const uint2 tl = tiles[it - n_chunks];
        const uint32_t r0 = tl.x, nr = tl.y;
        for (uint32_t j = threadIdx.x; j <= nr; j += kThreads) sp[j] = ld(S.ptr + r0 + j);
        for (uint32_t j = threadIdx.x; j < nr; j += kThreads) rm[j] = 0;
        __syncthreads();
        tile_masks(S.lab, sp, nr, rm, lut, P, codes);
        __syncthreads();
        if (!EVAL) {
            for (uint32_t j = threadIdx.x; j < nr; j += kThreads) mask_out[r0 + j] = rm[j];
        } else {
            // one warp per 32-vertex word overlapping the tile
            const uint32_t w0 = r0 >> 5, w1 = (r0 + nr - 1) >> 5;
            for (uint32_t wd = w0 + w; wd <= w1; wd += kScanWarps) {
                const uint32_t v = wd * 32 + lane;
                const bool in = v >= r0 && v < r0 + nr;
                const uint32_t mi = in ? rm[v - r0] : 0u;
                const uint32_t mo = in ? mask_out[v] : 0u;
                for (uint32_t u = 0; u < sd.n_bvars; ++u) {
                    uint32_t b = __ballot_sync(0xffffffffu, in && eval_bits(sd, mo, mi, u));
                    if (lane == 0 && b) atomicOr(bits + (uint64_t)u * words + wd, b);
                }
            }
        }
        __syncthreads();
    }
}

// Pass 3: vertices with a heavy column.
__global__ void k_scan_fixup(const uint32_t* __restrict__ hrow_in, uint32_t n_in_heavy,
                             ScanDev sd, const uint32_t* __restrict__ mask_out,
                             const uint32_t* __restrict__ hmask_in, uint32_t* __restrict__ bits,
                             uint32_t words) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < n_in_heavy;
         h += gridDim.x * blockDim.x) {
        uint32_t v = hrow_in[h];
        uint32_t mo = mask_out[v], mi = hmask_in[h];
        for (uint32_t u = 0; u < sd.n_bvars; ++u)
            if (eval_bits(sd, mo, mi, u)) atomicOr(bits + (uint64_t)u * words + (v >> 5), 1u << (v & 31));
    }
}

size_t scan_work_bytes(const gs_graph* g) {
    return sizeof(uint32_t) * ((uint64_t)g->N + 1) + sizeof(uint32_t) * (g->in.n_heavy + 1) + 512;
}

gs_status run_scan(const gs_graph* g, const ScanSpec& spec, uint32_t* bits, void* work,
                   cudaStream_t st) {
    ScanDev sd{};
    sd.n_bvars = spec.n_bvars;
    sd.n_out = spec.n_out;
    sd.n_in = spec.n_in;
    for (int i = 0; i < spec.n_out; ++i) sd.out_pred[i] = spec.out_pred[i];
    for (int i = 0; i < spec.n_in; ++i) sd.in_pred[i] = spec.in_pred[i];
    for (int u = 0; u < spec.n_bvars; ++u) {
        sd.need_out[u] = spec.need_out[u];
        sd.need_in[u] = spec.need_in[u];
    }
    uint32_t* mask_out = (uint32_t*)work;
    uint32_t* hmask_in = mask_out + ((uint64_t)g->N + 1);
    uint32_t* counters = hmask_in + (g->in.n_heavy + 1);    // two work counters
    const uint32_t words = (g->N + 31) / 32;
    const size_t smem = 2 * (size_t)kRound + 4 * (size_t)kSpWords + 4 * (size_t)kTileRows + g->P + 2;
    static int per_sm = 0;
    static size_t smem_set = 0;
    if (smem > smem_set) {
        GS_CUDA(cudaFuncSetAttribute(k_scan<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GS_CUDA(cudaFuncSetAttribute(k_scan<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        smem_set = smem;
        per_sm = 0;
    }
    if (per_sm == 0) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_scan<false>, kThreads, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scan<true>, kThreads, smem);
        per_sm = std::max(1, std::min(a, b));
    }
    const int nb = g->n_blocks;
    const int nbs = g->sm_count * per_sm;   // one wave of resident blocks
    k_scan_zero<<<nb, kThreads, 0, st>>>(g->out.hrow, g->out.n_heavy, mask_out, hmask_in,
                                         g->in.n_heavy, bits, (uint64_t)words * spec.n_bvars,
                                         counters);
    k_scan<false><<<nbs, kThreads, smem, st>>>(dview(g->out), g->P, g->out.tiles, g->out.n_tiles,
                                              g->out.chunk_h, g->out.chunk_start, g->out.hrow,
                                              g->out.n_chunks, sd, mask_out, hmask_in, bits,
                                              words, counters);
    k_scan<true><<<nbs, kThreads, smem, st>>>(dview(g->in), g->P, g->in.tiles, g->in.n_tiles,
                                             g->in.chunk_h, g->in.chunk_start, g->in.hrow,
                                             g->in.n_chunks, sd, mask_out, hmask_in, bits, words,
                                             counters + 1);
    k_scan_fixup<<<nb, kThreads, 0, st>>>(g->in.hrow, g->in.n_heavy, sd, mask_out, hmask_in, bits,
                                          words);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
