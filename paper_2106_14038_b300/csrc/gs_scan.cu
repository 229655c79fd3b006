// Triple scan: candidate vectors of query variables by grouped predicate
// selection (Sec. 5, Step 1). For a variable u with out-predicates O(u)
// (u is the subject) and in-predicates I(u) (u is the object):
//
//     v_u = AND_{p in O(u)} (A (x) u_p)  AND  AND_{p in I(u)} (A^T (x) u_p)
//
// (Eq. 17 with only outgoing edges, Eq. 21 with both; Eq. 4 and Eq. 5 for
// the single selections). All predicates of the query are tested in one
// pass over the label array of each orientation:
//   1. k_scan streams the CSR labels and the CSC labels (one grid, items of
//      both) and writes, per vertex, the mask of the query's out-predicates
//      its row holds (mask_out) and of its in-predicates its column holds
//      (mask_in);
//   2. k_scan_eval combines the two masks per vertex and writes one bit per
//      variable into the candidate vectors (warp ballot -> one word per 32
//      vertices, so the vectors need no clearing).
// k_scan_zero first clears the mask words that several items OR into; each
// kernel is launched to overlap the tail of the one before it
// (programmatic dependent launch) and waits for it where it must.
//
// Work decomposition. Each orientation is cut at store build into items of
// equal cost along the merge of row ends and labels (merge path), so rows
// of any degree and runs of empty rows cost the same per unit. A warp
// takes items round robin and double-buffers them in shared memory: lanes
// 0..2 move an item's labels, row-start bits and row pointers into its
// buffer with bulk asynchronous copies that complete on an mbarrier, while
// the warp works on the previous item. Warps never wait on one another.
// Per item (row starts come from a bitmap built with the store):
//   A. label phase: lane l takes 33 consecutive labels (an odd stride, so
//      the 32 lanes hit 32 banks), maps each to its one-hot slot bit
//      through a table and stores, per position, the OR since the later of
//      its row's start and its lane's start; a segmented OR-scan over the
//      lanes then gives, per lane, the OR of the row running through the
//      lane's end;
//   B. rows phase: one lane per row combines its last position's value with
//      the previous lane's running total and writes the row's mask; rows in
//      the 32-bit words of the item's first and last rows (which a
//      neighbouring item may also write) are ORed into those zeroed words.
// Bytes moved: per orientation 4(N+1) row pointers + 4M labels + M/8
// row-start bits, a 2N mask (16-bit slots) written and read once, and N/8
// per vector. The streamed inputs are read with an evict-first L2 policy,
// so the masks tend to stay in L2 until k_scan_eval reads them.
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "gs_device.cuh"

namespace gs {

// The predicates k_scan tests: slot i of a direction is predicate
// out_pred[i] (rows) / in_pred[i] (columns).
struct ScanPreds {
    uint32_t out_pred[kMaxSlotsWide];
    uint32_t in_pred[kMaxSlotsWide];
    uint32_t n_out, n_in;
    long long stall_cycles;   // limit of a warp's wait for its next item's copies
};

constexpr uint32_t kItemLabs = 32 * kScanLabPer;         // label slots of one item (1056)
constexpr uint32_t kGap = 36;                            // zeroed words after the labels
constexpr uint32_t kHeadCopy = 48;                       // room for an item's row-start words
constexpr uint32_t kBufWords = kItemLabs + 32 + kGap + kHeadCopy;   // labels | gap | starts | ptr | masks
constexpr uint32_t kNumBuf = 2;                          // items in shared memory per warp
constexpr uint32_t kScanWarps = 20;                      // most warps per CTA, each on its own items
// Per warp: kNumBuf item buffers, then the run ORs of one item (one mask
// per label position) and the 32 lane totals.
template <typename MaskT>
__host__ __device__ constexpr uint32_t pm_words() { return kItemLabs * (uint32_t)sizeof(MaskT) / 4 + 32; }
template <typename MaskT>
__host__ __device__ constexpr uint32_t warp_words() { return kNumBuf * kBufWords + pm_words<MaskT>(); }
constexpr long long kStallCycles = 4000000000LL;         // about 2 s at 2 GHz
static_assert(kBufWords % 4 == 0 && pm_words<uint16_t>() % 4 == 0 &&
                  pm_words<uint32_t>() % 4 == 0 && warp_words<uint16_t>() % 4 == 0 &&
                  warp_words<uint32_t>() % 4 == 0,
              "bulk-copy destinations must stay 16-byte aligned");

// ---- bulk copies and mbarriers (inline PTX) ----

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with parity `parity` of bar, for at most `limit`
// cycles; a limit <= 0 gives up at once (failure tests).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit) {
    if (limit <= 0) return false;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// L2 policy for data read once: its lines are the first to be evicted.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Global -> shared bulk copy under L2 policy pol; both addresses 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Item d = (r0, k0, r1, k1): rows r0..r1 (r1 only in part), labels
// [k0, k1). Its buffer holds three regions, each copied from a 16-byte
// boundary of global memory: labels from k0 & ~3 (nl words); after a gap
// of at least 33 words that the warp zeroes, the row-start words covering
// entries k0 .. k1 + 64 (nh words); row pointers from r0 & ~3 through row
// r1 + 1 (np words).
struct ItemLayout {
    uint32_t nl, nh, np;
    uint32_t ho, po;   // word offsets of the row starts and the row pointers
};

__device__ __forceinline__ uint32_t head_word0(uint32_t k0) { return (k0 >> 5) & ~3u; }

__device__ __forceinline__ ItemLayout item_layout(uint4 d) {
    ItemLayout L;
    L.nl = ((d.w + 3u) & ~3u) - (d.y & ~3u);
    L.nh = ((((d.w + 64u) >> 5) + 1u + 3u) & ~3u) - head_word0(d.y);
    L.np = ((d.z + 2u + 3u) & ~3u) - (d.x & ~3u);
    L.ho = (L.nl + 33u + 3u) & ~3u;
    L.po = L.ho + L.nh;
    return L;
}

// Lanes 0..2 of a warp put item d into buf behind bar, one region each,
// with one copy instruction (evict-first: every word is read once); lane 0
// first announces the bytes. Called by the whole warp.
__device__ __forceinline__ void issue_item(uint32_t lane, uint32_t* buf, uint64_t* bar, uint4 d,
                                           const DStore& S, const uint32_t* heads) {
    const ItemLayout L = item_layout(d);
    if (lane == 0) mbar_expect_tx(bar, 4u * (L.nl + L.nh + L.np));
    __syncwarp();
    const uint32_t* src = lane == 0 ? S.lab + (d.y & ~3u)
                        : lane == 1 ? heads + head_word0(d.y)
                                    : S.ptr + (d.x & ~3u);
    const uint32_t off = lane == 0 ? 0u : lane == 1 ? L.ho : L.po;
    const uint32_t n = lane == 0 ? L.nl : lane == 1 ? L.nh : L.np;
    if (lane < 3 && n) bulk_g2s(buf + off, src, 4u * n, bar, evict_first_policy());
}

// label -> one-hot slot bit of this direction's query predicates
template <typename LutT>
__device__ __forceinline__ uint32_t lut_bit(const LutT* lut, uint32_t l) {
    if constexpr (sizeof(LutT) == 1)
        return (uint32_t)((1ull << lut[l]) >> 1);   // the byte table holds slot + 1 (0: none)
    else
        return lut[l];                              // one-hot already
}

__device__ __forceinline__ uint32_t eval_bit(const EvalVec& v, uint32_t mo, uint32_t mi) {
    return ((mo & v.need_out) == v.need_out) && ((mi & v.need_in) == v.need_in);
}

// Dynamic shared memory: per warp kNumBuf buffers | run ORs | lane totals;
// then the two luts.
template <typename LutT, typename MaskT>
size_t scan_smem_bytes(uint32_t P, uint32_t warps) {
    return 4ull * warps * warp_words<MaskT>() + 2 * sizeof(LutT) * ((size_t)P + 2);
}

// Warps per CTA that fit beside two luts of P + 2 entries of lut_bytes each.
template <typename MaskT>
static uint32_t scan_warps_fit(uint32_t P, size_t lut_bytes) {
    const size_t avail = 227u * 1024u - 1536u;   // less the static shared memory
    const size_t lut = 2 * lut_bytes * ((size_t)P + 2);
    if (lut >= avail) return 0;
    return (uint32_t)std::min<size_t>(kScanWarps, (avail - lut) / (4ull * warp_words<MaskT>()));
}

// One orientation of the matrix as the scan sees it.
struct ScanSide {
    DStore S;
    const uint32_t* heads;
    const uint2* items;
    uint32_t n_items;
    void* mask;   // per vertex (MaskT): the query predicates of this direction its row holds
};

// Both orientations in one grid: items 0 .. out.n_items - 1 are the CSR's,
// the rest the CSC's. Every warp works alone on its own items (round robin
// over all warps of the grid) with its own buffers; it syncs only with
// itself. Launched dependent on k_scan_zero: the first copies are issued
// before waiting for it, the masks are written after.
template <typename LutT, typename MaskT>
__global__ void __launch_bounds__(kScanWarps * 32, 1) k_scan(ScanSide out, ScanSide in, uint32_t N,
                                                             uint32_t P, ScanPreds sd,
                                                             uint32_t* status) {
    extern __shared__ __align__(128) uint32_t dsm[];
    constexpr uint32_t kWarpWords = warp_words<MaskT>();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t n_warps = blockDim.x >> 5;
    uint32_t* bufs = dsm + warp * kWarpWords;
    MaskT* pm = (MaskT*)(bufs + kNumBuf * kBufWords);   // pm[p]: run OR at position p
    uint32_t* cont = bufs + kNumBuf * kBufWords + kItemLabs * (uint32_t)sizeof(MaskT) / 4;   // cont[l]: lane l's run total
    LutT* luts = (LutT*)(dsm + n_warps * kWarpWords);   // out-predicates | in-predicates
    __shared__ __align__(8) uint64_t full[kScanWarps][kNumBuf];
    __shared__ uint4 desc[kScanWarps][kNumBuf];
    __shared__ uint32_t side_of[kScanWarps][kNumBuf];
    const uint32_t n0 = out.n_items, n_items = out.n_items + in.n_items;

    for (uint32_t i = threadIdx.x; i < 2 * (P + 2); i += blockDim.x) luts[i] = 0;
    if (lane == 0) {
        for (uint32_t b = 0; b < kNumBuf; ++b) mbar_init(&full[warp][b], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x < sd.n_out)
        luts[sd.out_pred[threadIdx.x]] =
            sizeof(LutT) >= 2 ? (LutT)(1u << threadIdx.x) : (LutT)(threadIdx.x + 1);
    if (threadIdx.x < sd.n_in)
        luts[P + 2 + sd.in_pred[threadIdx.x]] =
            sizeof(LutT) >= 2 ? (LutT)(1u << threadIdx.x) : (LutT)(threadIdx.x + 1);
    __syncthreads();

    const uint32_t gw = blockIdx.x * n_warps + warp;
    const uint32_t GW = gridDim.x * n_warps;
    for (uint32_t b = 0; b < kNumBuf; ++b) {
        const uint32_t c = gw + b * GW;
        if (c < n_items) {
            const bool cols = c >= n0;
            const ScanSide& sd_ = cols ? in : out;
            const uint32_t cl = cols ? c - n0 : c;
            const uint2 a = sd_.items[cl], z = sd_.items[cl + 1];
            const uint4 d = make_uint4(a.x, a.y, z.x, z.y);
            if (lane == 0) { desc[warp][b] = d; side_of[warp][b] = cols; }
            issue_item(lane, bufs + b * kBufWords, &full[warp][b], d, sd_.S, sd_.heads);
        }
    }
    __syncwarp();
    // the slots zeroed by k_scan_zero are written below
    asm volatile("griddepcontrol.wait;" ::: "memory");

    bool stalled = false;
    uint32_t stall_i = 0;
    for (uint32_t i = 0;; ++i) {
        const uint32_t c = gw + i * GW;
        if (c >= n_items) break;
        const uint32_t b = i % kNumBuf;
        const uint32_t cn = c + kNumBuf * GW;   // the item this buffer takes next
        const bool ncols = cn >= n0;
        uint2 nx = make_uint2(0, 0);   // lane 0: items[cn], lane 1: items[cn + 1] of its side
        if (lane < 2 && cn < n_items)
            nx = (ncols ? in.items : out.items)[(ncols ? cn - n0 : cn) + lane];   // in flight meanwhile
        // every lane acquires the copies itself; all lanes agree on a stall
        const bool landed = mbar_wait_bounded(&full[warp][b], (i / kNumBuf) & 1u, sd.stall_cycles);
        if (!__all_sync(0xffffffffu, landed)) { stalled = true; stall_i = i; break; }

        const uint4 d = desc[warp][b];
        const uint32_t cols = side_of[warp][b];
        const LutT* lut = luts + (cols ? P + 2 : 0u);
        MaskT* mask = (MaskT*)(cols ? in.mask : out.mask);
        const uint32_t r0 = d.x, k0 = d.y, r1 = d.z, k1 = d.w;
        const ItemLayout L = item_layout(d);
        const uint32_t* buf = bufs + b * kBufWords;
        uint32_t* lab = bufs + b * kBufWords + (k0 & 3u);       // lab[p]: label k0 + p
        const uint32_t* hs = buf + L.ho;                       // row-start words from head_word0(k0)
        const uint32_t* pp = buf + L.po + (r0 & 3u);           // pp[j]: ptr[r0 + j]
        const uint32_t nk = k1 - k0;
        const uint32_t nt = r1 - r0 + (r1 < N ? 1u : 0u);     // rows touched
        // label 0 (no predicate) in the 33 positions after the item's labels
        lab[nk + lane] = 0;
        if (lane == 0) lab[nk + 32] = 0;

        // A. label phase: pm[p] = OR of the one-hot bits from the later of
        // (the head of p's row, the start of p's lane) through p
        const uint32_t base = lane * kScanLabPer;
        uint32_t acc = 0;
        bool has_head = false;
        if (base < nk) {   // positions past nk read label 0
            // row starts of entries k0 + base .. + 32; a start past k1 only
            // touches positions no row reads back
            const uint32_t gp = k0 + base;
            const uint32_t hwi = (gp >> 5) - head_word0(k0);
            const uint64_t h64 = ((((uint64_t)hs[hwi + 1]) << 32) | hs[hwi]) >> (gp & 31);
            // all loads first: the stores into pm below may not be
            // reordered before loads of the same shared array
            uint32_t v[kScanLabPer];
#pragma unroll
            for (uint32_t q = 0; q < kScanLabPer; ++q) v[q] = lab[base + q];
#pragma unroll
            for (uint32_t q = 0; q < kScanLabPer; ++q) v[q] = lut_bit<LutT>(lut, v[q]);
#pragma unroll
            for (uint32_t q = 0; q < kScanLabPer; ++q) {
                const uint32_t keep = (uint32_t)((h64 >> q) & 1ull) - 1u;   // 0 at a head
                acc = (acc & keep) | v[q];
                pm[base + q] = (MaskT)acc;
            }
            has_head = (h64 & ((1ull << kScanLabPer) - 1)) != 0;
        }
        // segmented inclusive OR-scan of the lanes' last runs; a lane holding
        // a head starts a segment: cont[l] = OR of the labels from the
        // head of the row at the end of lane l through that end
        {
            bool f = has_head;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, acc, o);
                const bool g = __shfl_up_sync(0xffffffffu, f, o);
                if (lane >= o && !f) acc |= v;
                if (lane >= o) f = f || g;
            }
            cont[lane] = acc;
        }
        __syncwarp();

        // B. rows phase: a row's labels [lo, hi) in the item end in lane lb;
        // the part in lane lb is pm[hi - 1 - k0], the part before it the run
        // total of lane lb - 1
        for (uint32_t j = lane; j < nt; j += 32) {
            const uint32_t r = r0 + j;
            const uint32_t s = pp[j], e = pp[j + 1];
            const uint32_t lo = max(s, k0), hi = min(e, k1);
            uint32_t m = 0;
            if (lo < hi) {
                const uint32_t la = (lo - k0) / kScanLabPer, lb = (hi - 1 - k0) / kScanLabPer;
                m = pm[hi - 1 - k0] | (lb > la ? cont[lb - 1] : 0u);
            }
            // rows sharing a 32-bit word with r0 or r1 (zeroed by
            // k_scan_zero) may be written by two items: ORed in whole words;
            // every other row lies in this item alone
            if constexpr (sizeof(MaskT) == 2) {
                if ((r >> 1) == (r0 >> 1) || (r >> 1) == (r1 >> 1)) {
                    if (m) atomicOr(reinterpret_cast<uint32_t*>(mask) + (r >> 1), m << (16 * (r & 1u)));
                } else {
                    mask[r] = (MaskT)m;
                }
            } else {
                if (r == r0 || r == r1) {
                    if (m) atomicOr(reinterpret_cast<uint32_t*>(mask) + r, m);
                } else {
                    mask[r] = (MaskT)m;
                }
            }
        }
        __syncwarp();   // buffer b and pm are free again
        if (cn < n_items) {
            const uint4 d2 = make_uint4(__shfl_sync(0xffffffffu, nx.x, 0), __shfl_sync(0xffffffffu, nx.y, 0),
                                        __shfl_sync(0xffffffffu, nx.x, 1), __shfl_sync(0xffffffffu, nx.y, 1));
            if (lane == 0) { desc[warp][b] = d2; side_of[warp][b] = ncols; }
            // the gap was zeroed through the generic proxy; the copies into
            // this buffer go through the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const ScanSide& ns = ncols ? in : out;
            issue_item(lane, bufs + b * kBufWords, &full[warp][b], d2, ns.S, ns.heads);
        }
        __syncwarp();
    }

    // the candidate-bit kernel may start launching (it waits for this grid)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (stalled && lane == 0) {
        // report, then let the copies still in flight (items stall_i ..
        // stall_i + kNumBuf - 1 of this warp) land before the warp exits;
        // this wait keeps the long limit whatever the first one was
        atomicOr(status, kStStall);
        for (uint32_t k = stall_i; k < stall_i + kNumBuf; ++k)
            if (gw + k * GW < n_items)
                mbar_wait_bounded(&full[warp][k % kNumBuf], (k / kNumBuf) & 1u, kStallCycles);
    }
}

// The 32-bit mask words holding an item's first row (so also the last row
// of the item before) start at zero: the items OR their rows into them.
// shift: 1 for 16-bit masks (two rows per word), 0 for 32-bit masks.
__global__ void k_scan_zero(const uint2* __restrict__ items_out, uint32_t n_out,
                            const uint2* __restrict__ items_in, uint32_t n_in,
                            uint32_t* __restrict__ mask_out, uint32_t* __restrict__ mask_in,
                            uint32_t shift) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // k_scan may start its copies
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t c = t; c <= n_out; c += stride) mask_out[items_out[c].x >> shift] = 0;
    for (uint32_t c = t; c <= n_in; c += stride) mask_in[items_in[c].x >> shift] = 0;
}

// Candidate bits: vertex v is in vector j when its row holds every
// out-predicate and its column every in-predicate the vector needs
// (Eq. 21). The test is done bit-sliced: a warp takes 1,024 vertices, 32
// consecutive ones per lane; the lane transposes its 32 masks (a 32 x 32
// bit matrix: one mask per row) into one word per predicate slot whose bit
// j is vertex j's slot bit, and a vector's word is then the AND of the
// slot words it needs. So a vector costs one AND per needed slot per 32
// vertices, and the 32 lanes of a warp write 128 consecutive bytes of it.
// 16-bit masks are packed two to a word (out low, in high) and transposed
// together; 32-bit masks are transposed one direction at a time.
constexpr uint32_t kEvalThreads = 128;

// In-place transpose of a 32 x 32 bit matrix (a[j] bit s -> a[s] bit j):
// exchange the off-diagonal halves of every 2w x 2w block, for w = 16, 8,
// 4, 2, 1 (each step swaps bits (j + w, s) and (j, s + w) of the blocks'
// rows through an XOR difference).
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t m = w == 16 ? 0x0000ffffu
                         : w == 8  ? 0x00ff00ffu
                         : w == 4  ? 0x0f0f0f0fu
                         : w == 2  ? 0x33333333u
                                   : 0x55555555u;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j & w) continue;
            const uint32_t t = ((a[j] >> w) ^ a[j + w]) & m;
            a[j + w] ^= t;
            a[j] ^= t << w;
        }
    }
}

// The 32 masks of vertices base..base+31 into a[] (16-bit masks: out in the
// low, in in the high half of each word; 32-bit masks: the one array m).
// Lanes past N load nothing; a lane that runs past N reads at most 31 slots
// past it (the mask arrays hold N + 256).
__device__ __forceinline__ void load_masks16(const uint16_t* __restrict__ mo,
                                             const uint16_t* __restrict__ mi, uint32_t base,
                                             uint32_t N, uint32_t (&a)[32]) {
    if (base >= N) {
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = 0;
        return;
    }
    const uint4* po = reinterpret_cast<const uint4*>(mo + base);
    const uint4* pi = reinterpret_cast<const uint4*>(mi + base);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const uint4 x = __ldcs(po + h), y = __ldcs(pi + h);
        const uint32_t xo[4] = {x.x, x.y, x.z, x.w}, yi[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // word k: vertices 8h + 2k (low half) and 8h + 2k + 1
            a[8 * h + 2 * k] = (xo[k] & 0xffffu) | (yi[k] << 16);
            a[8 * h + 2 * k + 1] = (xo[k] >> 16) | (yi[k] & 0xffff0000u);
        }
    }
}

__device__ __forceinline__ void load_masks32(const uint32_t* __restrict__ m, uint32_t base,
                                             uint32_t N, uint32_t (&a)[32]) {
    if (base >= N) {
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = 0;
        return;
    }
    const uint4* p = reinterpret_cast<const uint4*>(m + base);
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const uint4 x = __ldcs(p + h);
        a[4 * h] = x.x;
        a[4 * h + 1] = x.y;
        a[4 * h + 2] = x.z;
        a[4 * h + 3] = x.w;
    }
}

template <typename MaskT>
__global__ void __launch_bounds__(kEvalThreads) k_scan_eval(const MaskT* __restrict__ mask_out,
                                                            const MaskT* __restrict__ mask_in,
                                                            uint32_t N, EvalArgs ea, uint32_t words) {
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the masks of k_scan
    constexpr bool kNarrow = sizeof(MaskT) == 2;
    constexpr uint32_t kRows = kNarrow ? 32 : 64;        // slot words per lane
    constexpr uint32_t kInRow = kNarrow ? 16 : 32;       // first in-slot word
    // slot word s of lane l at sw[s][l]: each lane reads back only its own
    // column (a dynamically indexed register file), without bank conflicts
    __shared__ uint32_t sw_all[kEvalThreads / 32][kRows][32];
    uint32_t (*sw)[32] = sw_all[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); (uint64_t)c * 1024 < N;
         c += warps) {
        const uint32_t base = c * 1024 + lane * 32;
        const uint32_t valid = base >= N ? 0u : N - base >= 32 ? 0xffffffffu : (1u << (N - base)) - 1u;
        uint32_t a[32];
        if constexpr (kNarrow) {
            load_masks16(mask_out, mask_in, base, N, a);
            transpose32(a);
#pragma unroll
            for (int s = 0; s < 32; ++s) sw[s][lane] = a[s];
        } else {
            load_masks32(mask_out, base, N, a);
            transpose32(a);
#pragma unroll
            for (int s = 0; s < 32; ++s) sw[s][lane] = a[s];
            load_masks32(mask_in, base, N, a);
            transpose32(a);
#pragma unroll
            for (int s = 0; s < 32; ++s) sw[32 + s][lane] = a[s];
        }
        const uint32_t wi = c * 32 + lane;
        for (uint32_t j = 0; j < ea.n; ++j) {
            const EvalVec e = ea.list ? ea.list[j] : ea.inl[j];
            uint32_t acc = valid;
            for (uint32_t m = e.need_out; m; m &= m - 1) acc &= sw[__ffs(m) - 1][lane];
            for (uint32_t m = e.need_in; m; m &= m - 1) acc &= sw[kInRow + __ffs(m) - 1][lane];
            if (wi < words) e.dst[wi] = acc;
        }
    }
}

// Blocks of k_scan_eval that fit on one SM at once (asked once per device
// and mask width): the grid is one wave of them, so no block starts late.
// Per-device launch facts below share one mutex.
constexpr int kAttrDevices = 64;
static std::mutex g_attr_mu;
static int g_eval_fit[kAttrDevices][2];

template <typename MaskT>
static int eval_blocks_per_sm(int dev) {
    if (dev < 0 || dev >= kAttrDevices) return 1;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    int& fit = g_eval_fit[dev][sizeof(MaskT) == 2 ? 0 : 1];
    if (fit <= 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_scan_eval<MaskT>, kEvalThreads, 0) !=
                cudaSuccess || n <= 0)
            n = 1;
        fit = n;
    }
    return fit;
}

// Workspace: mask_out | mask_in (N + 256 slots of 16 or 32 bits each,
// 16-byte aligned).
static uint64_t mask_slots(uint32_t N) { return ((uint64_t)N + 256 + 7) & ~7ull; }

size_t scan_work_bytes(const gs_graph* g, bool wide) {
    return (wide ? 8ull : 4ull) * mask_slots(g->N) + 512;
}

// Cycles a warp of k_scan waits for the copies of its next item before it
// reports kStStall: about 2 s, or GS_SCAN_STALL_CYCLES when set (0: give up
// at once), which failure tests use to make the wait run out; the warp then
// still waits, with the long limit, for the copies it has in flight.
long long scan_stall_cycles() {
    if (const char* e = getenv("GS_SCAN_STALL_CYCLES")) {
        char* end = nullptr;
        const long long v = strtoll(e, &end, 10);
        if (end != e && v >= 0) return v;
    }
    return kStallCycles;
}

// Dynamic shared memory already allowed for each k_scan variant on each
// device (function attributes are per device); guarded by g_attr_mu.
static size_t g_smem_set[kAttrDevices][4];

template <typename LutT, typename MaskT>
static gs_status allow_smem(int dev, size_t smem) {
    if (dev < 0 || dev >= kAttrDevices) {
        set_error("triple scan: device %d outside 0..%d", dev, kAttrDevices - 1);
        return GS_EINVAL;
    }
    const int variant = (sizeof(LutT) == 1 ? 0 : 1) + (sizeof(MaskT) == 2 ? 0 : 2);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t& set = g_smem_set[dev][variant];
    if (smem > set) {
        GS_CUDA(cudaFuncSetAttribute(k_scan<LutT, MaskT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        set = smem;
    }
    return GS_OK;
}

template <typename LutT, typename MaskT>
static gs_status launch_scan(const gs_graph* g, const Store& so, const Store& si, const ScanPreds& sd,
                             void* mask_out, void* mask_in, uint32_t* status, uint32_t warps,
                             cudaStream_t st) {
    const size_t smem = scan_smem_bytes<LutT, MaskT>(g->P, warps);
    gs_status arc = allow_smem<LutT, MaskT>(g->device, smem);
    if (arc != GS_OK) return arc;
    // one CTA per SM (the shared memory admits no second one)
    const uint32_t n_items = so.n_items + si.n_items;
    const uint32_t grid = std::max(1u, std::min((uint32_t)g->sm_count, (n_items + warps - 1) / warps));
    const ScanSide out{dview(so), so.heads, so.items, so.n_items, mask_out};
    const ScanSide in{dview(si), si.heads, si.items, si.n_items, mask_in};
    GS_CUDA(launch_chained(k_scan<LutT, MaskT>, dim3(grid), dim3(warps * 32), smem, st, out, in,
                           g->N, g->P, sd, status));
    return GS_OK;
}

template <typename MaskT>
static gs_status scan_masks_as(const gs_graph* g, const Store& so, const Store& si,
                               const ScanPreds& sd, void* work, uint32_t* status, cudaStream_t st) {
    MaskT* mask_out = (MaskT*)work;
    MaskT* mask_in = mask_out + mask_slots(g->N);
    k_scan_zero<<<g->n_blocks, kThreads, 0, st>>>(so.items, so.n_items, si.items, si.n_items,
                                                  reinterpret_cast<uint32_t*>(mask_out),
                                                  reinterpret_cast<uint32_t*>(mask_in),
                                                  sizeof(MaskT) == 2 ? 1u : 0u);
    // the one-hot table unless it costs more than a few warps; else the
    // byte table (slot + 1)
    using Wide = typename std::conditional<sizeof(MaskT) == 2, uint16_t, uint32_t>::type;
    const uint32_t ww = scan_warps_fit<MaskT>(g->P, sizeof(Wide));
    const uint32_t w8 = scan_warps_fit<MaskT>(g->P, sizeof(uint8_t));
    if (ww >= 12 || ww >= w8)
        return launch_scan<Wide, MaskT>(g, so, si, sd, mask_out, mask_in, status, ww, st);
    return launch_scan<uint8_t, MaskT>(g, so, si, sd, mask_out, mask_in, status, w8, st);
}

gs_status scan_masks(const gs_graph* g, const uint32_t* out_pred, uint32_t n_out,
                     const uint32_t* in_pred, uint32_t n_in, void* work, uint32_t* status,
                     cudaStream_t st, const Store* so, const Store* si) {
    if (!so) so = &g->out;
    if (!si) si = &g->in;
    if (!status) { set_error("internal: the triple scan needs a status word"); return GS_EINVAL; }
    if (n_out > (uint32_t)kMaxSlotsWide || n_in > (uint32_t)kMaxSlotsWide) {
        set_error("internal: more than %d predicates per direction in one scan", kMaxSlotsWide);
        return GS_EINVAL;
    }
    ScanPreds sd{};
    sd.n_out = n_out;
    sd.n_in = n_in;
    for (uint32_t i = 0; i < n_out; ++i) sd.out_pred[i] = out_pred[i];
    for (uint32_t i = 0; i < n_in; ++i) sd.in_pred[i] = in_pred[i];
    sd.stall_cycles = scan_stall_cycles();
    const bool wide = n_out > (uint32_t)kMaxSlots || n_in > (uint32_t)kMaxSlots;
    return wide ? scan_masks_as<uint32_t>(g, *so, *si, sd, work, status, st)
                : scan_masks_as<uint16_t>(g, *so, *si, sd, work, status, st);
}

gs_status scan_eval(const gs_graph* g, const void* work, bool wide, const EvalArgs& ea,
                    cudaStream_t st) {
    const uint32_t words = (g->N + 31) / 32;
    const uint32_t chunks = (uint32_t)(((uint64_t)g->N + 1023) / 1024);
    const uint32_t want = std::max(1u, (chunks + kEvalThreads / 32 - 1) / (kEvalThreads / 32));
    const int fit = wide ? eval_blocks_per_sm<uint32_t>(g->device) : eval_blocks_per_sm<uint16_t>(g->device);
    const uint32_t eb = std::min<uint32_t>(want, (uint32_t)g->sm_count * (uint32_t)fit);
    if (wide) {
        const uint32_t* mo = (const uint32_t*)work;
        GS_CUDA(launch_chained(k_scan_eval<uint32_t>, dim3(eb), dim3(kEvalThreads), 0, st,
                               mo, mo + mask_slots(g->N), g->N, ea, words));
    } else {
        const uint16_t* mo = (const uint16_t*)work;
        GS_CUDA(launch_chained(k_scan_eval<uint16_t>, dim3(eb), dim3(kEvalThreads), 0, st,
                               mo, mo + mask_slots(g->N), g->N, ea, words));
    }
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status run_scan(const gs_graph* g, const ScanSpec& spec, uint32_t* bits, void* work,
                   cudaStream_t st, uint32_t* status, const Store* so, const Store* si) {
    gs_status rc = scan_masks(g, spec.out_pred, (uint32_t)spec.n_out, spec.in_pred,
                              (uint32_t)spec.n_in, work, status, st, so, si);
    if (rc != GS_OK) return rc;
    EvalArgs ea{};
    ea.n = (uint32_t)spec.n_bvars;
    const uint64_t words = (g->N + 31) / 32;
    for (int u = 0; u < spec.n_bvars; ++u)
        ea.inl[u] = EvalVec{spec.need_out[u], spec.need_in[u], bits + (uint64_t)spec.blevel[u] * words};
    return scan_eval(g, work, false, ea, st);
}

}  // namespace gs
