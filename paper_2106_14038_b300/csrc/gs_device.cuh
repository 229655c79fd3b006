// Device helpers shared by the kernels: searches in label-sorted rows,
// block-wide scans, and the three-launch device-wide reduce-then-scan the
// store build uses (the query path folds its count -> offset steps into the
// count kernels instead). No kernel waits on another block.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gs_internal.h"

namespace gs {

__device__ __forceinline__ uint32_t ld(const uint32_t* p) { return __ldg(p); }

// Searches in sorted uint32 ranges. They are latency-bound gathers, so they
// trade a few extra loads for fewer dependent round trips: a range of at
// most kShort entries is read with independent 16-byte loads and counted;
// a longer one is cut by 8 parallel probes per round (9-ary search).
constexpr uint32_t kShort = 32;

// Number of entries of a[lo..hi) (hi - lo <= kShort) below key and equal to key.
__device__ __forceinline__ void count_short(const uint32_t* __restrict__ a, uint32_t lo,
                                            uint32_t hi, uint32_t key, uint32_t& below,
                                            uint32_t& equal) {
    const uint4* v = reinterpret_cast<const uint4*>(a);
    const uint32_t q0 = lo >> 2, q1 = (hi + 3) >> 2;   // at most 9 words
    uint4 x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = (q0 + i < q1) ? __ldg(v + q0 + i) : make_uint4(0, 0, 0, 0);
    below = 0;
    equal = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const uint32_t k = (q0 + i) << 2;
        const uint32_t e[4] = {x[i].x, x[i].y, x[i].z, x[i].w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const bool in = k + t >= lo && k + t < hi;
            below += in && e[t] < key;
            equal += in && e[t] == key;
        }
    }
}

// First position in [lo, hi) (hi - lo <= kShort) of the sorted a whose
// value is >= key, by binary search: a handful of instructions per step,
// for callers bound by instruction issue rather than by load latency.
__device__ __forceinline__ uint32_t lower_bound_short(const uint32_t* __restrict__ a, uint32_t lo,
                                                      uint32_t hi, uint32_t key) {
    uint32_t n = hi - lo;
    while (n > 0) {
        const uint32_t half = n >> 1;
        if (__ldg(a + lo + half) < key) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}

// First position in [lo, hi) of the sorted array a whose value is >= key
// (hi when there is none). kSearchShort: finish the last <= kShort entries
// by binary search instead of counting them.
template <bool kSearchShort = false>
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t lo,
                                                    uint32_t hi, uint32_t key) {
    while (hi - lo > kShort) {
        // probes at lo + k * step, k = 1..8, step = floor(n / 9) >= 3: the
        // last probe stays below hi and every part is at most step + 8 long
        const uint32_t step = (hi - lo) / 9;
        uint32_t c = 0, last_lt = lo, first_ge = hi;
        uint32_t pos[8], val[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            pos[j] = lo + step * (uint32_t)(j + 1);
            val[j] = __ldg(a + pos[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (val[j] < key) { c = j + 1; last_lt = pos[j] + 1; }
        }
        if (c < 8) first_ge = pos[c];
        lo = last_lt;
        hi = first_ge;            // a[first_ge] >= key, so the answer is <= first_ge
        if (lo >= hi) return hi;
    }
    if (kSearchShort) return lower_bound_short(a, lo, hi, key);
    uint32_t below, equal;
    count_short(a, lo, hi, key, below, equal);
    return lo + below;
}

static_assert(kShort == kDirMin, "rows without a label directory are the short ones");

// Entries of predicate p in row r: [lo, lo + len) of S.idx. Rows are sorted
// by (label, idx), so this is Eq. 8's S_p (x) A restricted to one row. A
// long row is looked up in its label directory (one entry per run of equal
// labels, at most P) instead of its whole label array.
__device__ __forceinline__ void label_range(const DStore& S, uint32_t r, uint32_t p, uint32_t& lo,
                                            uint32_t& len) {
    const uint32_t b = ld(S.ptr + r), e = ld(S.ptr + r + 1);
    if (e - b <= kShort) {
        uint32_t below, equal;
        count_short(S.lab, b, e, p, below, equal);
        lo = b + below;
        len = equal;
        return;
    }
    if (S.dir_off) {
        const uint32_t d0 = ld(S.dir_off + r), d1 = ld(S.dir_off + r + 1);
        const uint32_t j = lower_bound_u32(S.dir_lab, d0, d1, p);
        if (j < d1 && ld(S.dir_lab + j) == p) {
            lo = ld(S.dir_pos + j);
            len = (j + 1 < d1 ? ld(S.dir_pos + j + 1) : e) - lo;
        } else {
            lo = b;
            len = 0;
        }
        return;
    }
    const uint32_t l = lower_bound_u32(S.lab, b, e, p);
    const uint32_t h = lower_bound_u32(S.lab, l, e, p + 1);
    lo = l;
    len = h - l;
}

// Does row r hold predicate p (Eq. 4 for one row)?
__device__ __forceinline__ bool has_label(const DStore& S, uint32_t r, uint32_t p) {
    const uint32_t b = ld(S.ptr + r), e = ld(S.ptr + r + 1);
    if (e - b <= kShort) {
        uint32_t below, equal;
        count_short(S.lab, b, e, p, below, equal);
        return equal != 0;
    }
    if (S.dir_off) {
        const uint32_t d0 = ld(S.dir_off + r), d1 = ld(S.dir_off + r + 1);
        const uint32_t j = lower_bound_u32(S.dir_lab, d0, d1, p);
        return j < d1 && ld(S.dir_lab + j) == p;
    }
    const uint32_t l = lower_bound_u32(S.lab, b, e, p);
    return l < e && ld(S.lab + l) == p;
}

// Is x in the sorted idx range [lo, lo + len)? (The candidate tests of the
// level expansion make many of these; they are bound by instruction issue,
// so short windows are searched rather than counted.)
__device__ __forceinline__ bool in_range(const DStore& S, uint32_t lo, uint32_t len, uint32_t x) {
    if (len == 0) return false;
    const uint32_t hi = lo + len;
    const uint32_t k = len <= kShort ? lower_bound_short(S.idx, lo, hi, x)
                                     : lower_bound_u32<true>(S.idx, lo, hi, x);
    return k < hi && ld(S.idx + k) == x;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= (uint32_t)d) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over a block of kThreads threads.
// Returns the thread's exclusive prefix; *total gets the block sum.
__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t v, uint64_t* total) {
    __shared__ uint64_t wsum[kThreads / 32];
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    uint64_t incl = warp_incl_scan_u64(v);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint64_t x = lane < kThreads / 32 ? wsum[lane] : 0;
        x = warp_incl_scan_u64(x);
        if (lane < kThreads / 32) wsum[lane] = x;
    }
    __syncthreads();
    uint64_t base = w ? wsum[w - 1] : 0;
    *total = wsum[kThreads / 32 - 1];
    __syncthreads();
    return base + incl - v;
}

// Exclusive max-scan of one value per thread over a block of kThreads
// threads (0 for thread 0).
__device__ __forceinline__ uint32_t block_excl_max_u32(uint32_t v) {
    __shared__ uint32_t wmax[kThreads / 32];
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (uint32_t)d) incl = max(incl, t);
    }
    if (lane == 31) wmax[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t x = lane < kThreads / 32 ? wmax[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= (uint32_t)d) x = max(x, t);
        }
        if (lane < kThreads / 32) wmax[lane] = x;
    }
    __syncthreads();
    uint32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) ex = 0;
    if (w > 0) ex = max(ex, wmax[w - 1]);
    __syncthreads();
    return ex;
}

__device__ __forceinline__ uint64_t block_sum_u64(uint64_t v) {
    uint64_t t;
    block_excl_scan_u64(v, &t);
    return t;
}

// Contiguous chunk of [0, n) owned by block b of nb blocks.
__device__ __forceinline__ void block_chunk(uint64_t n, uint32_t b, uint32_t nb, uint64_t& beg,
                                            uint64_t& end) {
    uint64_t chunk = (n + nb - 1) / nb;
    beg = (uint64_t)b * chunk;
    end = beg + chunk;
    if (beg > n) beg = n;
    if (end > n) end = n;
}

// Single-block exclusive scan of the per-block sums bsum[0..nb) into boff;
// writes the grand total to *total. Launch with one block of kThreads.
__global__ void k_scan_block_sums(const uint64_t* __restrict__ bsum, uint64_t* __restrict__ boff,
                                  uint32_t nb, uint64_t* total, const uint32_t* status);

// In-place exclusive scan of a[0..n) where n = *n_ptr; block b handles the
// chunk block_chunk(n, b, gridDim.x) and adds boff[b].
__global__ void k_scan_apply_u64(uint64_t* __restrict__ a, const uint64_t* n_ptr,
                                 const uint64_t* __restrict__ boff, const uint32_t* status);

// Per-block sums of a[0..n) for the reduce step.
__global__ void k_block_sums_u64(const uint64_t* __restrict__ a, const uint64_t* n_ptr,
                                 uint64_t* __restrict__ bsum, const uint32_t* status);

}  // namespace gs
