// Device helpers shared by the kernels: searches in label-sorted rows,
// block-wide scans and the device-wide reduce-then-scan used for every
// count -> offset step (no kernel waits on another block).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gs_internal.h"

namespace gs {

__device__ __forceinline__ uint32_t ld(const uint32_t* p) { return __ldg(p); }

// First position in [lo, hi) of the sorted array a whose value is >= key.
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ a, uint32_t lo,
                                                    uint32_t hi, uint32_t key) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (ld(a + mid) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Entries of predicate p in row r: [lo, lo + len) of S.idx. Rows are sorted
// by (label, idx), so this is Eq. 8's S_p (x) A restricted to one row.
__device__ __forceinline__ void label_range(const DStore& S, uint32_t r, uint32_t p, uint32_t& lo,
                                            uint32_t& len) {
    uint32_t b = ld(S.ptr + r), e = ld(S.ptr + r + 1);
    if (b == e || ld(S.lab + b) > p || ld(S.lab + e - 1) < p) { lo = b; len = 0; return; }
    uint32_t l = lower_bound_u32(S.lab, b, e, p);
    uint32_t h = lower_bound_u32(S.lab, l, e, p + 1);
    lo = l; len = h - l;
}

// Does row r hold predicate p (Eq. 4 for one row)?
__device__ __forceinline__ bool has_label(const DStore& S, uint32_t r, uint32_t p) {
    uint32_t b = ld(S.ptr + r), e = ld(S.ptr + r + 1);
    if (b == e || ld(S.lab + b) > p || ld(S.lab + e - 1) < p) return false;
    uint32_t l = lower_bound_u32(S.lab, b, e, p);
    return l < e && ld(S.lab + l) == p;
}

// Is x in the sorted idx range [lo, lo + len)?
__device__ __forceinline__ bool in_range(const DStore& S, uint32_t lo, uint32_t len, uint32_t x) {
    if (len == 0) return false;
    uint32_t hi = lo + len;
    if (ld(S.idx + lo) > x || ld(S.idx + hi - 1) < x) return false;
    uint32_t k = lower_bound_u32(S.idx, lo, hi, x);
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
