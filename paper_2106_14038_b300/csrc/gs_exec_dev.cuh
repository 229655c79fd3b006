// Device helpers of the executor shared by the grid path (gs_exec.cu)
// and the single-block path (gs_small.cu): workspace layout, the binding
// tree walk, the candidate tests and the level append.
#pragma once

#include "gs_device.cuh"
#include "gs_exec.h"

namespace gs {

__host__ __device__ __forceinline__ uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

__device__ __forceinline__ uint64_t level_off(const Ctl* c, int l) {
    uint64_t o = kCtlBytes;
    for (int j = 0; j < l; ++j) o += align256(8ull * c->n[j]);
    return o;
}

// scratch for producing level l from np parent nodes with nbm binder slots
__host__ __device__ __forceinline__ uint64_t scratch_bytes(uint64_t np, uint32_t nbm) {
    return align256(8ull * np) + align256(8ull * np * nbm) + align256(np);
}

struct Scratch {
    uint64_t* roff;
    uint2* rng;
    uint8_t* sel;
    uint64_t base;
};

__device__ __forceinline__ Scratch scratch_at(const ExecDev& E, uint64_t np, uint32_t nbm) {
    Scratch s;
    uint64_t sb = scratch_bytes(np, nbm);
    s.base = E.arena_bytes > sb ? E.arena_bytes - sb : 0;
    s.roff = (uint64_t*)(E.arena + s.base);
    s.rng = (uint2*)(E.arena + s.base + align256(8ull * np));
    s.sel = (uint8_t*)(E.arena + s.base + align256(8ull * np) + align256(8ull * np * nbm));
    return s;
}

__device__ __forceinline__ bool overflowed(const Ctl* c) {
    return (*(volatile const uint32_t*)&c->status) & kStOverflow;
}

// Level base pointers in shared memory (computed once per block).
__device__ __forceinline__ void load_levels(const ExecDev& E, int upto, const uint2** lv) {
    if (threadIdx.x == 0) {
        uint64_t o = kCtlBytes;
        for (int j = 0; j <= upto && j < kMaxLevels; ++j) {
            lv[j] = (const uint2*)(E.arena + o);
            o += align256(8ull * E.ctl->n[j]);
        }
    }
    __syncthreads();
}

// Bindings of levels 0..from of the node `idx` at level `from`.
__device__ __forceinline__ void walk(const uint2* const* lv, int from, uint32_t idx, uint32_t* vid) {
    for (int j = from; j >= 0; --j) {
        uint2 e = lv[j][idx];
        vid[j] = e.x;
        idx = e.y;
    }
}

__device__ __forceinline__ const DStore& store_of(const ExecDev& E, uint32_t dir) {
    return dir == 0 ? E.out : E.in;
}

// Candidate test of the pre-pruning step and of the other binders.
__device__ __forceinline__ bool keep_candidate(const ExecDev& E, const LevelSpec& L, int l,
                                               uint32_t x, const uint2* rng, uint32_t sel) {
    if (L.use_bitmap) {
        const uint32_t* bm = E.bits + (uint64_t)L.vec * E.words;
        if (!((__ldg(bm + (x >> 5)) >> (x & 31)) & 1u)) return false;
    }
    for (int b = 0; b < L.n_binders; ++b) {
        if ((uint32_t)b == sel) continue;
        uint2 r = rng[b];
        if (!in_range(store_of(E, L.b[b].dir), r.x, r.y, x)) return false;
    }
    for (int j = 0; j < L.n_probes; ++j)
        if (!has_label(store_of(E, L.pr[j].dir), x, L.pr[j].label)) return false;
    for (int j = 0; j < L.n_self; ++j) {
        uint32_t lo, len;
        label_range(E.out, x, L.self_label[j], lo, len);
        if (!in_range(E.out, lo, len, x)) return false;
    }
    return true;
}

// Warp-aggregated append of (x, parent) to a level with capacity cap.
__device__ __forceinline__ void append(Ctl* ctl, int l, uint2* dst, uint64_t cap, bool keep,
                                       uint32_t x, uint32_t parent) {
    const uint32_t lane = lane_id();
    uint32_t m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    uint64_t base = 0;
    uint32_t leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd((unsigned long long*)&ctl->n[l], (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep) {
        uint64_t pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < cap) dst[pos] = make_uint2(x, parent);
        else atomicOr(&ctl->status, kStOverflow);
    }
}

constexpr int kExpItems = 8;                         // candidates per thread per tile
constexpr uint64_t kExpTile = (uint64_t)kThreads * kExpItems;
constexpr uint32_t kExpTileNodes = 2048;             // node offsets of a tile kept in shared memory

__device__ __forceinline__ uint64_t upper_bound_u64(const uint64_t* a, uint64_t lo, uint64_t hi,
                                                    uint64_t key) {
    while (lo < hi) {
        uint64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Programmatic dependent launch. A kernel of the chain waits, before its
// first access to memory, for the one before it to finish (a no-op for a
// kernel launched without the attribute), and lets the next one be
// scheduled once its block has done its main work: the next kernel's
// blocks then hold no SM resources while this one still has work to do.
__device__ __forceinline__ void chain_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void chain_done() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Count kernels split n items (n <= 2^32) into nb chunks of `chunk`
// consecutive items, one per block (the last ones shorter or empty), so
// every block of the grid has work; a consumer finds an item's chunk by a
// 32-bit division.
__device__ __forceinline__ uint32_t even_chunk(uint64_t n, uint32_t nb) {
    const uint64_t c = (n + nb - 1) / nb;
    return c > 0 ? (uint32_t)c : 1u;
}

// End of a count kernel, called by every thread of every block: the block
// hands in its sum; the last block to arrive turns the sums into exclusive
// block offsets (ctl->boff) and writes the total. No block waits for
// another. The counter is left at zero for the next count kernel.
__device__ __forceinline__ void arrive_and_scan(Ctl* ctl, uint64_t block_total, uint64_t* total) {
    __shared__ uint32_t last;
    chain_done();
    if (threadIdx.x == 0) {
        ctl->bsum[blockIdx.x] = block_total;
        __threadfence();   // the sum (and the block's other writes) before the count
        last = atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();       // acquire: every block's sum
    uint64_t carry = 0;
    for (uint32_t base = 0; base < gridDim.x; base += kThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = i < gridDim.x ? __ldcg((const unsigned long long*)&ctl->bsum[i]) : 0;
        uint64_t t;
        const uint64_t ex = block_excl_scan_u64(v, &t);
        if (i < gridDim.x) ctl->boff[i] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0) {
        *total = carry;
        ctl->arrive = 0;
    }
}

// Global exclusive offset of item i of a count kernel's output: its offset
// within its block plus the block's offset.
__device__ __forceinline__ uint64_t roff_at(const uint64_t* roff, const Ctl* ctl, uint32_t chunk,
                                            uint64_t i) {
    return roff[i] + ctl->boff[(uint32_t)i / chunk];
}

// First i in [lo, hi) with roff_at(i) > key (hi when none).
__device__ __forceinline__ uint64_t upper_bound_roff(const uint64_t* roff, const Ctl* ctl,
                                                     uint32_t chunk, uint64_t lo, uint64_t hi,
                                                     uint64_t key) {
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (roff_at(roff, ctl, chunk, mid) <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Root range of a partitioned evaluation: is x a root the evaluation keeps,
// and which bits of candidate word w (vertices 32w .. 32w + 31) are roots it
// keeps.
__device__ __forceinline__ bool root_ok(const ExecDev& E, uint32_t x) {
    return !E.root_cut || (x >= E.root_lo && x < E.root_hi);
}

__device__ __forceinline__ uint32_t root_word_mask(const ExecDev& E, uint32_t w) {
    if (!E.root_cut) return 0xffffffffu;
    const uint64_t v0 = (uint64_t)w * 32, lo = E.root_lo, hi = E.root_hi;
    if (v0 + 32 <= lo || v0 >= hi) return 0u;
    uint32_t m = 0xffffffffu;
    if (lo > v0) m &= 0xffffffffu << (uint32_t)(lo - v0);          // lo - v0 in 1..31
    if (hi < v0 + 32) m &= (1u << (uint32_t)(hi - v0)) - 1u;       // hi - v0 in 1..31
    return m;
}

// upper_bound_roff computed by the whole block (every thread calls it with
// the same arguments and gets the answer): each round probes kThreads
// evenly spaced items at once and counts those <= key (the offsets are
// non-decreasing, so the true probes are a prefix), shrinking the interval
// kThreads-fold; a tile's node bounds then take a few barriers instead of
// one thread's chain of dependent loads while the block waits.
__device__ __forceinline__ uint64_t block_upper_bound_roff(const uint64_t* roff, const Ctl* ctl,
                                                           uint32_t chunk, uint64_t lo, uint64_t hi,
                                                           uint64_t key) {
    while (lo < hi) {
        const uint64_t n = hi - lo;
        const uint64_t step = (n + kThreads - 1) / kThreads;
        const uint64_t p = lo + (uint64_t)threadIdx.x * step;
        const int c = __syncthreads_count(p < hi && roff_at(roff, ctl, chunk, p) <= key);
        if (c == 0) return lo;
        if (step == 1) return lo + (uint64_t)c;
        const uint64_t nlo = lo + (uint64_t)(c - 1) * step + 1;
        hi = min(hi, lo + (uint64_t)c * step);
        lo = nlo;
    }
    return lo;
}

__device__ __forceinline__ bool self_ok(const ExecDev& E, const LevelSpec& L, uint32_t x) {
    for (int j = 0; j < L.n_self; ++j) {
        uint32_t lo, len;
        label_range(E.out, x, L.self_label[j], lo, len);
        if (!in_range(E.out, lo, len, x)) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t word_keep(const ExecDev& E, const LevelSpec& L, uint32_t w,
                                              uint32_t word) {
    if (L.n_self == 0 || word == 0) return word;
    uint32_t out = 0;
    for (uint32_t m = word; m; m &= m - 1) {
        uint32_t b = __ffs(m) - 1;
        if (self_ok(E, L, w * 32 + b)) out |= 1u << b;
    }
    return out;
}

}  // namespace gs
