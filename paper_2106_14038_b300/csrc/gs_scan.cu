// Triple scan: candidate vectors of query variables by grouped predicate
// selection (Sec. 5, Step 1). For a variable u with out-predicates O(u)
// (u is the subject) and in-predicates I(u) (u is the object):
//
//     v_u = AND_{p in O(u)} (A (x) u_p)  AND  AND_{p in I(u)} (A^T (x) u_p)
//
// (Eq. 17 with only outgoing edges, Eq. 21 with both; Eq. 4 and Eq. 5 for
// the single selections). All predicates of the query are tested in one
// pass over the label array of each orientation:
//   1. k_scan_rows streams the CSR labels and writes, per vertex, the mask
//      of query out-predicates its row holds;
//   2. k_scan_cols streams the CSC labels, forms the in-mask per vertex,
//      combines it with the out-mask and writes one bit per variable
//      (warp ballot -> one 32-bit word per 32 vertices);
//   3. k_scan_fixup finishes the vertices whose column is heavy.
// Light rows (<= kHeavyDeg entries) are read by one lane each with
// aligned 16-byte loads; heavy rows are cut into chunks of kHeavyChunk
// entries, one warp per chunk, with coalesced 16-byte loads and a warp OR
// reduction. Bytes moved per pass: 4(N+1) row pointers + 4M labels, plus a
// 4N mask written and read once and N/8 per produced vector.
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

// label -> slot bit lookup in shared memory (P + 1 bytes: slot + 1, 0 = none)
__device__ __forceinline__ void fill_lut(uint8_t* lut, uint32_t P, const uint32_t* preds,
                                         uint32_t n) {
    for (uint32_t i = threadIdx.x; i <= P; i += blockDim.x) lut[i] = 0;
    __syncthreads();
    if (threadIdx.x < n) lut[preds[threadIdx.x]] = (uint8_t)(threadIdx.x + 1);
    __syncthreads();
}

__device__ __forceinline__ uint32_t lut_bit(const uint8_t* lut, uint32_t P, uint32_t l) {
    uint32_t s = l <= P ? lut[l] : 0u;
    return s ? (1u << (s - 1)) : 0u;
}

// OR of the slot bits of lab[b..e) using aligned 16-byte loads.
__device__ __forceinline__ uint32_t row_mask(const uint32_t* __restrict__ lab, uint32_t b,
                                             uint32_t e, const uint8_t* lut, uint32_t P) {
    uint32_t m = 0;
    if (b >= e) return m;
    const uint4* v = reinterpret_cast<const uint4*>(lab);
    uint32_t q0 = b >> 2, q1 = (e + 3) >> 2;
#pragma unroll 4
    for (uint32_t q = q0; q < q1; ++q) {
        uint4 x = __ldg(v + q);
        uint32_t k = q << 2;
        if (k >= b && k < e) m |= lut_bit(lut, P, x.x);
        if (k + 1 >= b && k + 1 < e) m |= lut_bit(lut, P, x.y);
        if (k + 2 >= b && k + 2 < e) m |= lut_bit(lut, P, x.z);
        if (k + 3 >= b && k + 3 < e) m |= lut_bit(lut, P, x.w);
    }
    return m;
}

// Warp-cooperative OR over lab[b..e) (a heavy-row chunk).
__device__ __forceinline__ uint32_t chunk_mask(const uint32_t* __restrict__ lab, uint32_t b,
                                               uint32_t e, const uint8_t* lut, uint32_t P) {
    const uint32_t lane = lane_id();
    const uint4* v = reinterpret_cast<const uint4*>(lab);
    uint32_t q0 = b >> 2, q1 = (e + 3) >> 2;
    uint32_t m = 0;
#pragma unroll 4
    for (uint32_t q = q0 + lane; q < q1; q += 32) {
        uint4 x = __ldg(v + q);
        uint32_t k = q << 2;
        if (k >= b && k < e) m |= lut_bit(lut, P, x.x);
        if (k + 1 >= b && k + 1 < e) m |= lut_bit(lut, P, x.y);
        if (k + 2 >= b && k + 2 < e) m |= lut_bit(lut, P, x.z);
        if (k + 3 >= b && k + 3 < e) m |= lut_bit(lut, P, x.w);
    }
    return __reduce_or_sync(0xffffffffu, m);
}

// Heavy rows' mask slots start at zero; the chunks OR into them.
__global__ void k_scan_zero(const uint32_t* __restrict__ hrow_out, uint32_t n_out_heavy,
                            uint32_t* __restrict__ mask_out, uint32_t* __restrict__ hmask_in,
                            uint32_t n_in_heavy) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_out_heavy;
         i += gridDim.x * blockDim.x)
        mask_out[hrow_out[i]] = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_in_heavy;
         i += gridDim.x * blockDim.x)
        hmask_in[i] = 0;
}

// Pass 1: out-masks of all rows. Work items: N/32 groups of 32 rows (one
// lane per row), then the heavy chunks (one warp each).
__global__ void __launch_bounds__(kThreads) k_scan_rows(DStore S, uint32_t N, uint32_t P,
                                                        const uint32_t* __restrict__ chunk_h,
                                                        const uint32_t* __restrict__ chunk_start,
                                                        const uint32_t* __restrict__ hrow,
                                                        uint32_t n_chunks, ScanDev sd,
                                                        uint32_t* __restrict__ mask_out) {
    extern __shared__ uint8_t lut[];
    fill_lut(lut, P, sd.out_pred, sd.n_out);
    const uint32_t lane = lane_id();
    const uint32_t groups = (N + 31) / 32;
    const uint64_t items = (uint64_t)groups + n_chunks;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t it = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); it < items;
         it += warps) {
        if (it < groups) {
            uint32_t v = (uint32_t)it * 32 + lane;
            if (v < N) {
                uint32_t b = ld(S.ptr + v), e = ld(S.ptr + v + 1);
                if (e - b <= kHeavyDeg) mask_out[v] = row_mask(S.lab, b, e, lut, P);
            }
        } else {
            uint32_t c = (uint32_t)(it - groups);
            uint32_t r = ld(hrow + ld(chunk_h + c));
            uint32_t b = ld(chunk_start + c);
            uint32_t e = min(b + kHeavyChunk, ld(S.ptr + r + 1));
            uint32_t m = chunk_mask(S.lab, b, e, lut, P);
            if (lane == 0 && m) atomicOr(mask_out + r, m);
        }
    }
}

__device__ __forceinline__ uint32_t eval_bits(const ScanDev& sd, uint32_t mo, uint32_t mi,
                                              uint32_t u) {
    return ((mo & sd.need_out[u]) == sd.need_out[u]) && ((mi & sd.need_in[u]) == sd.need_in[u]);
}

// Pass 2: in-masks of the columns, combined with the out-masks into one
// bit per (variable, vertex). Heavy columns are left to k_scan_fixup.
__global__ void __launch_bounds__(kThreads) k_scan_cols(DStore S, uint32_t N, uint32_t P,
                                                        const uint32_t* __restrict__ chunk_h,
                                                        const uint32_t* __restrict__ chunk_start,
                                                        const uint32_t* __restrict__ hrow,
                                                        uint32_t n_chunks, ScanDev sd,
                                                        const uint32_t* __restrict__ mask_out,
                                                        uint32_t* __restrict__ hmask_in,
                                                        uint32_t* __restrict__ bits, uint32_t words) {
    extern __shared__ uint8_t lut[];
    fill_lut(lut, P, sd.in_pred, sd.n_in);
    const uint32_t lane = lane_id();
    const uint32_t groups = (N + 31) / 32;
    const uint64_t items = (uint64_t)groups + n_chunks;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t it = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); it < items;
         it += warps) {
        if (it < groups) {
            uint32_t v = (uint32_t)it * 32 + lane;
            uint32_t mo = 0, mi = 0;
            bool ok = false;
            if (v < N) {
                uint32_t b = ld(S.ptr + v), e = ld(S.ptr + v + 1);
                if (e - b <= kHeavyDeg) {
                    mi = row_mask(S.lab, b, e, lut, P);
                    mo = mask_out[v];
                    ok = true;
                }
            }
            for (uint32_t u = 0; u < sd.n_bvars; ++u) {
                uint32_t w = __ballot_sync(0xffffffffu, ok && eval_bits(sd, mo, mi, u));
                if (lane == 0) bits[(uint64_t)u * words + it] = w;
            }
        } else {
            uint32_t c = (uint32_t)(it - groups);
            uint32_t h = ld(chunk_h + c);
            uint32_t r = ld(hrow + h);
            uint32_t b = ld(chunk_start + c);
            uint32_t e = min(b + kHeavyChunk, ld(S.ptr + r + 1));
            uint32_t m = chunk_mask(S.lab, b, e, lut, P);
            if (lane == 0 && m) atomicOr(hmask_in + h, m);
        }
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
    const uint32_t words = (g->N + 31) / 32;
    const size_t smem = (size_t)g->P + 1;
    if (smem > 48 * 1024) {
        GS_CUDA(cudaFuncSetAttribute(k_scan_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GS_CUDA(cudaFuncSetAttribute(k_scan_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    const int nb = g->n_blocks;
    k_scan_zero<<<nb, kThreads, 0, st>>>(g->out.hrow, g->out.n_heavy, mask_out, hmask_in,
                                         g->in.n_heavy);
    k_scan_rows<<<nb, kThreads, smem, st>>>(dview(g->out), g->N, g->P, g->out.chunk_h,
                                             g->out.chunk_start, g->out.hrow, g->out.n_chunks, sd,
                                             mask_out);
    k_scan_cols<<<nb, kThreads, smem, st>>>(dview(g->in), g->N, g->P, g->in.chunk_h,
                                             g->in.chunk_start, g->in.hrow, g->in.n_chunks, sd,
                                             mask_out, hmask_in, bits, words);
    k_scan_fixup<<<nb, kThreads, 0, st>>>(g->in.hrow, g->in.n_heavy, sd, mask_out, hmask_in, bits,
                                          words);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs
