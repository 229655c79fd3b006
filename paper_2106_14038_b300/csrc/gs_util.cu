// Error reporting, the allocation hook and the device-wide scan kernels.
#include <cstdarg>
#include <cstdio>

#include "gs_device.cuh"

namespace gs {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char* last_error() { return g_err; }

gs_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return GS_ENOMEM;
    }
    return GS_ECUDA;
}

void* Alloc::get(size_t bytes, cudaStream_t st) const {
    if (bytes == 0) bytes = 256;
    if (has_hook) {
        // the bulk copies and 16-byte accesses rely on cudaMalloc's alignment
        void* p = hook.alloc(bytes, (void*)st, hook.ctx);
        if (p && ((uintptr_t)p & 255u)) {
            hook.free(p, (void*)st, hook.ctx);
            return nullptr;
        }
        return p;
    }
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Alloc::put(void* p, cudaStream_t st) const {
    if (!p) return;
    if (has_hook) hook.free(p, (void*)st, hook.ctx);
    else cudaFreeAsync(p, st);
}

__global__ void k_scan_block_sums(const uint64_t* __restrict__ bsum, uint64_t* __restrict__ boff,
                                  uint32_t nb, uint64_t* total, const uint32_t* status) {
    if (status && (*status & kStOverflow)) return;
    uint64_t carry = 0;
    for (uint32_t base = 0; base < nb; base += kThreads) {
        uint32_t i = base + threadIdx.x;
        uint64_t v = i < nb ? bsum[i] : 0, t;
        uint64_t ex = block_excl_scan_u64(v, &t);
        if (i < nb) boff[i] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply_u64(uint64_t* __restrict__ a, const uint64_t* n_ptr,
                                 const uint64_t* __restrict__ boff, const uint32_t* status) {
    if (status && (*status & kStOverflow)) return;
    uint64_t beg, end;
    block_chunk(*n_ptr, blockIdx.x, gridDim.x, beg, end);
    uint64_t carry = boff[blockIdx.x];
    for (uint64_t base = beg; base < end; base += kThreads) {
        uint64_t i = base + threadIdx.x;
        uint64_t v = i < end ? a[i] : 0, t;
        uint64_t ex = block_excl_scan_u64(v, &t);
        if (i < end) a[i] = carry + ex;
        carry += t;
    }
}

__global__ void k_block_sums_u64(const uint64_t* __restrict__ a, const uint64_t* n_ptr,
                                 uint64_t* __restrict__ bsum, const uint32_t* status) {
    if (status && (*status & kStOverflow)) return;
    uint64_t beg, end;
    block_chunk(*n_ptr, blockIdx.x, gridDim.x, beg, end);
    uint64_t s = 0;
    for (uint64_t i = beg + threadIdx.x; i < end; i += kThreads) s += a[i];
    s = block_sum_u64(s);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

}  // namespace gs
