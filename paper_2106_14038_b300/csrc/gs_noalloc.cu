// gs_scan_candidates_noalloc: the grouped predicate selection of
// gs_scan_candidates (Eq. 17, Eq. 21) with its workspace taken from a
// fixed static device array instead of the graph's allocator. The paper
// has no counterpart; the entry point exists for callers that must not
// allocate device memory on the call path.
//
// Scratch: kNoAllocScratchBytes in the file-scope array below. The call
// needs scan_work_bytes(g) of it (a little over 4 (N + 256) bytes) and
// rejects graphs that need more. Nothing in the array has to start at
// zero: the first kernel of every call zeroes every word the scan ORs into
// and the status word; all other masks are written before they are read.
//
// Set-up: the first call on a device looks the array's address up with
// cudaGetSymbolAddress (which may load this module) and caches it; make
// that first call before any stream capture begins.
//
// Races: every call on a device uses the same array. Two calls whose work
// overlaps in time on one device (different streams, or different host
// threads without ordering) corrupt each other's masks; calls on one
// stream are ordered and safe.
#include <mutex>

#include "gs_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(48) << 20;   // 48 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Address of the static array on `dev`, looked up once per device.
gs_status scratch_for(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        gs::set_error("gs_scan_candidates_noalloc: device %d outside 0..%d", dev, kMaxDevices - 1);
        return GS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return gs::cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                 "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

}  // namespace

extern "C" {

size_t gs_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

gs_status gs_scan_candidates_noalloc(gs_graph* g, const uint32_t* preds, const uint8_t* dirs,
                                     uint32_t n, uint32_t* out_bits, void* cuda_stream) {
    if (!g || !preds || !dirs || !out_bits || n == 0) {
        gs::set_error("gs_scan_candidates_noalloc: NULL argument or n == 0");
        return GS_EINVAL;
    }
    gs::ScanSpec S{};
    S.n_bvars = 1;
    S.bvar[0] = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (preds[i] < 1 || preds[i] > g->P || dirs[i] > 1) {
            gs::set_error("gs_scan_candidates_noalloc: entry %u: predicate outside 1..P or "
                          "direction not 0/1", i);
            return GS_EINVAL;
        }
        uint32_t* list = dirs[i] ? S.in_pred : S.out_pred;
        int32_t& cnt = dirs[i] ? S.n_in : S.n_out;
        int slot = -1;
        for (int j = 0; j < cnt; ++j)
            if (list[j] == preds[i]) slot = j;
        if (slot < 0) {
            if (cnt >= gs::kMaxSlots) {
                gs::set_error("gs_scan_candidates_noalloc: more than %d predicates in one "
                              "direction", gs::kMaxSlots);
                return GS_EINVAL;
            }
            list[cnt] = preds[i];
            slot = cnt++;
        }
        (dirs[i] ? S.need_in[0] : S.need_out[0]) |= 1u << slot;
    }
    const size_t need = gs::scan_work_bytes(g);
    if (need > kNoAllocScratchBytes) {
        gs::set_error("gs_scan_candidates_noalloc: graph needs %zu bytes of scratch (N = %u); "
                      "the static area holds %zu", need, g->N, kNoAllocScratchBytes);
        return GS_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gs::cuda_fail(e, "cudaGetDevice");
    if (dev != g->device) {
        gs::set_error("gs_scan_candidates_noalloc: current device %d is not the graph's (%d)",
                      dev, g->device);
        return GS_EINVAL;
    }
    void* work = nullptr;
    gs_status rc = scratch_for(dev, &work);
    if (rc != GS_OK) return rc;
    return gs::run_scan(g, S, out_bits, work, (cudaStream_t)cuda_stream);
}

}  // extern "C"
