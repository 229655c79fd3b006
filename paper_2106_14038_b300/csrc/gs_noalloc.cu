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
// that first call before any stream capture begins (a first call on a
// capturing stream returns GS_EINVAL).
//
// Stalls: a bounded wait of the scan that runs out is ORed into the graph's
// status word (set up at load, not here) and reported by gs_scan_status.
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

// Address of the static array on `dev`, looked up once per device. The
// look-up may load this module, which a stream capture does not allow: a
// first call on a capturing stream is refused.
gs_status scratch_for(int dev, cudaStream_t st, void** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        gs::set_error("gs_scan_candidates_noalloc: device %d outside 0..%d", dev, kMaxDevices - 1);
        return GS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing(st, &cap);
        if (ce != cudaSuccess) return gs::cuda_fail(ce, "cudaStreamIsCapturing");
        if (cap != cudaStreamCaptureStatusNone) {
            gs::set_error("gs_scan_candidates_noalloc: the first call on device %d must come "
                          "before any stream capture (it looks up the static workspace)", dev);
            return GS_EINVAL;
        }
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
    if (!out_bits) {
        gs::set_error("gs_scan_candidates_noalloc: out_bits is NULL");
        return GS_EINVAL;
    }
    gs::ScanSpec S{};
    gs_status rc = gs::scan_spec_from(g, preds, dirs, n, &S, "gs_scan_candidates_noalloc");
    if (rc != GS_OK) return rc;
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
    rc = scratch_for(dev, (cudaStream_t)cuda_stream, &work);
    if (rc != GS_OK) return rc;
    // a stalled wait is reported through the graph's status word (set up
    // when the graph was loaded), which gs_scan_status reads
    return gs::run_scan(g, S, out_bits, work, (cudaStream_t)cuda_stream, g->scan_status);
}

}  // extern "C"
