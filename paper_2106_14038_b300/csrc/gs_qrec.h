// Compact query record for the single-block executor: the schedule of one
// query (levels, leaves, constant checks) packed into a few hundred bytes,
// staged in shared memory by the kernels that run whole queries in one CTA
// (the plain single-block kernel and the batch kernel).
#pragma once

#include <cstring>

#include "gs_internal.h"

namespace gs {

constexpr int kRecLevels = 12;   // queries with more levels use the grid path
constexpr int kRecCC = 8;        // patterns with two constant ends

struct QHdr {
    int32_t n_levels, n_leaves, n_cc, n_vars;
    int32_t var_src[kMaxVars];
    uint32_t cc[3 * kRecCC];
    uint32_t bytes;               // size of the whole record
    uint32_t pad[3];
};

// Record layout: QHdr | LevelSpec[n_levels] | LeafSpec[n_leaves], 16-byte aligned.
constexpr size_t kRecMax =
    ((sizeof(QHdr) + kRecLevels * sizeof(LevelSpec) + kMaxVars * sizeof(LeafSpec)) + 15) & ~size_t(15);

struct QRec {
    const QHdr* h;
    const LevelSpec* lv;
    const LeafSpec* lf;
};

__host__ __device__ inline QRec rec_view(const void* base) {
    QRec q;
    q.h = (const QHdr*)base;
    q.lv = (const LevelSpec*)((const char*)base + sizeof(QHdr));
    q.lf = (const LeafSpec*)((const char*)base + sizeof(QHdr) + q.h->n_levels * sizeof(LevelSpec));
    return q;
}

inline bool rec_fits(const gs_plan* P) {
    return !P->needs_scan && P->n_levels > 0 && P->n_levels <= kRecLevels &&
           P->const_triples.size() / 3 <= (size_t)kRecCC;
}

// Packs the plan's schedule; returns the record size (0 when it does not fit).
inline size_t pack_record(const gs_plan* P, void* dst) {
    if (!rec_fits(P)) return 0;
    QHdr h;
    std::memset(&h, 0, sizeof(h));
    h.n_levels = P->n_levels;
    h.n_leaves = P->n_leaves;
    h.n_cc = (int32_t)(P->const_triples.size() / 3);
    h.n_vars = P->n_vars;
    for (int v = 0; v < P->n_vars; ++v) h.var_src[v] = P->var_src[v];
    for (size_t i = 0; i < P->const_triples.size(); ++i) h.cc[i] = P->const_triples[i];
    size_t bytes = sizeof(QHdr) + P->n_levels * sizeof(LevelSpec) + P->n_leaves * sizeof(LeafSpec);
    bytes = (bytes + 15) & ~size_t(15);
    h.bytes = (uint32_t)bytes;
    char* d = (char*)dst;
    std::memcpy(d, &h, sizeof(QHdr));
    std::memcpy(d + sizeof(QHdr), P->levels, P->n_levels * sizeof(LevelSpec));
    std::memcpy(d + sizeof(QHdr) + P->n_levels * sizeof(LevelSpec), P->leaves,
                P->n_leaves * sizeof(LeafSpec));
    return bytes;
}

// A query record passed by value to the plain single-block kernel.
struct RecParam {
    uint4 w[kRecMax / 16];
};

}  // namespace gs
