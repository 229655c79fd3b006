// Executor structures shared by gs_exec.cu and the C ABI.
#pragma once

#include "gs_internal.h"

namespace gs {

constexpr uint32_t kStHuge = 4u;   // a tree node has more than 2^40 answer rows

// Control block at the start of the workspace: level sizes and the
// partial sums of the device-wide scans. Zeroed before each evaluation.
struct Ctl {
    uint64_t n[kMaxLevels];        // nodes per level
    uint64_t list_n[kMaxLevels];   // candidate-list length of a list-fed level
    uint64_t cand;                 // candidates of the level being expanded
    uint64_t one;                  // 1: node count of the virtual parent of level 0
    uint64_t rows;                 // answer rows
    uint32_t status;               // kSt* bits
    uint32_t dead;                 // a pattern with two constant ends has no match
    uint64_t bsum[kBlocks];
    uint64_t boff[kBlocks];
};
constexpr uint64_t kCtlBytes = ((sizeof(Ctl) + 255) / 256) * 256;
constexpr uint64_t kCtlHead = offsetof(Ctl, bsum);   // bytes the host reads back

struct ExecDev {
    uint8_t* arena;
    uint64_t arena_bytes;
    Ctl* ctl;
    DStore out, in;
    uint32_t* bits;           // candidate vector of level l at bits + l * words
    uint64_t words;
    uint32_t* lists;          // candidate list of level l at lists + l * list_stride
    uint64_t list_stride;
};

struct ConstChecks {
    uint32_t n;
    uint32_t t[3 * kMaxPatterns];
};

struct EnumSpec {
    int32_t n_leaves;
    int32_t n_vars;
    LeafSpec leaf[kMaxVars];
    int32_t var_src[kMaxVars];
};

uint64_t host_level_off(const uint64_t* n, int l);
gs_status enqueue_eval(const gs_graph* g, const gs_plan* P, const ExecDev& E, void* scan_work, uint32_t* launches,
                       cudaStream_t st);

}  // namespace gs
