// Device-side launch interface of the matcher kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "xm_plan_ir.h"

namespace xm {

struct GraphDev {
    const int32_t* out_off;
    const int32_t* out_adj;
    const int32_t* in_off;
    const int32_t* in_adj;
    int32_t n;
};

// Layout of the per-graph control block (unsigned long long words).
enum {
    CTL_HEAD = 0,      // next work unit to hand out
    CTL_COUNT_LO = 1,  // 128-bit match count
    CTL_COUNT_HI = 2,
    CTL_EMIT = 3,      // enumeration cursor
    CTL_STATUS = 4,    // error bits
    CTL_STATS = 8,     // 8 stats words (xm_stats order)
    CTL_WORDS = 16
};

struct RunArgs {
    GraphDev g;
    int32_t* root_chunks;       // n + 1: first-level driver chunks per start node, scanned
    int32_t* chunk_cnt;         // cmax + 1: survivors per chunk, scanned into set offsets
    int32_t* l1set;             // first-level candidate sets of all start nodes
    int32_t* units;             // n + 1: work units per start node, scanned
    int64_t* block_sums;        // scan partials
    int64_t n_block_sums;
    unsigned long long* ctl;    // control block
    int32_t cmax;               // chunk_cnt has cmax + 1 entries
    int32_t r_lo, r_hi;         // start-node range
    int32_t unit;               // first-level candidates per work unit
    int32_t window;             // candidate window per deeper level (ids)
    int32_t* out;               // enumeration buffer (k ints per match)
    unsigned long long capacity;
};

enum { MODE_COUNT = 0, MODE_STATS = 1, MODE_EMIT = 2 };

// Tile of the in-place scans (elements per block).
constexpr int SCAN_TILE = 4096;
// First-level driver positions per chunk of the first-level set build.
constexpr int L1_CHUNK = 1024;

// Upper bound on the number of first-level chunks of a graph.
int64_t chunk_capacity(int32_t n, int64_t m);

// Bytes of shared memory a block of `warps` warps needs.
size_t match_smem_bytes(int k, int window, int warps);

// Enqueues the whole matching pass on `stream`: first-level sets, work
// units, persistent matcher. `plan_dev` is a device copy of the plan.
// `ev` (optional): events recorded before the preparation kernels, before
// the matcher and after it.
cudaError_t launch_match(int mode, const XmPlanDev& plan_host, const XmPlanDev* plan_dev, const RunArgs& a,
                         int warps_per_block, int blocks_per_sm, cudaStream_t stream, cudaEvent_t* ev);

}  // namespace xm
