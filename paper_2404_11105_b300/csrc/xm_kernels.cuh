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
    // optional hash index of the lists (null: binary search only): list of
    // node v has a table of out_hoff[v+1]-out_hoff[v] slots (0 or a power of
    // two >= 2 x its length) at out_htab + out_hoff[v]; empty slots hold -1
    const int64_t* out_hoff = nullptr;
    const int32_t* out_htab = nullptr;
    const int64_t* in_hoff = nullptr;
    const int32_t* in_htab = nullptr;
};

// Lists of at least this many ids get a hash table.
constexpr int HASH_MIN_LEN = 32;

// Multiplicative (Fibonacci) hashing, Knuth TAOCP vol. 3 sec. 6.4: the top
// log2(B) bits of x * 2654435769 mod 2^32 select the first bucket of a table
// of B buckets of HASH_BUCKET slots (one 32-byte sector); a full bucket
// continues in the next one (linear probing over buckets, wrapping). Slots
// fill in order within a bucket, so a bucket holding an empty slot (-1)
// ends a search.
constexpr int HASH_BUCKET = 8;

__host__ __device__ __forceinline__ uint32_t hash_bucket(int32_t x, uint32_t nbuckets) {
    // Fibonacci hashing: the top log2(nbuckets) bits of x * 2^32 / phi,
    // taken as the high word of (hash * nbuckets) (nbuckets a power of two)
    const uint32_t h = (uint32_t)x * 2654435769u;
#ifdef __CUDA_ARCH__
    return __umulhi(h, nbuckets);
#else
    return (uint32_t)(((uint64_t)h * nbuckets) >> 32);
#endif
}

// Table size in slots for a list of `len` ids (0: no table): a power of two
// at least twice the length, so tables are at most half full.
__host__ __device__ inline uint32_t hash_table_size(int64_t len) {
    if (len < HASH_MIN_LEN) return 0;
    uint32_t t = HASH_BUCKET;
    while ((int64_t)t < 2 * len) t <<= 1;
    return t;
}

// Ids of the longer list's tile of the merge intersection (shared memory
// per warp): up to four 16-byte loads per lane.
constexpr int MERGE_TILE = 512;
// Default list-length ratio below which two lists are merged instead of
// probing the longer one once per id of the shorter (RunArgs::merge_ratio).
constexpr int MERGE_RATIO_DEFAULT = 2;
// Shorter lists than this are never merged: one round of probes costs less
// than the merge's per-tile rounds.
constexpr int MERGE_MIN_RUN = 64;

// Builds the hash tables of one CSR side on `stream` (tables pre-filled with -1).
cudaError_t build_hash_index(const int32_t* off, const int32_t* adj, const int64_t* hoff, int32_t* htab, int32_t n,
                             cudaStream_t stream);

// Layout of the per-graph control block (unsigned long long words).
enum {
    CTL_HEAD = 0,      // next work unit to hand out
    CTL_COUNT_LO = 1,  // 128-bit match count
    CTL_COUNT_HI = 2,
    CTL_EMIT = 3,      // enumeration cursor
    CTL_STATUS = 4,    // error bits (1: unit count overflow, 2: time budget exceeded)
    CTL_T0 = 5,        // global-timer start of the matcher (budget reference)
    CTL_L1_HEAD = 6,   // next first-level chunk (count pass); 7: write pass
    CTL_STATS = 8,     // 8 stats words: algorithmic bytes, extensions, set operations, units, leaf
                       // elements (matcher); first-level bytes; touched bytes (matcher); unused
    CTL_W_START = 16,  // instrumented matcher: global timer when the first warp started,
    CTL_W_FIRST = 17,  // ~(earliest warp exit), latest warp exit, sum of warp exits after the
    CTL_W_LAST = 18,   // start, warps
    CTL_W_SUM = 19,
    CTL_W_COUNT = 20,
    CTL_ELEN = 21,     // low 32 bits: first-level candidates of the pass (e_units' terminal index)
    CTL_WORDS = 24
};

struct RunArgs {
    GraphDev g;
    int32_t* root_chunks;       // n + 1: first-level driver chunks per start node, scanned
    int32_t* chunk_cnt;         // cmax + 1: survivors per chunk, scanned into set offsets
    int32_t* l1set;             // first-level candidate sets of all start nodes
    int32_t* units;             // n + 1: work units per start node, scanned (two-level patterns)
    int32_t* l1root;            // per first-level candidate: index of its start node
    int32_t* e_units;           // emax + 1: work units per first-level candidate, scanned
    int32_t emax;               // capacity of l1set / l1root (>= any number of first-level candidates)
    int32_t l2_units;           // 1: work units per first-level candidate; 0: per start node
    int32_t leaf_kind;          // three-vertex plans: closed-form last level (leaf_closed_form_kind)
    int64_t* block_sums;        // scan partials
    int64_t n_block_sums;
    unsigned long long* ctl;    // control block
    int32_t cmax;               // chunk_cnt has cmax + 1 entries
    int32_t r_lo, r_hi;         // start-node range
    const int32_t* root_list;   // optional explicit start nodes (null: all nodes 0..n-1)
    int32_t n_idx;              // start-node index space: n, or the root-list length
    int32_t unit;               // first-level candidates per work unit
    int32_t window;             // candidate window per deeper level (ids)
    unsigned long long budget_ns;  // matcher time budget (0: none)
    int32_t* out;               // enumeration buffer (k ints per match)
    unsigned long long capacity;
    unsigned long long* root_counts = nullptr;  // count mode: per-start-node 128-bit counters
                                                // (2 words per node id), else null
    const XmLevel* pv = nullptr;  // leaf-product sets of the device plan when counting
                                  // with a product (set by launch_match), else null
    int32_t merge_ratio = MERGE_RATIO_DEFAULT;  // count-mode leaves with two lists: merge both when
                                                // the longer (cut to the shorter's id range) is at
                                                // most this many times the shorter; <= 0: never
};

enum { MODE_COUNT = 0, MODE_STATS = 1, MODE_EMIT = 2 };
enum { STATUS_OVERFLOW = 1, STATUS_TIMEOUT = 2, STATUS_BAD_ID = 4 };

// Descriptor of a batched launch (device pointers).
struct BatchDev {
    const GraphDev* graphs;          // ng graphs
    const XmPlanDev* plans;          // np plans
    const int2* pairs;               // npairs (plan index, graph index)
    const long long* unit_prefix;    // npairs + 1: scanned units (root blocks) per pair
    unsigned long long* counts;      // 2 per pair (128-bit count)
    unsigned long long* ctl;         // control block (unit counter)
    int32_t npairs;
    int32_t root_block;              // start nodes per work unit
    int32_t window;                  // candidate window per level (ids)
    unsigned long long budget_ns;    // time budget (0: none)
    int32_t kmax;                    // largest pattern in the batch
    int32_t merge_ratio;             // as RunArgs::merge_ratio
    unsigned long long pair_budget_ns = 0;  // per-pair budget of each work unit (0: none)
    unsigned long long* pair_status = nullptr;  // per pair: STATUS_TIMEOUT when its budget ran out
};

// Shared memory per warp of the batched matcher.
size_t batch_warp_bytes(int kmax, int window);

// Enqueues the batched matcher (counts and control block must be zeroed).
cudaError_t launch_batch(const BatchDev& b, int warps_per_block, int blocks_per_sm, cudaStream_t stream);

// Tile of the in-place scans (elements per block).
constexpr int SCAN_TILE = 4096;

// Exclusive scan of int32 v[0..len) in place, with the partials and status
// word of a (block_sums: at least ceil(len / SCAN_TILE) entries; ctl).
cudaError_t scan_int32_in_place(int32_t* v, int64_t len, const RunArgs& a, cudaStream_t stream);

// Device construction of the dual CSR (xm_csr_device.cu).
// Bits b of one key half (2^b >= n).
int csr_key_bits(int32_t n);
// int32 scratch the build needs for m input arcs and n nodes.
int64_t csr_int_scratch(int64_t m, int32_t n);
// Sorts the packed (src, dst) keys of the m input arcs (device arrays) and
// keeps one copy of every arc that is not a self-loop: *keys_out (k0 or k1,
// each m keys) holds the *m_out distinct keys in ascending order.
// Synchronises `stream` once (the distinct count).
cudaError_t csr_sort_unique(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, unsigned long long* k0,
                            unsigned long long* k1, int32_t* ints, const RunArgs& sa, unsigned long long** keys_out,
                            int64_t* m_out, cudaStream_t stream);
// From the mm distinct ascending keys: out_off/out_adj, then in_off/in_adj
// (the keys with halves swapped, sorted; `spare` holds mm keys, `keys` is
// overwritten).
cudaError_t csr_emit(int32_t n, unsigned long long* keys, unsigned long long* spare, int64_t mm, int32_t* ints,
                     const RunArgs& sa, int32_t* out_off, int32_t* out_adj, int32_t* in_off, int32_t* in_adj,
                     cudaStream_t stream);
// Per-node hash-table offsets of one CSR side: hoff[v] = slots of the
// tables of nodes < v (hash_table_size of each list), using ints[n + 1].
cudaError_t hash_offsets(const int32_t* off, int32_t n, int32_t* ints, const RunArgs& sa, int64_t* hoff,
                         cudaStream_t stream);
// First-level driver positions per chunk of the first-level set build.
constexpr int L1_CHUNK = 1024;
// Second-level driver positions per work unit when the second level is the
// last one (three-vertex patterns): leaf intersections are cheap per id.
constexpr int LEAF_UNIT = 1024;

// Common last-level lists longer than this shrink the work units of
// four-level walks (l2_piece).
constexpr int HEAVY_LIST = 4096;

// Upper bound on the number of first-level chunks of a graph.
int64_t chunk_capacity(int32_t n, int64_t m);

// Bytes of shared memory a block of `warps` warps needs (merge: with the
// per-warp merge tiles, when the tuning lets last levels merge).
size_t match_smem_bytes(int k, int window, int warps, bool merge);

// Whether a plan's work units split below the first level (RunArgs::l2_units)
// for a counting (count/stats) or an enumerating pass.
bool use_l2_units(const XmPlanDev& P, bool counting);
// 0, or the closed form that counts a three-vertex plan's last level
// without an intersection per partial match (RunArgs::leaf_kind).
int leaf_closed_form_kind(const XmPlanDev& P);

// Enqueues out[0..1] = sum over v < n of prod_{i < t} cnt_i(v) (mod 2^128),
// cnt_i(v) the 128-bit counter at cnt + i * 2n + 2v.
cudaError_t launch_root_product(const unsigned long long* cnt, int t, int32_t n, unsigned long long* out,
                                cudaStream_t stream);

// Enqueues the whole matching pass on `stream`: first-level sets, work
// units, persistent matcher. `plan_dev` is a device copy of the plan.
// `ev` (optional): events recorded before the preparation kernels, before
// the matcher and after it.
cudaError_t launch_match(int mode, const XmPlanDev& plan_host, const XmPlanDev* plan_dev, const RunArgs& a,
                         int warps_per_block, int blocks_per_sm, cudaStream_t stream, cudaEvent_t* ev);

}  // namespace xm
