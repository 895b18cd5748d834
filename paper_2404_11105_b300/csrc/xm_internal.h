// Internal declarations of the matcher library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/xm.h"
#include "xm_plan_ir.h"

struct xm_plan_s;
struct xm_graph_s;

namespace xm {

struct Decomp;

struct Plan {
    XmPlanDev dev;
    int k = 0, e = 0, flags = 0;
    int aut_size = 1;
    int stab_size = 1;  // rooted plans: automorphisms that fix the root
    int n_reuse = 0;
    int start = 0;
    std::vector<int> split;
    std::vector<int> covered_by;
    std::vector<int32_t> psrc, pdst;
    std::shared_ptr<Decomp> decomp;  // counting by a cut vertex, or null
};

// Count by a cut vertex c of the pattern: the pattern minus c falls apart
// into parts A_1..A_t (each taken with c). A map that is injective on every
// A_i + c is an embedding of the pattern exactly when no two parts share a
// node; otherwise the shared nodes identify vertices of different parts (a
// partition s of V \ {c} whose blocks hold at most one vertex of each part)
// and the map is an embedding of the quotient pattern P/s. Hence
//   emb(P) = sum_v prod_i emb_i(v) - sum_{s not finest} emb(P/s),
// with emb_i(v) the embeddings of A_i + c that map c to node v.
struct Decomp {
    int cut = -1;
    std::vector<std::vector<int>> part_vertices;  // pattern vertices of A_i + c (c first)
    std::vector<Plan> parts;     // rooted plans of A_i + c (vertices relabelled in that order, root 0)
    long long part_factor = 1;   // prod_i |Stab(c) in Aut(A_i + c)|: rooted matches -> embeddings
    std::vector<Plan> quots;     // the quotients P/s, one per isomorphism class
    std::vector<long long> quot_mult;  // number of partitions s in each class
    // Counts restricted to start nodes. When the cut vertex is the plan's
    // start vertex and every automorphism fixes it, all embeddings of one
    // match map c to the same node, and for any node set R
    //   emb_R(P) = part_factor * sum_{v in R} prod_i m_i(v)
    //              - sum_j mult_j * |Stab_j(c)| * sum_{v in R} r_j(v),
    // r_j(v) the rooted matches of quotient j with c mapped to v: rquots[j],
    // Q_j compiled rooted at c (its label 0).
    bool rooted = false;
    std::vector<Plan> rquots;
};

int compile_pattern(int32_t k, int32_t e, const int32_t* psrc, const int32_t* pdst, int flags, Plan& out,
                    std::string& err, int root = -1);
std::string describe_plan(const Plan& p);

void set_error(const std::string& msg);

// Every device allocation of the library goes through these: they keep a
// count of the bytes the library holds (xm_device_bytes_live) and let tests
// make a chosen allocation fail (xm_fault_inject) without touching the GPU.
cudaError_t dev_alloc_raw(void** p, size_t bytes);
void dev_free(void* p);
cudaError_t dev_alloc_async_raw(void** p, size_t bytes, cudaStream_t stream);
cudaError_t dev_free_async(void* p, cudaStream_t stream);
template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
    return dev_alloc_raw(reinterpret_cast<void**>(p), bytes);
}
template <class T>
cudaError_t dev_alloc_async(T** p, size_t bytes, cudaStream_t stream) {
    return dev_alloc_async_raw(reinterpret_cast<void**>(p), bytes, stream);
}
// true when an injected fault makes this pattern compile fail
bool compile_fault();

}  // namespace xm

struct xm_plan_s {
    xm::Plan plan;
    xm_tuning tuning;
};

struct xm_graph_s {
    int32_t n = 0;
    int64_t m = 0;
    int device = 0;
    int32_t* d_out_off = nullptr;
    int32_t* d_out_adj = nullptr;
    int32_t* d_in_off = nullptr;
    int32_t* d_in_adj = nullptr;
    // hash index of the lists (see xm_index.cu)
    int64_t* d_out_hoff = nullptr;
    int32_t* d_out_htab = nullptr;
    int64_t* d_in_hoff = nullptr;
    int32_t* d_in_htab = nullptr;
    int64_t hash_slots = 0;
    // scratch of the matching pipeline (see xm_kernels.cu): first-level
    // chunk counts and offsets, first-level candidate sets, work units, scan
    // partials, and a small control block (counters, accumulators, plan)
    int32_t* d_roots = nullptr;        // n: explicit start nodes (allocated on first use)
    unsigned long long* d_root_counts = nullptr;  // per-node part counters of split counts (on first use)
    size_t root_count_words = 0;
    int32_t* d_root_chunks = nullptr;  // n + 1
    int32_t* d_chunk_cnt = nullptr;    // cmax + 1
    int32_t* d_l1set = nullptr;        // max(m, 1)
    int32_t* d_units = nullptr;        // n + 1
    int32_t* d_l1root = nullptr;       // max(m, 1): start-node index of each first-level candidate
    int32_t* d_e_units = nullptr;      // max(m, 1) + 1: work units per first-level candidate
    int64_t* d_block_sums = nullptr;
    unsigned long long* d_ctl = nullptr;
    int64_t n_block_sums = 0;
    int64_t cmax = 0;
    // events around the last matching pass's kernels (prep start, match
    // start, match end), and the sums of those times over the passes of the
    // last public call (several for a cut-vertex split)
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    bool timed = false;
    float sum_prep_ms = 0.f, sum_match_ms = 0.f;
};
