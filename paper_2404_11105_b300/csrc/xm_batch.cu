// Batched matching: many (pattern, graph) pairs in one persistent launch,
// optionally replayed from a captured CUDA graph, with a small autotuner for
// the launch parameters. The pairs are independent matching problems; the
// kernel (k_match_batch) hands out blocks of start nodes of every pair from
// one global counter.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "xm_internal.h"
#include "xm_kernels.cuh"

struct xm_batch_s {
    int device = 0;
    int64_t npairs = 0;
    int kmax = 2;
    xm_tuning tuning{256, 64, 8, 0, 0, xm::MERGE_RATIO_DEFAULT};
    std::vector<int32_t> pair_n;  // start nodes of each pair's graph
    xm::GraphDev* d_graphs = nullptr;
    XmPlanDev* d_plans = nullptr;
    int2* d_pairs = nullptr;
    long long* d_prefix = nullptr;
    unsigned long long* d_counts = nullptr;
    unsigned long long* d_ctl = nullptr;
    unsigned long long* d_pair_words = nullptr;  // per pair: unused word, status (per-pair budgets)
    int32_t pair_budget_ms = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

namespace xm {
namespace {

int fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA;
}

void drop_graph(xm_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

void free_batch(xm_batch_s* b) {
    if (!b) return;
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    dev_free(b->d_graphs);
    dev_free(b->d_plans);
    dev_free(b->d_pairs);
    dev_free(b->d_prefix);
    dev_free(b->d_counts);
    dev_free(b->d_ctl);
    dev_free(b->d_pair_words);
    delete b;
}

// Work-unit prefix for a root block size (host), uploaded synchronously.
int upload_prefix(xm_batch_s* b, int root_block) {
    std::vector<long long> prefix(b->npairs + 1, 0);
    for (int64_t i = 0; i < b->npairs; i++)
        prefix[i + 1] = prefix[i] + (b->pair_n[i] + root_block - 1) / root_block;
    cudaError_t e = cudaMemcpy(b->d_prefix, prefix.data(), prefix.size() * sizeof(long long), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? XM_OK : fail(e, "batch prefix upload");
}

BatchDev descriptor(const xm_batch_s* b) {
    BatchDev d;
    d.graphs = b->d_graphs;
    d.plans = b->d_plans;
    d.pairs = b->d_pairs;
    d.unit_prefix = b->d_prefix;
    d.counts = b->d_counts;
    d.ctl = b->d_ctl;
    d.npairs = (int32_t)b->npairs;
    d.root_block = b->tuning.unit;
    d.window = b->tuning.window;
    d.kmax = b->kmax;
    d.budget_ns = (unsigned long long)b->tuning.budget_ms * 1000000ull;
    d.merge_ratio = b->tuning.merge_ratio;
    d.pair_budget_ns = (unsigned long long)b->pair_budget_ms * 1000000ull;
    d.pair_status = b->d_pair_words + b->npairs;
    return d;
}

cudaError_t enqueue(xm_batch_s* b, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(b->d_counts, 0, (size_t)b->npairs * 2 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctl, 0, CTL_WORDS * sizeof(unsigned long long), stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_pair_words, 0, (size_t)b->npairs * 2 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = launch_batch(descriptor(b), b->tuning.warps_per_block, b->tuning.blocks_per_sm, stream);
    return e;
}

int check_device(const xm_batch_s* b) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e, "cudaGetDevice");
    if (dev != b->device) { set_error("batch lives on another device than the current one"); return XM_EINVAL; }
    return XM_OK;
}

}  // namespace
}  // namespace xm

using namespace xm;

extern "C" {

int xm_batch_create(int32_t np, const xm_plan* plans, int32_t ng, const xm_graph* graphs, int64_t npairs,
                    const int32_t* pair_pg, xm_batch* out) {
    if (!out || np < 1 || ng < 1 || npairs < 1 || !plans || !graphs || !pair_pg) {
        set_error("bad batch arguments");
        return XM_EINVAL;
    }
    if (npairs >= INT32_MAX) { set_error("too many pairs"); return XM_EINVAL; }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e, "cudaGetDevice");
    std::vector<GraphDev> hg(ng);
    for (int i = 0; i < ng; i++) {
        const xm_graph g = graphs[i];
        if (!g) { set_error("NULL graph in batch"); return XM_EINVAL; }
        if (g->device != dev) { set_error("batch graph lives on another device"); return XM_EINVAL; }
        hg[i] = {g->d_out_off, g->d_out_adj, g->d_in_off, g->d_in_adj, g->n,
                 g->d_out_hoff, g->d_out_htab, g->d_in_hoff, g->d_in_htab};
    }
    std::vector<XmPlanDev> hp(np);
    int kmax = 2;
    for (int i = 0; i < np; i++) {
        if (!plans[i]) { set_error("NULL plan in batch"); return XM_EINVAL; }
        hp[i] = plans[i]->plan.dev;
        kmax = std::max(kmax, plans[i]->plan.k);
    }
    xm_batch_s* b = new xm_batch_s();
    b->device = dev;
    b->npairs = npairs;
    b->kmax = kmax;
    b->pair_n.resize(npairs);
    std::vector<int2> hpairs(npairs);
    for (int64_t i = 0; i < npairs; i++) {
        const int32_t pi = pair_pg[2 * i], gi = pair_pg[2 * i + 1];
        if (pi < 0 || pi >= np || gi < 0 || gi >= ng) {
            delete b;
            set_error("pair index out of range");
            return XM_EINVAL;
        }
        hpairs[i] = make_int2(pi, gi);
        b->pair_n[i] = hg[gi].n;
    }
    e = dev_alloc(&b->d_graphs, ng * sizeof(GraphDev));
    if (e == cudaSuccess) e = dev_alloc(&b->d_plans, np * sizeof(XmPlanDev));
    if (e == cudaSuccess) e = dev_alloc(&b->d_pairs, npairs * sizeof(int2));
    if (e == cudaSuccess) e = dev_alloc(&b->d_prefix, (npairs + 1) * sizeof(long long));
    if (e == cudaSuccess) e = dev_alloc(&b->d_counts, npairs * 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = dev_alloc(&b->d_ctl, CTL_WORDS * sizeof(unsigned long long));
    if (e == cudaSuccess) e = dev_alloc(&b->d_pair_words, (size_t)npairs * 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_graphs, hg.data(), ng * sizeof(GraphDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_plans, hp.data(), np * sizeof(XmPlanDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_pairs, hpairs.data(), npairs * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int rc = fail(e, "batch set-up");
        free_batch(b);
        return rc;
    }
    int rc = upload_prefix(b, b->tuning.unit);
    if (rc) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return XM_OK;
}

int xm_batch_set_tuning(xm_batch b, const xm_tuning* t) {
    if (!b || !t) { set_error("NULL argument"); return XM_EINVAL; }
    xm_tuning v = *t;
    if (v.window == 0) v.window = 256;
    if (v.unit == 0) v.unit = 64;
    if (v.warps_per_block == 0) v.warps_per_block = 8;
    if (v.window < 64 || v.window > 4096 || (v.window & 31)) { set_error("window must be a multiple of 32 in [64, 4096]"); return XM_EINVAL; }
    if (v.unit < 1 || v.unit > 65536) { set_error("unit (start nodes per work unit) must be in [1, 65536]"); return XM_EINVAL; }
    if (v.warps_per_block < 1 || v.warps_per_block > 16) { set_error("warps_per_block must be in [1, 16]"); return XM_EINVAL; }
    if (v.blocks_per_sm < 0 || v.blocks_per_sm > 64) { set_error("blocks_per_sm must be in [0, 64]"); return XM_EINVAL; }
    if (v.budget_ms < 0) { set_error("budget_ms must be >= 0"); return XM_EINVAL; }
    if (v.merge_ratio == 0) v.merge_ratio = MERGE_RATIO_DEFAULT;
    if (v.merge_ratio != -1 && (v.merge_ratio < 1 || v.merge_ratio > 1024)) {
        set_error("merge_ratio must be -1 or in [1, 1024] (0: default)");
        return XM_EINVAL;
    }
    int rc = check_device(b);
    if (rc) return rc;
    if (v.unit != b->tuning.unit && (rc = upload_prefix(b, v.unit))) return rc;
    b->tuning = v;
    drop_graph(b);
    return XM_OK;
}

int xm_batch_get_tuning(xm_batch b, xm_tuning* t) {
    if (!b || !t) { set_error("NULL argument"); return XM_EINVAL; }
    *t = b->tuning;
    return XM_OK;
}

int xm_batch_run(xm_batch b, void* stream) {
    if (!b) { set_error("NULL batch"); return XM_EINVAL; }
    int rc = check_device(b);
    if (rc) return rc;
    cudaError_t e = enqueue(b, (cudaStream_t)stream);
    return e == cudaSuccess ? XM_OK : fail(e, "batch launch");
}

int xm_batch_run_graph(xm_batch b, void* stream) {
    if (!b) { set_error("NULL batch"); return XM_EINVAL; }
    int rc = check_device(b);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (!b->exec) {
        // one eager launch sets the kernel attributes outside the capture
        e = enqueue(b, b->cap_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap_stream);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue(b, b->cap_stream);
            e = cudaStreamEndCapture(b->cap_stream, &b->graph);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return fail(e, "batch graph capture");
        }
    }
    e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? XM_OK : fail(e, "batch graph launch");
}

int xm_batch_counts(xm_batch b, uint64_t* out_counts, void* stream) {
    if (!b || !out_counts) { set_error("NULL argument"); return XM_EINVAL; }
    int rc = check_device(b);
    if (rc) return rc;
    unsigned long long ctl[CTL_WORDS];
    cudaError_t e = cudaMemcpyAsync(out_counts, b->d_counts, (size_t)b->npairs * 2 * sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, b->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail(e, "batch readback");
    if (ctl[CTL_STATUS] & STATUS_TIMEOUT) { set_error("time budget of the batch exceeded; counts incomplete"); return XM_ETIMEOUT; }
    return XM_OK;
}

int xm_batch_tune(xm_batch b, const xm_tuning* cand, int32_t ncand, int32_t reps, xm_tuning* best, float* best_ms,
                  void* stream_) {
    if (!b || !cand || ncand < 1 || reps < 1) { set_error("bad tuning arguments"); return XM_EINVAL; }
    cudaStream_t stream = (cudaStream_t)stream_;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return fail(e, "cudaEventCreate");
    float best_t = -1.0f;
    xm_tuning best_c = b->tuning;
    int rc = XM_OK;
    for (int c = 0; c < ncand && rc == XM_OK; c++) {
        if ((rc = xm_batch_set_tuning(b, &cand[c]))) break;
        // warm-up launch, then the fastest of `reps` timed launches
        if ((rc = xm_batch_run(b, stream))) break;
        float t_min = -1.0f;
        for (int r = 0; r < reps && rc == XM_OK; r++) {
            e = cudaEventRecord(e0, stream);
            if (e == cudaSuccess && (rc = xm_batch_run(b, stream))) break;
            if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { rc = fail(e, "tuning timing"); break; }
            if (t_min < 0 || ms < t_min) t_min = ms;
        }
        if (rc == XM_OK && (best_t < 0 || t_min < best_t)) {
            best_t = t_min;
            best_c = b->tuning;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = xm_batch_set_tuning(b, &best_c))) return rc;
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return XM_OK;
}

void xm_batch_free(xm_batch b) { free_batch(b); }

int xm_batch_set_pair_budget(xm_batch b, int32_t budget_ms) {
    if (!b || budget_ms < 0) { set_error("bad per-pair budget"); return XM_EINVAL; }
    b->pair_budget_ms = budget_ms;
    drop_graph(b);
    return XM_OK;
}

int xm_batch_pair_status(xm_batch b, int32_t* status, void* stream) {
    if (!b || !status) { set_error("NULL argument"); return XM_EINVAL; }
    int rc = check_device(b);
    if (rc) return rc;
    std::vector<unsigned long long> st(b->npairs);
    cudaError_t e = cudaMemcpyAsync(st.data(), b->d_pair_words + b->npairs, st.size() * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail(e, "pair status readback");
    for (int64_t i = 0; i < b->npairs; i++) status[i] = (st[i] & STATUS_TIMEOUT) ? XM_ETIMEOUT : XM_OK;
    return XM_OK;
}

int xm_count_batch(int32_t np, const xm_plan* plans, int32_t ng, const xm_graph* graphs, int64_t npairs,
                   const int32_t* pair_pg, uint64_t* out_counts, void* stream) {
    if (!out_counts) { set_error("NULL output"); return XM_EINVAL; }
    xm_batch b = nullptr;
    int rc = xm_batch_create(np, plans, ng, graphs, npairs, pair_pg, &b);
    if (rc) return rc;
    rc = xm_batch_run(b, stream);
    if (rc == XM_OK) rc = xm_batch_counts(b, out_counts, stream);
    xm_batch_free(b);
    return rc;
}

}  // extern "C"
