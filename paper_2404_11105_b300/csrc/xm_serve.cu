// Serving: resident graphs, queries admitted into slots by their scratch
// memory, each slot running its query's kernels on its own stream so that
// queries that arrive while others are on the GPU overlap with them
// (continuous batching driven from the host). Submission and polling never
// block on the GPU; stream-ordered allocation (cudaMallocAsync) takes and
// returns each query's scratch on the slot's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "xm_internal.h"
#include "xm_kernels.cuh"

namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned char* host = nullptr;  // pinned: [plan copy | control block readback]
    void* scratch = nullptr;
    uint64_t bytes = 0;
    int64_t tag = 0;
    uint64_t seq = 0;  // admission order
    bool busy = false;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr size_t kHostPlan = 0;
constexpr size_t kHostCtl = (sizeof(XmPlanDev) + 255) & ~size_t(255);
constexpr size_t kHostBytes = kHostCtl + xm::CTL_WORDS * sizeof(unsigned long long);

// scratch layout of one query (same pieces as a graph handle's scratch)
struct Layout {
    size_t nodes, chunks, l1, e, sums, ctl, plan, total;
    int64_t cmax, emax, n_block_sums;
};

Layout layout_for(int32_t n, int64_t m) {
    Layout L;
    L.cmax = xm::chunk_capacity(n, m);
    L.emax = std::max<int64_t>(m, 1);
    L.n_block_sums = (std::max<int64_t>(std::max<int64_t>((int64_t)n + 1, L.cmax + 1), L.emax + 1) +
                      xm::SCAN_TILE - 1) / xm::SCAN_TILE;
    L.nodes = align256(((size_t)n + 1) * sizeof(int32_t));
    L.chunks = align256((size_t)(L.cmax + 1) * sizeof(int32_t));
    L.l1 = align256((size_t)L.emax * sizeof(int32_t));
    L.e = align256((size_t)(L.emax + 1) * sizeof(int32_t));
    L.sums = align256((size_t)L.n_block_sums * sizeof(int64_t));
    L.ctl = align256(xm::CTL_WORDS * sizeof(unsigned long long));
    L.plan = align256(sizeof(XmPlanDev));
    L.total = 2 * L.nodes + L.chunks + 2 * L.l1 + L.e + L.sums + L.ctl + L.plan;
    return L;
}

}  // namespace

struct xm_server_s {
    int device = 0;
    std::vector<xm_graph> graphs;
    std::vector<Slot> slots;
    uint64_t budget = 0;
    uint64_t in_flight = 0;
    uint64_t next_seq = 0;
};

namespace xm {
namespace {

int fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA;
}

void destroy(xm_server_s* s) {
    if (!s) return;
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.host) cudaFreeHost(sl.host);
    }
    delete s;
}

}  // namespace
}  // namespace xm

using namespace xm;

extern "C" {

uint64_t xm_query_bytes(xm_graph g, xm_plan p) {
    if (!g || !p) return 0;
    return layout_for(g->n, g->m).total;
}

int xm_server_create(int32_t ng, const xm_graph* graphs, int32_t nslots, uint64_t mem_budget_bytes, xm_server* out) {
    if (!out || ng < 1 || !graphs || nslots < 1 || nslots > 256) {
        set_error("bad server arguments");
        return XM_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e, "cudaGetDevice");
    xm_server_s* s = new xm_server_s();
    s->device = dev;
    s->budget = mem_budget_bytes;
    for (int i = 0; i < ng; i++) {
        if (!graphs[i] || graphs[i]->device != dev) {
            delete s;
            set_error("NULL graph or graph on another device");
            return XM_EINVAL;
        }
        s->graphs.push_back(graphs[i]);
    }
    s->slots.resize(nslots);
    for (Slot& sl : s->slots) {
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.host, kHostBytes);
        if (e != cudaSuccess) {
            int rc = fail(e, "server slot set-up");
            destroy(s);
            return rc;
        }
    }
    *out = s;
    return XM_OK;
}

int xm_server_submit(xm_server s, xm_plan p, int32_t graph_index, int64_t tag, int32_t* admitted) {
    if (!s || !p || !admitted) { set_error("NULL argument"); return XM_EINVAL; }
    *admitted = 0;
    if (graph_index < 0 || graph_index >= (int32_t)s->graphs.size()) { set_error("graph index out of range"); return XM_EINVAL; }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e, "cudaGetDevice");
    if (dev != s->device) { set_error("server lives on another device than the current one"); return XM_EINVAL; }
    const xm_graph g = s->graphs[graph_index];
    const Layout L = layout_for(g->n, g->m);
    if (L.total > s->budget) { set_error("query needs more scratch than the whole memory budget"); return XM_EINVAL; }
    Slot* sl = nullptr;
    for (Slot& c : s->slots)
        if (!c.busy) { sl = &c; break; }
    if (!sl || s->in_flight + L.total > s->budget) return XM_OK;  // not now: no slot or memory
    e = dev_alloc_async(&sl->scratch, L.total, sl->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return XM_OK;  // the pool could not serve it now: retry later
    }
    unsigned char* q = static_cast<unsigned char*>(sl->scratch);
    RunArgs a{};
    a.g = {g->d_out_off, g->d_out_adj, g->d_in_off, g->d_in_adj, g->n,
           g->d_out_hoff, g->d_out_htab, g->d_in_hoff, g->d_in_htab};
    a.root_chunks = reinterpret_cast<int32_t*>(q); q += L.nodes;
    a.chunk_cnt = reinterpret_cast<int32_t*>(q); q += L.chunks;
    a.l1set = reinterpret_cast<int32_t*>(q); q += L.l1;
    a.l1root = reinterpret_cast<int32_t*>(q); q += L.l1;
    a.units = reinterpret_cast<int32_t*>(q); q += L.nodes;
    a.e_units = reinterpret_cast<int32_t*>(q); q += L.e;
    a.emax = (int32_t)L.emax;
    a.l2_units = use_l2_units(p->plan.dev, true) ? 1 : 0;
    a.leaf_kind = a.l2_units ? 0 : leaf_closed_form_kind(p->plan.dev);
    a.block_sums = reinterpret_cast<int64_t*>(q); q += L.sums;
    a.ctl = reinterpret_cast<unsigned long long*>(q); q += L.ctl;
    XmPlanDev* plan_dev = reinterpret_cast<XmPlanDev*>(q);
    a.n_block_sums = L.n_block_sums;
    a.cmax = (int32_t)L.cmax;
    a.r_lo = 0;
    a.r_hi = g->n;
    a.root_list = nullptr;
    a.n_idx = g->n;
    a.unit = p->tuning.unit;
    a.window = p->tuning.window;
    a.budget_ns = (unsigned long long)p->tuning.budget_ms * 1000000ull;
    a.merge_ratio = p->tuning.merge_ratio;
    memcpy(sl->host + kHostPlan, &p->plan.dev, sizeof(XmPlanDev));
    e = cudaMemsetAsync(a.ctl, 0, CTL_WORDS * sizeof(unsigned long long), sl->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(plan_dev, sl->host + kHostPlan, sizeof(XmPlanDev), cudaMemcpyHostToDevice, sl->stream);
    if (e == cudaSuccess)
        e = launch_match(MODE_COUNT, p->plan.dev, plan_dev, a, p->tuning.warps_per_block, p->tuning.blocks_per_sm,
                         sl->stream, nullptr);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl->host + kHostCtl, a.ctl, CTL_WORDS * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, sl->stream);
    if (e == cudaSuccess) e = dev_free_async(sl->scratch, sl->stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl->done, sl->stream);
    if (e != cudaSuccess) return fail(e, "query launch");
    sl->busy = true;
    sl->bytes = L.total;
    sl->tag = tag;
    sl->seq = s->next_seq++;
    s->in_flight += L.total;
    *admitted = 1;
    return XM_OK;
}

int xm_server_poll(xm_server s, int32_t wait, int32_t max_results, int64_t* tags, uint64_t* counts, int32_t* status,
                   int32_t* n_done) {
    if (!s || !n_done || max_results < 0 || (max_results > 0 && (!tags || !counts || !status))) {
        set_error("bad poll arguments");
        return XM_EINVAL;
    }
    *n_done = 0;
    if (wait) {
        // block until the oldest query in flight has finished
        Slot* oldest = nullptr;
        for (Slot& c : s->slots)
            if (c.busy && (!oldest || c.seq < oldest->seq)) oldest = &c;
        if (oldest) {
            cudaError_t e = cudaEventSynchronize(oldest->done);
            if (e != cudaSuccess) return fail(e, "query execution");
        }
    }
    for (Slot& c : s->slots) {
        if (!c.busy || *n_done >= max_results) continue;
        cudaError_t e = cudaEventQuery(c.done);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) return fail(e, "query execution");
        const unsigned long long* ctl = reinterpret_cast<const unsigned long long*>(c.host + kHostCtl);
        const int i = (*n_done)++;
        tags[i] = c.tag;
        counts[2 * i] = ctl[CTL_COUNT_LO];
        counts[2 * i + 1] = ctl[CTL_COUNT_HI];
        status[i] = (ctl[CTL_STATUS] & STATUS_TIMEOUT) ? XM_ETIMEOUT : ctl[CTL_STATUS] ? XM_EINVAL : XM_OK;
        c.busy = false;
        s->in_flight -= c.bytes;
        c.bytes = 0;
    }
    return XM_OK;
}

int xm_server_info(xm_server s, int32_t* busy_slots, uint64_t* bytes_in_flight) {
    if (!s) { set_error("NULL server"); return XM_EINVAL; }
    int b = 0;
    for (const Slot& c : s->slots) b += c.busy;
    if (busy_slots) *busy_slots = b;
    if (bytes_in_flight) *bytes_in_flight = s->in_flight;
    return XM_OK;
}

void xm_server_free(xm_server s) { destroy(s); }

}  // extern "C"
