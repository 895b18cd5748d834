// C ABI of the matcher library: graph loading, pattern compilation, and the
// count / enumerate entry points declared in include/xm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <new>
#include <string>
#include <vector>

#include "xm_internal.h"
#include "xm_kernels.cuh"

namespace xm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// ---------------------------------------------- device memory, fault hooks
// Injected faults: the countdown-th next device allocation (or pattern
// compile) fails; 0 = none. Set by xm_fault_inject or, when the library
// loads, by the environment variable XM_FAULT ("alloc:N", "compile:N",
// comma-separated).
static std::mutex g_mem_mu;
static std::unordered_map<void*, size_t> g_live;
static uint64_t g_live_bytes = 0;
static long long g_alloc_countdown = 0, g_compile_countdown = 0;

static int parse_fault(const char* spec) {
    if (!spec || !*spec) return XM_EINVAL;
    std::string s(spec);
    long long a = 0, c = 0;
    size_t i = 0;
    while (i < s.size()) {
        size_t j = s.find(',', i);
        if (j == std::string::npos) j = s.size();
        const std::string item = s.substr(i, j - i);
        const size_t colon = item.find(':');
        const std::string kind = item.substr(0, colon);
        long long nth = 0;
        if (colon != std::string::npos) {
            char* end = nullptr;
            nth = std::strtoll(item.c_str() + colon + 1, &end, 10);
            if (!end || *end || nth < 1) return XM_EINVAL;
        }
        if (kind == "alloc" && nth) a = nth;
        else if (kind == "compile" && nth) c = nth;
        else if (kind == "none" && colon == std::string::npos) a = c = 0;
        else return XM_EINVAL;
        i = j + 1;
    }
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_alloc_countdown = a;
    g_compile_countdown = c;
    return XM_OK;
}

static const int g_env_fault = []() {
    const char* e = std::getenv("XM_FAULT");
    return e ? parse_fault(e) : XM_OK;
}();

static bool take_fault(long long& countdown) {
    if (countdown <= 0) return false;
    return --countdown == 0;
}

bool compile_fault() {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    return take_fault(g_compile_countdown);
}

cudaError_t dev_alloc_raw(void** p, size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        if (take_fault(g_alloc_countdown)) return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        g_live[*p] = bytes;
        g_live_bytes += bytes;
    }
    return e;
}

cudaError_t dev_alloc_async_raw(void** p, size_t bytes, cudaStream_t stream) {
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        if (take_fault(g_alloc_countdown)) return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, stream);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        g_live[*p] = bytes;
        g_live_bytes += bytes;
    }
    return e;
}

static void forget(void* p) {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    auto it = g_live.find(p);
    if (it != g_live.end()) {
        g_live_bytes -= it->second;
        g_live.erase(it);
    }
}

void dev_free(void* p) {
    if (!p) return;
    forget(p);
    cudaFree(p);
}

cudaError_t dev_free_async(void* p, cudaStream_t stream) {
    if (!p) return cudaSuccess;
    forget(p);
    return cudaFreeAsync(p, stream);
}

static int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return XM_ECUDA;
}

#define XM_CUDA(call, what)                        \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

static const xm_tuning kDefaultTuning = {512, 32, 8, 0, 0, MERGE_RATIO_DEFAULT};

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static void free_graph(xm_graph_s* g) {
    if (!g) return;
    dev_free(g->d_out_off);
    dev_free(g->d_out_adj);
    dev_free(g->d_in_off);
    dev_free(g->d_in_adj);
    dev_free(g->d_out_hoff);
    dev_free(g->d_out_htab);
    dev_free(g->d_in_hoff);
    dev_free(g->d_in_htab);
    dev_free(g->d_roots);
    dev_free(g->d_root_chunks);
    dev_free(g->d_chunk_cnt);
    dev_free(g->d_l1set);
    dev_free(g->d_units);
    dev_free(g->d_l1root);
    dev_free(g->d_e_units);
    dev_free(g->d_block_sums);
    dev_free(g->d_ctl);
    dev_free(g->d_root_counts);
    for (auto& e : g->ev)
        if (e) cudaEventDestroy(e);
    delete g;
}

// control block: CTL_WORDS words, then a device copy of the plan
static size_t ctl_bytes() { return CTL_WORDS * sizeof(unsigned long long) + ((sizeof(XmPlanDev) + 255) & ~size_t(255)); }

static XmPlanDev* ctl_plan(xm_graph_s* g) {
    return reinterpret_cast<XmPlanDev*>(reinterpret_cast<unsigned char*>(g->d_ctl) + CTL_WORDS * sizeof(unsigned long long));
}

// One matching pass of plan P over start nodes [r_lo, r_hi) (or the staged
// root list). With root_counts (count mode) the counts go per start node
// to root_counts[2 v .. 2 v + 1] instead of *lo, *hi.
static int run_plan(xm_graph g, const Plan& P, const xm_tuning& t, int mode, int64_t r_lo, int64_t r_hi,
                    int32_t* out, uint64_t capacity, uint64_t* lo, uint64_t* hi, xm_stats* stats, uint64_t* written,
                    cudaStream_t stream, const int32_t* roots = nullptr, int64_t nroots = 0,
                    unsigned long long* root_counts = nullptr) {
    if (mode == MODE_EMIT && capacity > 0 && !out) { set_error("NULL output buffer"); return XM_EINVAL; }
    int cur = -1;
    XM_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != g->device) { set_error("graph lives on another device than the current one"); return XM_EINVAL; }
    r_lo = std::max<int64_t>(r_lo, 0);
    r_hi = std::min<int64_t>(r_hi, g->n);
    RunArgs a;
    a.g = {g->d_out_off, g->d_out_adj, g->d_in_off, g->d_in_adj, g->n,
           g->d_out_hoff, g->d_out_htab, g->d_in_hoff, g->d_in_htab};
    a.root_chunks = g->d_root_chunks;
    a.chunk_cnt = g->d_chunk_cnt;
    a.l1set = g->d_l1set;
    a.units = g->d_units;
    a.l1root = g->d_l1root;
    a.e_units = g->d_e_units;
    a.emax = (int32_t)std::max<int64_t>(g->m, 1);
    a.l2_units = use_l2_units(P.dev, mode != MODE_EMIT) ? 1 : 0;
    a.leaf_kind = a.l2_units ? 0 : leaf_closed_form_kind(P.dev);
    a.block_sums = g->d_block_sums;
    a.n_block_sums = g->n_block_sums;
    a.ctl = g->d_ctl;
    a.cmax = (int32_t)g->cmax;
    a.r_lo = (int32_t)std::min<int64_t>(r_lo, g->n);
    a.r_hi = (int32_t)std::max<int64_t>(r_hi, a.r_lo);
    a.root_list = roots;
    a.n_idx = roots ? (int32_t)nroots : g->n;
    a.unit = t.unit;
    a.window = t.window;
    a.out = out;
    a.capacity = capacity;
    a.budget_ns = (unsigned long long)t.budget_ms * 1000000ull;
    a.root_counts = root_counts;
    a.merge_ratio = t.merge_ratio;
  retry:
    XM_CUDA(cudaMemsetAsync(g->d_ctl, 0, CTL_WORDS * sizeof(unsigned long long), stream), "cudaMemsetAsync");
    XM_CUDA(cudaMemcpyAsync(ctl_plan(g), &P.dev, sizeof(XmPlanDev), cudaMemcpyHostToDevice, stream),
            "plan upload");
    cudaError_t e = launch_match(mode, P.dev, ctl_plan(g), a, t.warps_per_block, t.blocks_per_sm, stream, g->ev);
    if (e != cudaSuccess) return cuda_fail(e, "matcher launch");
    g->timed = true;
    unsigned long long ctl[CTL_WORDS];
    XM_CUDA(cudaMemcpyAsync(ctl, g->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost, stream), "result readback");
    XM_CUDA(cudaStreamSynchronize(stream), "matcher execution");
    {
        float a = 0.f, b = 0.f;
        XM_CUDA(cudaEventElapsedTime(&a, g->ev[0], g->ev[1]), "cudaEventElapsedTime");
        XM_CUDA(cudaEventElapsedTime(&b, g->ev[1], g->ev[2]), "cudaEventElapsedTime");
        g->sum_prep_ms += a;
        g->sum_match_ms += b;
    }
    if (ctl[CTL_STATUS] & STATUS_TIMEOUT) { set_error("time budget of the matcher exceeded; no count"); return XM_ETIMEOUT; }
    if ((ctl[CTL_STATUS] & STATUS_OVERFLOW) && a.unit <= (1 << 20)) {
        // more work units than an int32 index space holds: the matcher
        // walked nothing (the per-node counters are untouched); again with
        // eight times larger units
        a.unit *= 8;
        goto retry;
    }
    if (ctl[CTL_STATUS]) { set_error("work-unit count exceeds 2^31-1 (raise the unit size)"); return XM_EINVAL; }
    if (mode == MODE_EMIT) {
        *lo = ctl[CTL_EMIT];
        *hi = 0;
        if (written) *written = std::min<uint64_t>(ctl[CTL_EMIT], capacity);
    } else {
        *lo = ctl[CTL_COUNT_LO];
        *hi = ctl[CTL_COUNT_HI];
    }
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->alg_bytes = ctl[CTL_STATS + 0];
        stats->extensions = ctl[CTL_STATS + 1];
        stats->set_ops = ctl[CTL_STATS + 2];
        stats->units = ctl[CTL_STATS + 3];
        stats->leaf_elems = ctl[CTL_STATS + 4];
        // the first-level pass, plus its start-node degree checks: 16 B per
        // node in range
        stats->l1_bytes = ctl[CTL_STATS + 5] + 16ull * (uint64_t)(roots ? nroots : (int64_t)(a.r_hi - a.r_lo));
        stats->touched_bytes = ctl[CTL_STATS + 6];
        const unsigned long long t0 = ctl[CTL_W_START];
        if (t0 && ctl[CTL_W_COUNT]) {
            stats->warp_exit_first_ns = ~ctl[CTL_W_FIRST] - t0;
            stats->warp_exit_mean_ns = ctl[CTL_W_SUM] / ctl[CTL_W_COUNT];
            stats->warp_exit_last_ns = ctl[CTL_W_LAST] - t0;
        }
    }
    if (mode == MODE_EMIT && ctl[CTL_EMIT] > capacity) {
        set_error("enumeration buffer too small");
        return XM_EOVERFLOW;
    }
    return XM_OK;
}

// Start of a public call: its passes' event times are summed from zero.
static void begin_call(xm_graph g) {
    if (!g) return;
    g->sum_prep_ms = 0.f;
    g->sum_match_ms = 0.f;
}

static int run(xm_graph g, xm_plan p, int mode, int64_t r_lo, int64_t r_hi, int32_t* out, uint64_t capacity,
               uint64_t* lo, uint64_t* hi, xm_stats* stats, uint64_t* written, cudaStream_t stream,
               const int32_t* roots = nullptr, int64_t nroots = 0) {
    if (!g || !p || !lo || !hi) { set_error("NULL argument"); return XM_EINVAL; }
    return run_plan(g, p->plan, p->tuning, mode, r_lo, r_hi, out, capacity, lo, hi, stats, written, stream, roots,
                    nroots);
}

typedef unsigned __int128 u128;

// The graph's per-node 128-bit counters (split parts, per-root counts):
// at least `words` words, grown on demand.
static int ensure_root_counts(xm_graph g, size_t words) {
    if (g->root_count_words >= words) return XM_OK;
    dev_free(g->d_root_counts);
    g->d_root_counts = nullptr;
    g->root_count_words = 0;
    cudaError_t e = dev_alloc(&g->d_root_counts, words * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("per-node counters: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA;
    }
    g->root_count_words = words;
    return XM_OK;
}

// Whole-graph count of plan P (matches, or embeddings with XM_EMBEDDINGS),
// through its cut-vertex decomposition when it has one:
//   emb(P) = part_factor * sum_v prod_i m_i(v) - sum_j mult_j * emb(Q_j)
// with m_i(v) the rooted matches of part i at node v and Q_j the quotient
// patterns (counted the same way, recursively).
static int count_plan(xm_graph g, const Plan& P, const xm_tuning& t, u128& result, cudaStream_t stream) {
    const Decomp* d = P.decomp.get();
    if (!d) {
        uint64_t lo = 0, hi = 0;
        int rc = run_plan(g, P, t, MODE_COUNT, 0, INT32_MAX, nullptr, 0, &lo, &hi, nullptr, nullptr, stream);
        result = ((u128)hi << 64) | lo;
        return rc;
    }
    const int nparts = (int)d->parts.size();
    const size_t words = (size_t)nparts * 2 * (size_t)g->n + 2;
    int rc0 = ensure_root_counts(g, words);
    if (rc0) return rc0;
    unsigned long long* cnt = g->d_root_counts;
    unsigned long long* sum = cnt + (size_t)nparts * 2 * g->n;
    XM_CUDA(cudaMemsetAsync(cnt, 0, (size_t)nparts * 2 * g->n * sizeof(unsigned long long), stream), "memset");
    for (int i = 0; i < nparts; i++) {
        uint64_t lo = 0, hi = 0;
        int rc = run_plan(g, d->parts[i], t, MODE_COUNT, 0, INT32_MAX, nullptr, 0, &lo, &hi, nullptr, nullptr, stream,
                          nullptr, 0, cnt + (size_t)i * 2 * g->n);
        if (rc) return rc;
    }
    cudaError_t e = launch_root_product(cnt, nparts, g->n, sum, stream);
    if (e != cudaSuccess) return cuda_fail(e, "part products");
    unsigned long long s2[2];
    XM_CUDA(cudaMemcpyAsync(s2, sum, sizeof s2, cudaMemcpyDeviceToHost, stream), "product readback");
    XM_CUDA(cudaStreamSynchronize(stream), "part products");
    u128 emb = (((u128)s2[1] << 64) | s2[0]) * (u128)d->part_factor;
    for (size_t j = 0; j < d->quots.size(); j++) {
        u128 q = 0;
        int rc = count_plan(g, d->quots[j], t, q, stream);
        if (rc) return rc;
        // quotient plans count matches: embeddings = matches x |Aut(Q)|
        emb -= q * (u128)d->quots[j].aut_size * (u128)d->quot_mult[j];
    }
    result = (P.flags & XM_EMBEDDINGS) ? emb : emb / (u128)P.aut_size;
    return XM_OK;
}

// Adds the counters of one pass to a running total (load-balance times: the
// latest pass's).
static void add_stats(xm_stats& acc, const xm_stats& s) {
    acc.alg_bytes += s.alg_bytes;
    acc.extensions += s.extensions;
    acc.set_ops += s.set_ops;
    acc.units += s.units;
    acc.leaf_elems += s.leaf_elems;
    acc.l1_bytes += s.l1_bytes;
    acc.touched_bytes += s.touched_bytes;
    acc.warp_exit_first_ns = s.warp_exit_first_ns;
    acc.warp_exit_mean_ns = s.warp_exit_mean_ns;
    acc.warp_exit_last_ns = s.warp_exit_last_ns;
}

// Whether counts of P over a subset of its start nodes go through its
// cut-vertex decomposition (Decomp::rooted).
static bool rooted_split(const Plan& P) { return P.decomp && P.decomp->rooted; }

// Count (MODE_COUNT) or instrumented count (MODE_STATS, *stats summed over
// the passes) of plan P over start nodes [r_lo, r_hi) or the staged root
// list, through the cut-vertex decomposition rooted at the start vertex
// (rooted_split(P)): per start-node part counts, their product sum (one
// kernel), minus the rooted quotient counts over the same start nodes.
static int count_split_sub(xm_graph g, const Plan& P, const xm_tuning& t, int mode, int64_t r_lo, int64_t r_hi,
                           const int32_t* roots, int64_t nroots, u128& result, xm_stats* stats, cudaStream_t stream) {
    const Decomp* d = P.decomp.get();
    const int nparts = (int)d->parts.size();
    const int64_t N = roots ? nroots : (int64_t)g->n;  // counter index space
    const size_t words = (size_t)nparts * 2 * (size_t)N + 2;
    int rc = ensure_root_counts(g, words);
    if (rc) return rc;
    unsigned long long* cnt = g->d_root_counts;
    unsigned long long* sum = cnt + (size_t)nparts * 2 * N;
    XM_CUDA(cudaMemsetAsync(cnt, 0, words * sizeof(unsigned long long), stream), "memset");
    if (stats) memset(stats, 0, sizeof *stats);
    xm_stats st{};
    for (int i = 0; i < nparts; i++) {
        uint64_t lo = 0, hi = 0;
        // per-node counters need count mode; the stats pass of a part runs
        // after it over the same start nodes
        rc = run_plan(g, d->parts[i], t, MODE_COUNT, r_lo, r_hi, nullptr, 0, &lo, &hi, nullptr, nullptr, stream,
                      roots, nroots, cnt + (size_t)i * 2 * N);
        if (rc) return rc;
        if (mode == MODE_STATS) {
            rc = run_plan(g, d->parts[i], t, MODE_STATS, r_lo, r_hi, nullptr, 0, &lo, &hi, &st, nullptr, stream,
                          roots, nroots);
            if (rc) return rc;
            add_stats(*stats, st);
        }
    }
    cudaError_t e = launch_root_product(cnt, nparts, (int32_t)N, sum, stream);
    if (e != cudaSuccess) return cuda_fail(e, "part products");
    unsigned long long s2[2];
    XM_CUDA(cudaMemcpyAsync(s2, sum, sizeof s2, cudaMemcpyDeviceToHost, stream), "product readback");
    XM_CUDA(cudaStreamSynchronize(stream), "part products");
    u128 emb = (((u128)s2[1] << 64) | s2[0]) * (u128)d->part_factor;
    for (size_t j = 0; j < d->rquots.size(); j++) {
        uint64_t lo = 0, hi = 0;
        rc = run_plan(g, d->rquots[j], t, mode, r_lo, r_hi, nullptr, 0, &lo, &hi, mode == MODE_STATS ? &st : nullptr,
                      nullptr, stream, roots, nroots);
        if (rc) return rc;
        if (mode == MODE_STATS) add_stats(*stats, st);
        const u128 q = ((u128)hi << 64) | lo;
        emb -= q * (u128)d->rquots[j].stab_size * (u128)d->quot_mult[j];
    }
    result = (P.flags & XM_EMBEDDINGS) ? emb : emb / (u128)P.aut_size;
    return XM_OK;
}

// Count or instrumented count of plan p over a start-node range or the staged
// root list: the cut-vertex decomposition when it applies, else one pass.
static int count_sub(xm_graph g, xm_plan p, int mode, int64_t r_lo, int64_t r_hi, const int32_t* roots,
                     int64_t nroots, uint64_t* lo, uint64_t* hi, xm_stats* stats, cudaStream_t stream) {
    if (!rooted_split(p->plan))
        return run(g, p, mode, r_lo, r_hi, nullptr, 0, lo, hi, stats, nullptr, stream, roots, nroots);
    u128 r = 0;
    int rc = count_split_sub(g, p->plan, p->tuning, mode, r_lo, r_hi, roots, nroots, r, stats, stream);
    if (rc) return rc;
    *lo = (uint64_t)r;
    *hi = (uint64_t)(r >> 64);
    return XM_OK;
}

}  // namespace xm

using namespace xm;

extern "C" {

const char* xm_strerror(int status) {
    switch (status) {
        case XM_OK: return "XM_OK";
        case XM_EINVAL: return "XM_EINVAL";
        case XM_ENOMEM: return "XM_ENOMEM";
        case XM_EOVERFLOW: return "XM_EOVERFLOW";
        case XM_ECUDA: return "XM_ECUDA";
        case XM_ETIMEOUT: return "XM_ETIMEOUT";
        case XM_EBUSY: return "XM_EBUSY";
        default: return "XM_UNKNOWN";
    }
}

const char* xm_last_error(void) { return g_last_error.c_str(); }

int xm_version(void) { return 200; }

int xm_fault_inject(const char* spec) {
    int rc = parse_fault(spec);
    if (rc) set_error("fault spec must be \"none\" or \"alloc:N\" / \"compile:N\" (N >= 1), comma-separated");
    return rc;
}

uint64_t xm_device_bytes_live(void) {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    return g_live_bytes;
}

int xm_load_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int flags, void* stream_,
                  xm_graph* out) {
    if (!out) { set_error("NULL output handle"); return XM_EINVAL; }
    if (flags != 0) { set_error("flags must be 0"); return XM_EINVAL; }
    if (n < 1 || m < 0) { set_error("n must be >= 1 and m >= 0"); return XM_EINVAL; }
    if (m > 0 && (!src || !dst)) { set_error("NULL arc arrays"); return XM_EINVAL; }
    if (m >= (int64_t)INT32_MAX) { set_error("fewer than 2^31 input arcs are supported"); return XM_EINVAL; }
    cudaStream_t stream = (cudaStream_t)stream_;
    xm_graph_s* g = new (std::nothrow) xm_graph_s();
    if (!g) { set_error("host allocation failed"); return XM_ENOMEM; }
    g->n = n;
    // temporaries of the build, released before returning
    int32_t *d_src = nullptr, *d_dst = nullptr, *ints = nullptr;
    unsigned long long *k0 = nullptr, *k1 = nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(stream);
        dev_free(d_src);
        dev_free(d_dst);
        dev_free(ints);
        dev_free(k0);
        dev_free(k1);
    };
    auto fail = [&](cudaError_t e, const char* what) {
        cudaGetLastError();
        release();
        free_graph(g);
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA;
    };
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) return fail(e, "cudaGetDevice");
    // host arcs are uploaded; arc ids are checked on the device as the
    // keys are packed
    const bool on_device = m > 0 && is_device_ptr(src) && is_device_ptr(dst);
    // scan partials and the control block first: the build's scans use them
    const int64_t cmax_in = chunk_capacity(n, m);
    const int64_t iscratch = csr_int_scratch(m, n);
    g->n_block_sums = (std::max<int64_t>(std::max<int64_t>((int64_t)n + 1, cmax_in + 1), std::max(m + 2, iscratch)) +
                       SCAN_TILE - 1) /
                      SCAN_TILE;
    if ((e = dev_alloc(&g->d_block_sums, g->n_block_sums * sizeof(int64_t))) != cudaSuccess)
        return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_ctl, ctl_bytes())) != cudaSuccess) return fail(e, "device allocation");
    if ((e = cudaMemsetAsync(g->d_ctl, 0, ctl_bytes(), stream)) != cudaSuccess) return fail(e, "memset");
    RunArgs sa{};
    sa.block_sums = g->d_block_sums;
    sa.n_block_sums = g->n_block_sums;
    sa.ctl = g->d_ctl;
    if ((e = dev_alloc(&ints, (size_t)iscratch * sizeof(int32_t))) != cudaSuccess) return fail(e, "device allocation");
    unsigned long long* keys = nullptr;
    int64_t mm = 0;
    if (m > 0) {
        const int32_t *s = src, *d = dst;
        if (!on_device) {
            if ((e = dev_alloc(&d_src, (size_t)m * sizeof(int32_t))) != cudaSuccess) return fail(e, "device allocation");
            if ((e = dev_alloc(&d_dst, (size_t)m * sizeof(int32_t))) != cudaSuccess) return fail(e, "device allocation");
            if ((e = cudaMemcpyAsync(d_src, src, (size_t)m * sizeof(int32_t), cudaMemcpyDefault, stream)) != cudaSuccess)
                return fail(e, "arc upload");
            if ((e = cudaMemcpyAsync(d_dst, dst, (size_t)m * sizeof(int32_t), cudaMemcpyDefault, stream)) != cudaSuccess)
                return fail(e, "arc upload");
            s = d_src;
            d = d_dst;
        }
        if ((e = dev_alloc(&k0, (size_t)m * sizeof(unsigned long long))) != cudaSuccess)
            return fail(e, "device allocation");
        if ((e = dev_alloc(&k1, (size_t)m * sizeof(unsigned long long))) != cudaSuccess)
            return fail(e, "device allocation");
        if ((e = csr_sort_unique(n, m, s, d, k0, k1, ints, sa, &keys, &mm, stream)) != cudaSuccess)
            return fail(e, "CSR sort");
        unsigned long long status = 0;
        if ((e = cudaMemcpy(&status, g->d_ctl + CTL_STATUS, sizeof status, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return fail(e, "status readback");
        if (status & STATUS_BAD_ID) {
            release();
            free_graph(g);
            set_error("arc endpoint outside [0, n)");
            return XM_EINVAL;
        }
    }
    if ((int64_t)n + mm >= (int64_t)INT32_MAX) {
        release();
        free_graph(g);
        set_error("n + arcs must stay below 2^31");
        return XM_EINVAL;
    }
    g->m = mm;
    const size_t off_b = ((size_t)n + 1) * sizeof(int32_t);
    const size_t adj_b = (size_t)std::max<int64_t>(mm, 1) * sizeof(int32_t);
    g->cmax = chunk_capacity(n, mm);
    if ((e = dev_alloc(&g->d_out_off, off_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_in_off, off_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_out_adj, adj_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_in_adj, adj_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = csr_emit(n, keys, keys == k0 ? k1 : k0, mm, ints, sa, g->d_out_off, g->d_out_adj, g->d_in_off,
                      g->d_in_adj, stream)) != cudaSuccess)
        return fail(e, "CSR emit");
    // scratch of the matching pipeline
    if ((e = dev_alloc(&g->d_root_chunks, off_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_chunk_cnt, (size_t)(g->cmax + 1) * sizeof(int32_t))) != cudaSuccess)
        return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_l1set, adj_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_units, off_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_l1root, adj_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_e_units, adj_b + sizeof(int32_t))) != cudaSuccess) return fail(e, "device allocation");
    for (auto& ev : g->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(e, "cudaEventCreate");
    // hash index: per-node table offsets (device scan), then the tables
    const size_t hoff_b = ((size_t)n + 1) * sizeof(int64_t);
    if ((e = dev_alloc(&g->d_out_hoff, hoff_b)) != cudaSuccess) return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_in_hoff, hoff_b)) != cudaSuccess) return fail(e, "device allocation");
    int64_t slots[2] = {0, 0};
    if ((e = hash_offsets(g->d_out_off, n, ints, sa, g->d_out_hoff, stream)) != cudaSuccess)
        return fail(e, "hash offsets");
    if ((e = cudaMemcpyAsync(&slots[0], g->d_out_hoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream)) !=
        cudaSuccess)
        return fail(e, "hash offsets");
    if ((e = hash_offsets(g->d_in_off, n, ints, sa, g->d_in_hoff, stream)) != cudaSuccess)
        return fail(e, "hash offsets");
    if ((e = cudaMemcpyAsync(&slots[1], g->d_in_hoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream)) !=
        cudaSuccess)
        return fail(e, "hash offsets");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return fail(e, "graph build");
    g->hash_slots = slots[0] + slots[1];
    if ((e = dev_alloc(&g->d_out_htab, (size_t)std::max<int64_t>(slots[0], 1) * sizeof(int32_t))) != cudaSuccess)
        return fail(e, "device allocation");
    if ((e = dev_alloc(&g->d_in_htab, (size_t)std::max<int64_t>(slots[1], 1) * sizeof(int32_t))) != cudaSuccess)
        return fail(e, "device allocation");
    if (slots[0] && (e = cudaMemsetAsync(g->d_out_htab, 0xFF, (size_t)slots[0] * sizeof(int32_t), stream)) != cudaSuccess)
        return fail(e, "memset");
    if (slots[1] && (e = cudaMemsetAsync(g->d_in_htab, 0xFF, (size_t)slots[1] * sizeof(int32_t), stream)) != cudaSuccess)
        return fail(e, "memset");
    if ((e = build_hash_index(g->d_out_off, g->d_out_adj, g->d_out_hoff, g->d_out_htab, n, stream)) != cudaSuccess)
        return fail(e, "hash index");
    if ((e = build_hash_index(g->d_in_off, g->d_in_adj, g->d_in_hoff, g->d_in_htab, n, stream)) != cudaSuccess)
        return fail(e, "hash index");
    release();
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "graph build");
    *out = g;
    return XM_OK;
}

int xm_graph_info(xm_graph g, int32_t* n, int64_t* m) {
    if (!g) { set_error("NULL graph"); return XM_EINVAL; }
    if (n) *n = g->n;
    if (m) *m = g->m;
    return XM_OK;
}

int xm_graph_csr(xm_graph g, const int32_t** out_off, const int32_t** out_adj, const int32_t** in_off,
                 const int32_t** in_adj) {
    if (!g) { set_error("NULL graph"); return XM_EINVAL; }
    if (out_off) *out_off = g->d_out_off;
    if (out_adj) *out_adj = g->d_out_adj;
    if (in_off) *in_off = g->d_in_off;
    if (in_adj) *in_adj = g->d_in_adj;
    return XM_OK;
}

void xm_graph_free(xm_graph g) { free_graph(g); }

int xm_graph_last_timing(xm_graph g, float* prep_ms, float* match_ms) {
    if (!g || !g->timed) { set_error("no timed call on this graph yet"); return XM_EINVAL; }
    // every pass of the last call synchronised its stream before returning,
    // so the sums are complete
    if (prep_ms) *prep_ms = g->sum_prep_ms;
    if (match_ms) *match_ms = g->sum_match_ms;
    return XM_OK;
}

int xm_compile_pattern(int32_t k, int32_t e, const int32_t* psrc, const int32_t* pdst, int flags, xm_plan* out) {
    if (!out) { set_error("NULL output handle"); return XM_EINVAL; }
    if (compile_fault()) { set_error("injected fault: pattern compile"); return XM_ENOMEM; }
    try {
        xm_plan_s* p = new xm_plan_s();
        std::string err;
        int rc = compile_pattern(k, e, psrc, pdst, flags, p->plan, err);
        if (rc) {
            delete p;
            set_error(err);
            return rc;
        }
        p->tuning = kDefaultTuning;
        *out = p;
        return XM_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return XM_ENOMEM;
    }
}

int xm_plan_info(xm_plan p, int32_t* k, int32_t* aut_size, int32_t* n_levels, int32_t* n_reuse, int32_t* start) {
    if (!p) { set_error("NULL plan"); return XM_EINVAL; }
    if (k) *k = p->plan.k;
    if (aut_size) *aut_size = p->plan.aut_size;
    if (n_levels) *n_levels = p->plan.dev.k;
    if (n_reuse) *n_reuse = p->plan.n_reuse;
    if (start) *start = p->plan.start;
    return XM_OK;
}

int xm_plan_order(xm_plan p, int32_t* order) {
    if (!p || !order) { set_error("NULL argument"); return XM_EINVAL; }
    for (int l = 0; l < p->plan.k; l++) order[l] = p->plan.dev.order[l];
    return XM_OK;
}

static void level_record(const XmLevel& L, int32_t vertex, xm_level_info* out) {
    memset(out, 0, sizeof *out);
    out->vertex = vertex;
    out->nops = L.nops;
    for (int i = 0; i < L.nops; i++) {
        out->op_level[i] = L.op_level[i];
        out->op_dir[i] = L.op_dir[i];
    }
    out->reuse = L.reuse;
    out->reuse_ops = L.reuse_ops;
    out->dout_min = L.dout_min;
    out->din_min = L.din_min;
    out->lo_mask = L.lo_mask;
    out->hi_mask = L.hi_mask;
    out->neq_mask = L.neq_mask;
    out->ndiff = L.ndiff;
    for (int i = 0; i < L.ndiff; i++) {
        out->diff_level[i] = L.diff_level[i];
        out->diff_dir[i] = L.diff_dir[i];
    }
}

int xm_plan_level(xm_plan p, int32_t level, xm_level_info* out) {
    if (!p || !out) { set_error("NULL argument"); return XM_EINVAL; }
    if (level < 0 || level >= p->plan.k) { set_error("level out of range"); return XM_EINVAL; }
    level_record(p->plan.dev.lv[level], p->plan.dev.order[level], out);
    return XM_OK;
}

int xm_plan_product(xm_plan p, int32_t* level, int32_t* r, int32_t* kind, int32_t* n_sets) {
    if (!p) { set_error("NULL plan"); return XM_EINVAL; }
    const XmPlanDev& D = p->plan.dev;
    if (level) *level = D.prod_p;
    if (r) *r = D.prod_r;
    if (kind) *kind = D.prod_kind;
    if (n_sets) *n_sets = D.prod_nv;
    return XM_OK;
}

int xm_plan_product_set(xm_plan p, int32_t i, xm_level_info* out) {
    if (!p || !out) { set_error("NULL argument"); return XM_EINVAL; }
    if (i < 0 || i >= p->plan.dev.prod_nv) { set_error("product set index out of range"); return XM_EINVAL; }
    level_record(p->plan.dev.pv[i], -1, out);
    return XM_OK;
}

int xm_plan_split(xm_plan p, int32_t* cut, int32_t* n_parts, int32_t* n_quotients, int64_t* part_factor) {
    if (!p) { set_error("NULL plan"); return XM_EINVAL; }
    const Decomp* d = p->plan.decomp.get();
    if (cut) *cut = d ? d->cut : -1;
    if (n_parts) *n_parts = d ? (int32_t)d->parts.size() : 0;
    if (n_quotients) *n_quotients = d ? (int32_t)d->quots.size() : 0;
    if (part_factor) *part_factor = d ? d->part_factor : 1;
    return XM_OK;
}

static void pattern_out(const Plan& q, int32_t* k, int32_t* e, int32_t* psrc, int32_t* pdst) {
    if (k) *k = q.k;
    if (e) *e = q.e;
    for (int a = 0; a < q.e; a++) {
        if (psrc) psrc[a] = q.psrc[a];
        if (pdst) pdst[a] = q.pdst[a];
    }
}

int xm_plan_split_part(xm_plan p, int32_t i, int32_t* k, int32_t* e, int32_t* psrc, int32_t* pdst,
                       int32_t* vertices, int32_t* stab) {
    if (!p) { set_error("NULL plan"); return XM_EINVAL; }
    const Decomp* d = p->plan.decomp.get();
    if (!d || i < 0 || i >= (int32_t)d->parts.size()) { set_error("no such part"); return XM_EINVAL; }
    const Plan& q = d->parts[i];
    pattern_out(q, k, e, psrc, pdst);
    if (vertices)
        for (size_t j = 0; j < d->part_vertices[i].size(); j++) vertices[j] = d->part_vertices[i][j];
    if (stab) *stab = q.stab_size;
    return XM_OK;
}

int xm_plan_split_quotient(xm_plan p, int32_t i, int32_t* k, int32_t* e, int32_t* psrc, int32_t* pdst,
                           int64_t* mult) {
    if (!p) { set_error("NULL plan"); return XM_EINVAL; }
    const Decomp* d = p->plan.decomp.get();
    if (!d || i < 0 || i >= (int32_t)d->quots.size()) { set_error("no such quotient"); return XM_EINVAL; }
    pattern_out(d->quots[i], k, e, psrc, pdst);
    if (mult) *mult = d->quot_mult[i];
    return XM_OK;
}

int xm_plan_describe(xm_plan p, char* buf, int32_t cap) {
    if (!p) { set_error("NULL plan"); return -XM_EINVAL; }
    std::string s = describe_plan(p->plan);
    if (buf && cap > 0) {
        size_t nb = std::min<size_t>(s.size(), (size_t)cap - 1);
        memcpy(buf, s.data(), nb);
        buf[nb] = 0;
    }
    return (int)s.size();
}

void xm_plan_free(xm_plan p) { delete p; }

int xm_plan_set_tuning(xm_plan p, const xm_tuning* t) {
    if (!p || !t) { set_error("NULL argument"); return XM_EINVAL; }
    xm_tuning v = *t;
    if (v.window == 0) v.window = kDefaultTuning.window;
    if (v.unit == 0) v.unit = kDefaultTuning.unit;
    if (v.warps_per_block == 0) v.warps_per_block = kDefaultTuning.warps_per_block;
    if (v.window < 64 || v.window > 4096 || (v.window & 31)) { set_error("window must be a multiple of 32 in [64, 4096]"); return XM_EINVAL; }
    if (v.unit < 1 || v.unit > 65536) { set_error("unit must be in [1, 65536]"); return XM_EINVAL; }
    if (v.warps_per_block < 1 || v.warps_per_block > 16) { set_error("warps_per_block must be in [1, 16]"); return XM_EINVAL; }
    if (v.blocks_per_sm < 0 || v.blocks_per_sm > 64) { set_error("blocks_per_sm must be in [0, 64]"); return XM_EINVAL; }
    if (v.budget_ms < 0) { set_error("budget_ms must be >= 0"); return XM_EINVAL; }
    if (v.merge_ratio == 0) v.merge_ratio = MERGE_RATIO_DEFAULT;
    if (v.merge_ratio != -1 && (v.merge_ratio < 1 || v.merge_ratio > 1024)) {
        set_error("merge_ratio must be -1 or in [1, 1024] (0: default)");
        return XM_EINVAL;
    }
    p->tuning = v;
    return XM_OK;
}

int xm_plan_get_tuning(xm_plan p, xm_tuning* t) {
    if (!p || !t) { set_error("NULL argument"); return XM_EINVAL; }
    *t = p->tuning;
    return XM_OK;
}

static int tune(xm_graph g, xm_plan p, const int32_t* roots, int64_t nroots, const xm_tuning* cand, int32_t ncand,
                int32_t reps, xm_tuning* best, float* best_ms, void* stream);

int xm_plan_tune(xm_graph g, xm_plan p, const xm_tuning* cand, int32_t ncand, int32_t reps, xm_tuning* best,
                 float* best_ms, void* stream) {
    return tune(g, p, nullptr, 0, cand, ncand, reps, best, best_ms, stream);
}

int xm_plan_tune_roots(xm_graph g, xm_plan p, const int32_t* roots, int64_t nroots, const xm_tuning* cand,
                       int32_t ncand, int32_t reps, xm_tuning* best, float* best_ms, void* stream) {
    if (!roots) { set_error("NULL root list"); return XM_EINVAL; }
    return tune(g, p, roots, nroots, cand, ncand, reps, best, best_ms, stream);
}

// The autotuner: each candidate runs the count once to warm up, then `reps`
// times timed with the graph's events (first-level pass + matcher); the
// fastest candidate is kept. On the whole graph (xm_count) or a root list
// (xm_count_roots).
static int tune(xm_graph g, xm_plan p, const int32_t* roots, int64_t nroots, const xm_tuning* cand, int32_t ncand,
                int32_t reps, xm_tuning* best, float* best_ms, void* stream) {
    if (!g || !p || !cand || ncand < 1 || reps < 1) { set_error("bad tuning arguments"); return XM_EINVAL; }
    const xm_tuning keep = p->tuning;
    float best_t = -1.0f;
    xm_tuning best_c = keep;
    uint64_t want_lo = 0, want_hi = 0;
    for (int c = 0; c < ncand; c++) {
        int rc = xm_plan_set_tuning(p, &cand[c]);
        if (rc) { p->tuning = keep; return rc; }
        float t_min = -1.0f;
        for (int r = 0; r <= reps; r++) {  // the first run warms up
            uint64_t lo = 0, hi = 0;
            rc = roots ? xm_count_roots(g, p, roots, nroots, &lo, &hi, stream) : xm_count(g, p, &lo, &hi, stream);
            if (rc) { p->tuning = keep; return rc; }
            if (c == 0 && r == 0) { want_lo = lo; want_hi = hi; }
            if (lo != want_lo || hi != want_hi) {
                p->tuning = keep;
                set_error("tunings disagree on the count");
                return XM_EINVAL;
            }
            float a = 0, b = 0;
            if ((rc = xm_graph_last_timing(g, &a, &b))) { p->tuning = keep; return rc; }
            if (r > 0 && (t_min < 0 || a + b < t_min)) t_min = a + b;
        }
        if (best_t < 0 || t_min < best_t) {
            best_t = t_min;
            best_c = p->tuning;
        }
    }
    p->tuning = best_c;
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return XM_OK;
}

int xm_count(xm_graph g, xm_plan p, uint64_t* lo, uint64_t* hi, void* stream) {
    if (!g || !p || !lo || !hi) { set_error("NULL argument"); return XM_EINVAL; }
    begin_call(g);
    u128 r = 0;
    int rc = count_plan(g, p->plan, p->tuning, r, (cudaStream_t)stream);
    if (rc) return rc;
    *lo = (uint64_t)r;
    *hi = (uint64_t)(r >> 64);
    return XM_OK;
}

int xm_count_range(xm_graph g, xm_plan p, int64_t root_lo, int64_t root_hi, uint64_t* lo, uint64_t* hi,
                   void* stream) {
    if (!g || !p || !lo || !hi) { set_error("NULL argument"); return XM_EINVAL; }
    begin_call(g);
    return count_sub(g, p, MODE_COUNT, root_lo, root_hi, nullptr, 0, lo, hi, nullptr, (cudaStream_t)stream);
}

int xm_count_stats(xm_graph g, xm_plan p, int64_t root_lo, int64_t root_hi, uint64_t* lo, uint64_t* hi,
                   xm_stats* stats, void* stream) {
    if (!stats) { set_error("NULL stats"); return XM_EINVAL; }
    if (!g || !p || !lo || !hi) { set_error("NULL argument"); return XM_EINVAL; }
    begin_call(g);
    return count_sub(g, p, MODE_STATS, root_lo, root_hi, nullptr, 0, lo, hi, stats, (cudaStream_t)stream);
}

// Uploads a validated, sorted, repeat-free copy of a host root list into the
// graph's root buffer (allocated on first use).
static int stage_roots(xm_graph g, const int32_t* roots, int64_t nroots, int64_t* kept, cudaStream_t stream) {
    if (!roots || nroots < 0 || nroots > g->n) { set_error("bad root list"); return XM_EINVAL; }
    std::vector<int32_t> r(roots, roots + nroots);
    for (int32_t v : r)
        if (v < 0 || v >= g->n) { set_error("root id outside [0, n)"); return XM_EINVAL; }
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    if (!g->d_roots) {
        cudaError_t e = dev_alloc(&g->d_roots, (size_t)g->n * sizeof(int32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->d_roots = nullptr;
            set_error(std::string("root buffer: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA;
        }
    }
    if (!r.empty())
        XM_CUDA(cudaMemcpyAsync(g->d_roots, r.data(), r.size() * sizeof(int32_t), cudaMemcpyHostToDevice, stream),
                "root upload");
    XM_CUDA(cudaStreamSynchronize(stream), "root upload");
    if (kept) *kept = (int64_t)r.size();
    return XM_OK;
}

int xm_count_roots(xm_graph g, xm_plan p, const int32_t* roots, int64_t nroots, uint64_t* lo, uint64_t* hi,
                   void* stream) {
    if (!g || !p || !lo || !hi) { set_error("NULL argument"); return XM_EINVAL; }
    int64_t kept = 0;
    int rc = stage_roots(g, roots, nroots, &kept, (cudaStream_t)stream);
    if (rc) return rc;
    if (kept == 0) { *lo = *hi = 0; return XM_OK; }
    begin_call(g);
    return count_sub(g, p, MODE_COUNT, 0, INT32_MAX, g->d_roots, kept, lo, hi, nullptr, (cudaStream_t)stream);
}

int xm_count_roots_each(xm_graph g, xm_plan p, const int32_t* roots, int64_t nroots, uint64_t* counts,
                        void* stream_) {
    if (!g || !p || (nroots > 0 && !counts)) { set_error("NULL argument"); return XM_EINVAL; }
    if (!roots || nroots < 0) { set_error("bad root list"); return XM_EINVAL; }
    cudaStream_t stream = (cudaStream_t)stream_;
    for (int64_t i = 0; i < nroots; i++)
        if (roots[i] < 0 || roots[i] >= g->n) { set_error("root id outside [0, n)"); return XM_EINVAL; }
    // distinct roots, sorted; each caller entry maps to its position
    std::vector<int32_t> r(roots, roots + nroots);
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    const int64_t kept = (int64_t)r.size();
    if (kept == 0) return XM_OK;
    int rc = stage_roots(g, r.data(), kept, nullptr, stream);
    if (rc) return rc;
    begin_call(g);
    // one pass of the plan, or (rooted cut-vertex split) one pass per part
    // and per rooted quotient, each with its own per-root counters
    const Plan& P = p->plan;
    const Decomp* d = rooted_split(P) ? P.decomp.get() : nullptr;
    std::vector<const Plan*> passes;
    if (d) {
        for (const Plan& q : d->parts) passes.push_back(&q);
        for (const Plan& q : d->rquots) passes.push_back(&q);
    } else {
        passes.push_back(&P);
    }
    const size_t per_pass = 2 * (size_t)kept;
    if ((rc = ensure_root_counts(g, per_pass * passes.size()))) return rc;
    XM_CUDA(cudaMemsetAsync(g->d_root_counts, 0, per_pass * passes.size() * sizeof(unsigned long long), stream),
            "memset");
    for (size_t i = 0; i < passes.size(); i++) {
        uint64_t lo = 0, hi = 0;
        rc = run_plan(g, *passes[i], p->tuning, MODE_COUNT, 0, INT32_MAX, nullptr, 0, &lo, &hi, nullptr, nullptr,
                      stream, g->d_roots, kept, g->d_root_counts + i * per_pass);
        if (rc) return rc;
    }
    std::vector<uint64_t> per(per_pass * passes.size());
    XM_CUDA(cudaMemcpyAsync(per.data(), g->d_root_counts, per.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                            stream),
            "per-root readback");
    XM_CUDA(cudaStreamSynchronize(stream), "per-root readback");
    auto at = [&](size_t pass, int64_t j) { return ((u128)per[pass * per_pass + 2 * j + 1] << 64) | per[pass * per_pass + 2 * j]; };
    std::vector<u128> res((size_t)kept);
    for (int64_t j = 0; j < kept; j++) {
        if (!d) { res[j] = at(0, j); continue; }
        // the per-node form of the split identity (Decomp::rooted)
        const size_t np = d->parts.size();
        u128 emb = (u128)d->part_factor;
        for (size_t i = 0; i < np; i++) emb *= at(i, j);
        for (size_t q = 0; q < d->rquots.size(); q++)
            emb -= at(np + q, j) * (u128)d->rquots[q].stab_size * (u128)d->quot_mult[q];
        res[j] = (P.flags & XM_EMBEDDINGS) ? emb : emb / (u128)P.aut_size;
    }
    for (int64_t i = 0; i < nroots; i++) {
        const int64_t j = std::lower_bound(r.begin(), r.end(), roots[i]) - r.begin();
        counts[2 * i] = (uint64_t)res[j];
        counts[2 * i + 1] = (uint64_t)(res[j] >> 64);
    }
    return XM_OK;
}

int xm_count_roots_stats(xm_graph g, xm_plan p, const int32_t* roots, int64_t nroots, uint64_t* lo, uint64_t* hi,
                         xm_stats* stats, void* stream) {
    if (!g || !p || !lo || !hi || !stats) { set_error("NULL argument"); return XM_EINVAL; }
    int64_t kept = 0;
    int rc = stage_roots(g, roots, nroots, &kept, (cudaStream_t)stream);
    if (rc) return rc;
    if (kept == 0) {
        *lo = *hi = 0;
        memset(stats, 0, sizeof *stats);
        return XM_OK;
    }
    begin_call(g);
    return count_sub(g, p, MODE_STATS, 0, INT32_MAX, g->d_roots, kept, lo, hi, stats, (cudaStream_t)stream);
}

int xm_enumerate_roots(xm_graph g, xm_plan p, const int32_t* roots, int64_t nroots, int32_t* dev_out,
                       uint64_t capacity, uint64_t* total, uint64_t* written, void* stream) {
    if (!g || !p || !total || !written) { set_error("NULL argument"); return XM_EINVAL; }
    int64_t kept = 0;
    int rc = stage_roots(g, roots, nroots, &kept, (cudaStream_t)stream);
    if (rc) return rc;
    if (kept == 0) { *total = *written = 0; return XM_OK; }
    begin_call(g);
    uint64_t lo = 0, hi = 0, w = 0;
    rc = run(g, p, MODE_EMIT, 0, INT32_MAX, dev_out, capacity, &lo, &hi, nullptr, &w, (cudaStream_t)stream,
             g->d_roots, kept);
    if (rc == XM_OK || rc == XM_EOVERFLOW) {
        *total = lo;
        *written = w;
    }
    return rc;
}

int xm_enumerate_range(xm_graph g, xm_plan p, int64_t root_lo, int64_t root_hi, int32_t* dev_out,
                       uint64_t capacity, uint64_t* total, uint64_t* written, void* stream) {
    if (!total || !written) { set_error("NULL output"); return XM_EINVAL; }
    begin_call(g);
    uint64_t lo = 0, hi = 0, w = 0;
    int rc = run(g, p, MODE_EMIT, root_lo, root_hi, dev_out, capacity, &lo, &hi, nullptr, &w, (cudaStream_t)stream);
    if (rc == XM_OK || rc == XM_EOVERFLOW) {
        *total = lo;
        *written = w;
    }
    return rc;
}

int xm_enumerate(xm_graph g, xm_plan p, int32_t* dev_out, uint64_t capacity, uint64_t* total, uint64_t* written,
                 void* stream) {
    return xm_enumerate_range(g, p, 0, INT32_MAX, dev_out, capacity, total, written, stream);
}

}  // extern "C"
