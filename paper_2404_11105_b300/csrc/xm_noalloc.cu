// xm_count_noalloc: the count pipeline on a fixed, library-owned scratch
// area, for callers that cannot allocate device memory.
//
// The regular entry points keep their scratch in buffers that xm_load_graph
// allocates with cudaMalloc. Some callers cannot do that: a process that has
// handed all device memory to its own pool allocator up front, or a
// latency-critical loop that must not pay for cudaMalloc/cudaFree (which may
// synchronise the whole device). This entry point runs the same kernels as
// xm_count, but every scratch array lives in one file-scope __device__ array
// of XM_NOALLOC_SCRATCH_BYTES that each device loading the library holds
// until the process exits. The caller passes the graph as its own device CSR
// arrays and gets the count back; nothing is allocated.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "xm_internal.h"
#include "xm_kernels.cuh"

namespace {

static __device__ __align__(256) unsigned char xm_noalloc_scratch[XM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current. The host-side symbol itself is only
// a stand-in and must never reach a kernel.
int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { xm::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return XM_ECUDA; }
    if (dev < 0 || dev >= kMaxDevices) { xm::set_error("device index beyond the supported range"); return XM_EINVAL; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, xm_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            xm::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return XM_ECUDA;
        }
        g_scratch[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch[dev];
    return XM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int xm_count_noalloc(const int32_t* out_off, const int32_t* out_adj, const int32_t* in_off,
                                const int32_t* in_adj, int32_t n, int64_t m, xm_plan p, uint64_t* lo, uint64_t* hi,
                                void* stream_) {
    using namespace xm;
    if (!p || !lo || !hi || !out_off || !in_off || (m > 0 && (!out_adj || !in_adj))) {
        set_error("NULL argument");
        return XM_EINVAL;
    }
    if (n < 1 || m < 0 || (int64_t)n + m >= (int64_t)INT32_MAX) {
        set_error("n must be >= 1, m >= 0 and n + m < 2^31");
        return XM_EINVAL;
    }
    // scratch layout, each piece 256-byte aligned: root_chunks[n+1],
    // chunk_cnt[cmax+1], l1set[max(m,1)], l1root[max(m,1)], units[n+1],
    // e_units[max(m,1)+1], block sums, control block (counters + plan copy)
    const int64_t cmax = chunk_capacity(n, m);
    const int64_t emax = std::max<int64_t>(m, 1);
    const int64_t n_block_sums =
        (std::max<int64_t>(std::max<int64_t>((int64_t)n + 1, cmax + 1), emax + 1) + SCAN_TILE - 1) / SCAN_TILE;
    const size_t b_nodes = align256(((size_t)n + 1) * sizeof(int32_t));
    const size_t b_chunks = align256((size_t)(cmax + 1) * sizeof(int32_t));
    const size_t b_l1 = align256((size_t)emax * sizeof(int32_t));
    const size_t b_e = align256((size_t)(emax + 1) * sizeof(int32_t));
    const size_t b_sums = align256((size_t)n_block_sums * sizeof(int64_t));
    const size_t b_ctl = align256(CTL_WORDS * sizeof(unsigned long long)) + align256(sizeof(XmPlanDev));
    const size_t need = 2 * b_nodes + b_chunks + 2 * b_l1 + b_e + b_sums + b_ctl;
    if (need > (size_t)XM_NOALLOC_SCRATCH_BYTES) {
        set_error("graph too large for the fixed scratch area of xm_count_noalloc (needs " + std::to_string(need) +
                  " bytes, has " + std::to_string((size_t)XM_NOALLOC_SCRATCH_BYTES) + "); use xm_count");
        return XM_EINVAL;
    }
    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    cudaStream_t stream = (cudaStream_t)stream_;
    {
        // the kernels size their scans and first-level arrays from m: both
        // CSRs must end at m, or they would read past the lists and the
        // scratch pieces (two 4-byte reads into host memory, no allocation)
        int32_t ends[2] = {-1, -1};
        cudaError_t e = cudaMemcpyAsync(&ends[0], out_off + n, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], in_off + n, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            set_error(std::string("xm_count_noalloc: reading the CSR ends: ") + cudaGetErrorString(e));
            return XM_ECUDA;
        }
        if (ends[0] != m || ends[1] != m) {
            set_error("xm_count_noalloc: out_off[n] and in_off[n] must both equal m (got " + std::to_string(ends[0]) +
                      ", " + std::to_string(ends[1]) + ", m = " + std::to_string(m) + ")");
            return XM_EINVAL;
        }
    }
    unsigned char* q = base;
    RunArgs a;
    a.g = {out_off, out_adj, in_off, in_adj, n};
    a.root_chunks = reinterpret_cast<int32_t*>(q); q += b_nodes;
    a.chunk_cnt = reinterpret_cast<int32_t*>(q); q += b_chunks;
    a.l1set = reinterpret_cast<int32_t*>(q); q += b_l1;
    a.l1root = reinterpret_cast<int32_t*>(q); q += b_l1;
    a.units = reinterpret_cast<int32_t*>(q); q += b_nodes;
    a.e_units = reinterpret_cast<int32_t*>(q); q += b_e;
    a.emax = (int32_t)emax;
    a.l2_units = use_l2_units(p->plan.dev, true) ? 1 : 0;
    a.leaf_kind = a.l2_units ? 0 : leaf_closed_form_kind(p->plan.dev);
    a.block_sums = reinterpret_cast<int64_t*>(q); q += b_sums;
    a.ctl = reinterpret_cast<unsigned long long*>(q);
    XmPlanDev* plan_dev = reinterpret_cast<XmPlanDev*>(q + align256(CTL_WORDS * sizeof(unsigned long long)));
    a.n_block_sums = n_block_sums;
    a.cmax = (int32_t)cmax;
    a.r_lo = 0;
    a.r_hi = n;
    a.root_list = nullptr;
    a.n_idx = n;
    a.unit = p->tuning.unit;
    a.window = p->tuning.window;
    a.out = nullptr;
    a.capacity = 0;
    a.budget_ns = (unsigned long long)p->tuning.budget_ms * 1000000ull;
    a.merge_ratio = p->tuning.merge_ratio;
    // the control block (work counter, count accumulators, status) must
    // start at zero; every other array is fully written before it is read
    cudaError_t e = cudaMemsetAsync(a.ctl, 0, CTL_WORDS * sizeof(unsigned long long), stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(plan_dev, &p->plan.dev, sizeof(XmPlanDev), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = launch_match(MODE_COUNT, p->plan.dev, plan_dev, a, p->tuning.warps_per_block, p->tuning.blocks_per_sm,
                         stream, nullptr);
    unsigned long long ctl[CTL_WORDS];
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, a.ctl, sizeof ctl, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        set_error(std::string("xm_count_noalloc: ") + cudaGetErrorString(e));
        return XM_ECUDA;
    }
    if (ctl[CTL_STATUS] & STATUS_TIMEOUT) {
        set_error("time budget of the matcher exceeded; no count");
        return XM_ETIMEOUT;
    }
    if (ctl[CTL_STATUS]) {
        set_error("work-unit count exceeds 2^31-1 (raise the unit size)");
        return XM_EINVAL;
    }
    *lo = ctl[CTL_COUNT_LO];
    *hi = ctl[CTL_COUNT_HI];
    return XM_OK;
}
