// Host-side construction of the dual sorted CSR (out-lists and in-lists).
// Graph loading is outside the timed matching work, as in the paper's
// measurements (Sec. 6.1), so this is plain multi-threaded host code.
#include <algorithm>
#include <atomic>
#include <climits>
#include <thread>
#include <vector>

#include "xm_internal.h"

namespace xm {

namespace {

template <class F>
void parallel_for(int64_t n, F f) {
    unsigned hw = std::thread::hardware_concurrency();
    int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 1, 64));
    if (n < (1 << 16)) nt = 1;
    if (nt == 1) { f(0, n); return; }
    std::vector<std::thread> th;
    for (int64_t t = 0; t < nt; t++) {
        int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
        th.emplace_back([=] { f(lo, hi); });
    }
    for (auto& x : th) x.join();
}

}  // namespace

int build_host_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, HostCsr& G, std::string& err) {
    if (n < 1) { err = "n must be >= 1"; return XM_EINVAL; }
    if (m < 0) { err = "m must be >= 0"; return XM_EINVAL; }
    if (m > 0 && (!src || !dst)) { err = "NULL arc array"; return XM_EINVAL; }
    std::atomic<bool> bad{false};
    parallel_for(m, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; i++)
            if ((uint32_t)src[i] >= (uint32_t)n || (uint32_t)dst[i] >= (uint32_t)n) { bad = true; return; }
    });
    if (bad) { err = "arc endpoint outside [0, n)"; return XM_EINVAL; }

    // bucket by source (self-loops dropped)
    std::vector<int64_t> off(n + 1, 0);
    for (int64_t i = 0; i < m; i++)
        if (src[i] != dst[i]) off[src[i] + 1]++;
    for (int32_t v = 0; v < n; v++) off[v + 1] += off[v];
    std::vector<int32_t> adj(std::max<int64_t>(off[n], 1));
    {
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int64_t i = 0; i < m; i++)
            if (src[i] != dst[i]) adj[fill[src[i]]++] = dst[i];
    }
    // sort each list, drop repeats, record new lengths
    std::vector<int64_t> len(n + 1, 0);
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; v++) {
            int32_t* b = adj.data() + off[v];
            int32_t* e = adj.data() + off[v + 1];
            std::sort(b, e);
            len[v] = std::unique(b, e) - b;
        }
    });
    int64_t total = 0;
    for (int32_t v = 0; v < n; v++) total += len[v];
    if (total > INT32_MAX) { err = "more than 2^31-1 arcs after deduplication"; return XM_EINVAL; }
    G.n = n;
    G.m = total;
    G.out_off.assign(n + 1, 0);
    for (int32_t v = 0; v < n; v++) G.out_off[v + 1] = G.out_off[v] + (int32_t)len[v];
    G.out_adj.resize(std::max<int64_t>(total, 1));
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; v++)
            std::copy(adj.data() + off[v], adj.data() + off[v] + len[v], G.out_adj.data() + G.out_off[v]);
    });
    std::vector<int32_t>().swap(adj);

    // in-lists: bucket by destination, scanning sources in ascending order,
    // so every in-list comes out sorted and free of repeats
    G.in_off.assign(n + 1, 0);
    for (int64_t i = 0; i < total; i++) G.in_off[G.out_adj[i] + 1]++;
    for (int32_t v = 0; v < n; v++) G.in_off[v + 1] += G.in_off[v];
    G.in_adj.resize(std::max<int64_t>(total, 1));
    {
        std::vector<int32_t> fill(G.in_off.begin(), G.in_off.end() - 1);
        for (int32_t u = 0; u < n; u++)
            for (int32_t i = G.out_off[u]; i < G.out_off[u + 1]; i++) G.in_adj[fill[G.out_adj[i]]++] = u;
    }
    return XM_OK;
}

}  // namespace xm
