// Host-side construction of the dual sorted CSR (out-lists and in-lists).
// Graph loading is outside the timed matching work, as in the paper's
// measurements (Sec. 6.1), but it is the whole of an end-to-end call's
// host time, so it is a parallel bucket sort: arcs are scattered into
// buckets of consecutive source ids (per-thread counts, one prefix sum), each
// bucket is sorted as packed 64-bit (source, destination) keys and
// deduplicated on its own, and the buckets are concatenated. The in-lists
// are built the same way from the deduplicated arcs with the key halves
// swapped. The staging arrays are kept between builds (see Staging): pages
// that are already mapped cost nothing to reuse, while fresh ones cost a page
// fault each on first touch, which made up half of a scale-20 build.
#include <algorithm>
#include <atomic>
#include <climits>
#include <mutex>
#include <thread>
#include <vector>

#include "xm_internal.h"

namespace xm {

namespace {

// one thread per 2^17 items, at most the hardware threads (and 64)
int n_threads(int64_t work) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int64_t cap = std::min<int64_t>(hw ? hw : 1, 64);
    return (int)std::max<int64_t>(1, std::min<int64_t>(cap, work >> 17));
}

// Host staging arrays of the CSR build, grown to the largest graph built so
// far and kept until the process exits (about 16 B per arc plus 12 B per
// node); builds take turns on them.
struct Staging {
    std::mutex mu;
    HostVec<uint64_t> keys;
    HostVec<int32_t> cols, deg, row_of;
    HostVec<int64_t> rstart;
};

Staging& staging() {
    static Staging s;
    return s;
}

template <class F>
void parallel_for(int64_t n, int nt, F f) {
    if (nt <= 1 || n < 2) { f(0, 0, n); return; }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; t++) {
        int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
        th.emplace_back([=] { f(t, lo, hi); });
    }
    for (auto& x : th) x.join();
}

// Sorted, repeat-free CSR of the keys (key_of(i) -> (row, col)) for rows
// [0, n): off[n+1], adj[count]. Self-loops are dropped. Returns the number of
// distinct arcs; above 2^31-1 nothing is filled (int32 offsets).
template <class KeyOf>
int64_t build_side(int32_t n, int64_t m, KeyOf key_of, HostVec<int32_t>& off, HostVec<int32_t>& adj,
                   Staging& st) {
    const int nt = n_threads(m);
    // buckets of consecutive rows
    const int64_t nb = std::max<int64_t>(1, std::min<int64_t>({(int64_t)n, 8192, m >> 10}));
    auto bucket = [&](uint32_t row) { return (int64_t)row * nb / n; };
    std::vector<int64_t> cnt((size_t)nt * nb, 0);
    parallel_for(m, nt, [&](int t, int64_t lo, int64_t hi) {
        int64_t* c = cnt.data() + (size_t)t * nb;
        for (int64_t i = lo; i < hi; i++) {
            const uint64_t k = key_of(i);
            const uint32_t r = (uint32_t)(k >> 32), col = (uint32_t)k;
            if (r != col) c[bucket(r)]++;
        }
    });
    // prefix over (bucket, thread)
    std::vector<int64_t> start((size_t)nt * nb);
    std::vector<int64_t> bstart(nb + 1, 0);
    int64_t run = 0;
    for (int64_t b = 0; b < nb; b++) {
        bstart[b] = run;
        for (int t = 0; t < nt; t++) {
            start[(size_t)t * nb + b] = run;
            run += cnt[(size_t)t * nb + b];
        }
    }
    bstart[nb] = run;
    HostVec<uint64_t>& keys = st.keys;
    keys.resize((size_t)std::max<int64_t>(run, 1));
    parallel_for(m, nt, [&](int t, int64_t lo, int64_t hi) {
        int64_t* s = start.data() + (size_t)t * nb;
        for (int64_t i = lo; i < hi; i++) {
            const uint64_t k = key_of(i);
            const uint32_t r = (uint32_t)(k >> 32), col = (uint32_t)k;
            if (r != col) keys[s[bucket(r)]++] = k;
        }
    });
    // per bucket: counting sort of its keys by row into int32 columns, then
    // sort + dedup each row; deg[r] = distinct columns of row r, compacted to
    // the front of the row's slot
    auto rows_of = [&](int64_t b, int64_t& lo, int64_t& hi) {
        lo = (b * n + nb - 1) / nb;
        hi = ((b + 1) * n + nb - 1) / nb;
    };
    HostVec<int32_t>& cols = st.cols;
    HostVec<int64_t>& rstart = st.rstart;
    HostVec<int32_t>& deg = st.deg;
    cols.resize((size_t)std::max<int64_t>(run, 1));
    rstart.resize((size_t)n);
    deg.resize((size_t)n);
    std::vector<int64_t> kept(nb, 0);
    std::atomic<int64_t> next{0};
    auto sort_rows = [&](int, int64_t, int64_t) {
        for (;;) {
            const int64_t b = next.fetch_add(1);
            if (b >= nb) break;
            int64_t row_lo, row_hi;
            rows_of(b, row_lo, row_hi);
            const uint64_t* k = keys.data() + bstart[b];
            const int64_t c = bstart[b + 1] - bstart[b];
            const int64_t nr = row_hi - row_lo;
            std::vector<int64_t> pos((size_t)nr + 1, 0);
            for (int64_t i = 0; i < c; i++) pos[(int64_t)(k[i] >> 32) - row_lo + 1]++;
            pos[0] = bstart[b];
            for (int64_t r = 1; r <= nr; r++) pos[r] += pos[r - 1];
            std::vector<int64_t> cur(pos.begin(), pos.end() - 1);
            for (int64_t i = 0; i < c; i++) {
                const int64_t r = (int64_t)(k[i] >> 32) - row_lo;
                cols[cur[r]++] = (int32_t)(uint32_t)k[i];
            }
            int64_t d = 0;
            for (int64_t r = 0; r < nr; r++) {
                int32_t* a = cols.data() + pos[r];
                int32_t* e = cols.data() + pos[r + 1];
                rstart[row_lo + r] = pos[r];
                std::sort(a, e);
                deg[row_lo + r] = (int32_t)(std::unique(a, e) - a);
                d += deg[row_lo + r];
            }
            kept[b] = d;
        }
    };
    parallel_for(nt, nt, sort_rows);
    std::vector<int64_t> kstart(nb + 1, 0);
    for (int64_t b = 0; b < nb; b++) kstart[b + 1] = kstart[b] + kept[b];
    const int64_t total = kstart[nb];
    if (total > INT32_MAX) return total;
    adj.resize((size_t)std::max<int64_t>(total, 1));
    off.resize((size_t)n + 1);
    // concatenate the deduplicated rows
    next = 0;
    auto fill = [&](int, int64_t, int64_t) {
        for (;;) {
            const int64_t b = next.fetch_add(1);
            if (b >= nb) break;
            int64_t row_lo, row_hi;
            rows_of(b, row_lo, row_hi);
            int64_t w = kstart[b];
            for (int64_t r = row_lo; r < row_hi; r++) {
                off[r] = (int32_t)w;
                std::copy(cols.data() + rstart[r], cols.data() + rstart[r] + deg[r], adj.data() + w);
                w += deg[r];
            }
        }
    };
    parallel_for(nt, nt, fill);
    off[n] = (int32_t)total;
    return total;
}

}  // namespace

int build_host_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, HostCsr& G, std::string& err) {
    if (n < 1) { err = "n must be >= 1"; return XM_EINVAL; }
    if (m < 0) { err = "m must be >= 0"; return XM_EINVAL; }
    if (m > 0 && (!src || !dst)) { err = "NULL arc array"; return XM_EINVAL; }
    std::atomic<bool> bad{false};
    parallel_for(m, n_threads(m), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; i++)
            if ((uint32_t)src[i] >= (uint32_t)n || (uint32_t)dst[i] >= (uint32_t)n) { bad = true; return; }
    });
    if (bad) { err = "arc endpoint outside [0, n)"; return XM_EINVAL; }
    // the arc count after deduplication must fit the int32 offsets
    if (m > (int64_t)INT32_MAX * 2) { err = "too many arcs"; return XM_EINVAL; }
    Staging& st = staging();
    std::lock_guard<std::mutex> lock(st.mu);

    const int64_t total = build_side(
        n, m, [&](int64_t i) { return ((uint64_t)(uint32_t)src[i] << 32) | (uint32_t)dst[i]; }, G.out_off, G.out_adj, st);
    if (total > INT32_MAX) { err = "more than 2^31-1 arcs after deduplication"; return XM_EINVAL; }
    G.n = n;
    G.m = total;
    // in-lists from the deduplicated out-arcs: row of arc i is the source,
    // found by walking the offsets (build an explicit source array once)
    HostVec<int32_t>& row_of = st.row_of;
    row_of.resize((size_t)std::max<int64_t>(total, 1));
    parallel_for(n, n_threads(total), [&](int, int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; v++)
            for (int32_t i = G.out_off[v]; i < G.out_off[v + 1]; i++) row_of[i] = (int32_t)v;
    });
    build_side(n, total,
               [&](int64_t i) { return ((uint64_t)(uint32_t)G.out_adj[i] << 32) | (uint32_t)row_of[i]; }, G.in_off,
               G.in_adj, st);
    return XM_OK;
}

}  // namespace xm
