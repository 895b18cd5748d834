// Device matcher for directed subgraph matching (plan execution, Alg. 2 of
// the XMiner paper, re-designed for one B300 GPU).
//
// Pipeline of one count/enumerate call (all kernels on the caller's stream):
//   1. first-level candidate sets. Alg. 2 materialises A^{p.start} and, for
//      every start node, the endpoint set of the first explored edge. Here
//      the first plan level's set C_1(v) = AND of v's operand lists (order
//      bounds and degree filter applied) is built once per start node v into
//      a global buffer, in fixed chunks of the driver list so that hub nodes
//      are spread over many warps: k_l1_chunks (chunks per node), a scan,
//      k_l1_count (survivors per chunk), a scan, k_l1_write (compaction).
//   2. work units: each C_1(v) is cut into units of `unit` candidates
//      (k_units + scan); the units of all start nodes form one index space.
//   3. k_match: a persistent grid of warps takes units from a global counter
//      (guided self-scheduling) and runs the depth-first Explore() recursion
//      below the unit's first-level candidates as an explicit stack of plan
//      levels in shared memory.
//
// Per deeper level the warp builds the candidate set (Alg. 2: A^{e.dest} =
// A^{e.dest} cap Pi A^e) in chunks into a shared-memory window: lanes take 32
// consecutive ids of the shortest operand list (the driver), test each
// against the other operand lists by binary search, apply the order,
// injectivity and degree filters, and compact the survivors with
// __ballot_sync/__popc. A level whose whole candidate set is held (the
// first level always, deeper levels when the set fits the window) is
// "complete" and can replace, for later levels, the operand lists it already
// intersected (Sec. 5.2 intermediate-result reuse). The last level is never
// materialised: its candidates are counted (Sec. 5.3 count-only result
// generation) or written out.
#include <algorithm>
#include <climits>
#include <cstddef>

#include "xm_kernels.cuh"

namespace xm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Work budget of a launch (or of one pair of a batch): the first warp to
// start records the start time in *t0; a warp whose check finds the budget
// spent raises the timeout bit in *status, and every warp that checks the
// same words stops at its next check.
struct Budget {
    unsigned long long deadline = 0;  // 0: unlimited
    unsigned long long* status = nullptr;
    __device__ void start(unsigned long long* c, unsigned long long budget_ns, int lane) {
        start_at(c + CTL_T0, c + CTL_STATUS, budget_ns, lane);
    }
    __device__ void start_at(unsigned long long* t0w, unsigned long long* st, unsigned long long budget_ns, int lane) {
        status = st;
        deadline = 0;
        if (!budget_ns) return;
        unsigned long long t0 = 0;
        if (lane == 0) {
            const unsigned long long now = global_ns();
            const unsigned long long prev = atomicCAS(t0w, 0ull, now);
            t0 = prev ? prev : now;
        }
        deadline = __shfl_sync(FULL, t0, 0) + budget_ns;
    }
#ifdef XM_BATCH_TU
    // A budget of one work unit: the deadline counts from this warp's start
    // of the unit; `st` is shared by all units of the same work (one pair).
    __device__ void start_unit(unsigned long long* st, unsigned long long budget_ns, int lane) {
        status = st;
        deadline = 0;
        if (!budget_ns) return;
        const unsigned long long now = lane == 0 ? global_ns() : 0ull;
        deadline = __shfl_sync(FULL, now, 0) + budget_ns;
    }
#endif
    // true when the work must stop (warp-uniform)
    __device__ bool expired(int lane) const {
        if (!deadline) return false;
        int stop = 0;
        if (lane == 0) {
            stop = (*((volatile unsigned long long*)status) & STATUS_TIMEOUT) != 0;
            if (!stop && global_ns() > deadline) {
                atomicOr(status, (unsigned long long)STATUS_TIMEOUT);
                stop = 1;
            }
        }
        return __shfl_sync(FULL, stop, 0) != 0;
    }
};

struct ListRef {
    const int32_t* p;
    int32_t len;
    int32_t shared;
    const int32_t* tab;  // hash table of the list, or null
    uint32_t T;          // its size (0: none)
};

struct LvState {
    const int32_t* drv;
    const int32_t* probe[XM_MAXOPS];
    const int32_t* ptab[XM_MAXOPS];  // probe hash tables (null: binary search)
    uint32_t pT[XM_MAXOPS];
    const int32_t* it_ptr;   // materialised candidates being iterated
    const int32_t* set_ptr;  // the complete candidate set (when complete)
    int32_t plo[XM_MAXOPS];
    int32_t phi[XM_MAXOPS];
    int32_t drv_shared;
    int32_t probe_shared;  // bit i: probe i lives in shared memory
    int32_t nprobe;
    int32_t c0, c1;        // cut driver range (order bounds applied)
    int32_t drv_pos, drv_end;
    int32_t wcnt, wpos, it_hi, it_shared;
    int32_t set_len, set_shared, complete;
    int32_t empty;
};

// Per-warp state in shared memory. Only the first k entries of st[] exist
// (the layout is cut to the plan's size so that more of the SM's on-chip
// memory stays L1 cache); never index st[] at or beyond k.
// Probes each lane issues per round of the batched last level, with the
// next round's driver ids already loaded (measured on the scale-24
// four-level patterns: 2 beats 4 and 6 by 2-13 %; 8 needs more than 64
// registers).
constexpr int LEAF_PPL = 2;

// One pair of a batched last level: its driver ids at d[t] for flattened
// positions t < end (d is offset by the pair's first position), and the list
// it probes (a hash table of n > 0 slots, or -n ascending ids).
struct LeafPair {
    const int32_t* d;
    const int32_t* tab;
    int32_t end;
    int32_t n;
};

struct WarpSmem {
    int32_t* mtile;  // this warp's MERGE_TILE-id tile for merge intersections
    int32_t m[XM_MAXK];
    LeafPair lp[32];  // the batched last level's pairs
    LvState st[XM_MAXK];
};

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Bytes of a plan copy holding levels 0..k-1, and of a warp's state for k levels.
__host__ __device__ constexpr size_t plan_bytes(int k) {
    return al16(offsetof(XmPlanDev, lv) + (size_t)k * sizeof(XmLevel));
}
__host__ __device__ constexpr size_t warp_state_bytes(int k) {
    return al16(offsetof(WarpSmem, st) + (size_t)k * sizeof(LvState));
}

#ifdef XM_BATCH_TU
__host__ __device__ size_t batch_warp_bytes_impl(int kmax, int window) {
    return plan_bytes(kmax) + warp_state_bytes(kmax) + (size_t)(kmax > 2 ? kmax - 2 : 0) * window * sizeof(int32_t) +
           MERGE_TILE * sizeof(int32_t);
}
#endif


__host__ __device__ constexpr int n_windows(int k) { return k > 3 ? k - 3 : 0; }

// Per-warp shared memory of k_match: level state, windows of levels
// 2..k-2, and the merge tile when merging is enabled (shared memory not
// taken stays L1 cache, which the probe loops live on).
__host__ __device__ constexpr size_t match_warp_bytes(int k, int window, bool merge) {
    return warp_state_bytes(k) + (size_t)n_windows(k) * window * sizeof(int32_t) +
           (merge ? MERGE_TILE * sizeof(int32_t) : 0);
}



// Sum of a 32-bit value over the warp (every lane gets the total).
__device__ __forceinline__ unsigned warp_sum(unsigned v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ int32_t ld(const int32_t* p, int i, bool shared) {
    return shared ? p[i] : __ldg(p + i);
}

// first index in [lo, hi) with p[idx] >= x
__device__ __forceinline__ int lbound(const int32_t* p, int lo, int hi, int32_t x, bool shared) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (ld(p, mid, shared) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Warp-cooperative lower bounds on a sorted global list, for the
// instrumented kernel's accounting: the first index in [lo0, hi0) with
// p[idx] >= x0 and the first in [lo1, hi1) with p[idx] >= x1, computed by
// all 32 lanes together (every lane gets the results). Each round the lanes
// read 32 evenly spaced ids of each remaining range and one ballot narrows
// it 32-fold: about log32(L) + 1 rounds for a list of L ids.
__device__ __forceinline__ void warp_lbound2(const int32_t* p, int lo0, int hi0, int32_t x0, int lo1, int hi1,
                                             int32_t x1, int& r0, int& r1, int lane) {
    bool d0 = false, d1 = false;
    for (;;) {
        const bool w0 = !d0 && hi0 - lo0 > 32, w1 = !d1 && hi1 - lo1 > 32;
        if (!w0 && !w1) break;
        const int s0 = (hi0 - lo0 + 31) >> 5, s1 = (hi1 - lo1 + 31) >> 5;
        const int q0 = lo0 + lane * s0, q1 = lo1 + lane * s1;
        const int32_t v0 = (w0 && q0 < hi0) ? __ldg(p + q0) : INT_MAX;
        const int32_t v1 = (w1 && q1 < hi1) ? __ldg(p + q1) : INT_MAX;
        const int c0 = __popc(__ballot_sync(FULL, v0 < x0));
        const int c1 = __popc(__ballot_sync(FULL, v1 < x1));
        if (w0) {
            if (c0 == 0) { hi0 = lo0; d0 = true; }
            else { const int nlo = lo0 + (c0 - 1) * s0 + 1; hi0 = min(hi0, lo0 + c0 * s0); lo0 = nlo; }
        }
        if (w1) {
            if (c1 == 0) { hi1 = lo1; d1 = true; }
            else { const int nlo = lo1 + (c1 - 1) * s1 + 1; hi1 = min(hi1, lo1 + c1 * s1); lo1 = nlo; }
        }
    }
    const int32_t v0 = lo0 + lane < hi0 ? __ldg(p + lo0 + lane) : INT_MAX;
    const int32_t v1 = lo1 + lane < hi1 ? __ldg(p + lo1 + lane) : INT_MAX;
    r0 = lo0 + __popc(__ballot_sync(FULL, v0 < x0));
    r1 = lo1 + __popc(__ballot_sync(FULL, v1 < x1));
}

__device__ __forceinline__ ListRef op_list(const GraphDev& g, int dir, int32_t v) {
    const bool out = dir == XM_DIR_OUT;
    const int32_t* off = out ? g.out_off : g.in_off;
    const int b = __ldg(off + v), e = __ldg(off + v + 1);
    ListRef r{(out ? g.out_adj : g.in_adj) + b, e - b, 0, nullptr, 0};
    const int64_t* hoff = out ? g.out_hoff : g.in_hoff;
    if (hoff && r.len >= HASH_MIN_LEN) {
        const int64_t t0 = __ldg(hoff + v);
        r.T = (uint32_t)(__ldg(hoff + v + 1) - t0);
        r.tab = (out ? g.out_htab : g.in_htab) + t0;
    }
    return r;
}

// One hash bucket (8 slots, one 32-byte sector) in a single 256-bit
// read-only load. Buckets are 32-byte aligned: every table holds a power of
// two >= 64 slots and starts at a multiple of 64 slots of a 256-byte aligned
// allocation. One load per lane halves the L1 wavefronts of the two 16-byte
// loads it replaces (the probe loops were L1-throughput bound); random
// buckets are not kept in L1, which stays for the lists and offsets.
struct Bucket {
    int32_t v[HASH_BUCKET];
};
__device__ __forceinline__ Bucket load_bucket(const int32_t* p) {
    Bucket b;
    asm("ld.global.nc.L1::no_allocate.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(b.v[0]), "=r"(b.v[1]), "=r"(b.v[2]), "=r"(b.v[3]), "=r"(b.v[4]), "=r"(b.v[5]), "=r"(b.v[6]),
          "=r"(b.v[7])
        : "l"(p));
    return b;
}
__device__ __forceinline__ bool bucket_has(const Bucket& q, int32_t x) {
    return q.v[0] == x || q.v[1] == x || q.v[2] == x || q.v[3] == x || q.v[4] == x || q.v[5] == x ||
           q.v[6] == x || q.v[7] == x;
}
__device__ __forceinline__ bool bucket_open(const Bucket& q) {  // an empty slot (-1)
    return (q.v[0] | q.v[1] | q.v[2] | q.v[3] | q.v[4] | q.v[5] | q.v[6] | q.v[7]) < 0;
}

// Is x in the list whose hash table is tab[0..T)? A bucket with an empty
// slot ends the search (tables are at most half full).
__device__ __forceinline__ bool hash_has(const int32_t* __restrict__ tab, uint32_t T, int32_t x) {
    const uint32_t nb = T / HASH_BUCKET;
    uint32_t b = hash_bucket(x, nb);
    for (uint32_t step = 0; step < nb; step++) {
        const Bucket q = load_bucket(tab + (size_t)b * HASH_BUCKET);
        if (bucket_has(q, x)) return true;
        if (bucket_open(q)) return false;
        b = (b + 1) & (nb - 1);
    }
    return false;
}

// First bucket of a probe, split from the rest so that several probes can be
// in flight at once: sets `found`, and returns true when the first bucket
// settles the answer (x found, or an empty slot seen).
__device__ __forceinline__ bool hash_first(const int32_t* __restrict__ tab, uint32_t T, int32_t x, bool& found) {
    const uint32_t b = hash_bucket(x, T / HASH_BUCKET);
    const Bucket q = load_bucket(tab + (size_t)b * HASH_BUCKET);
    found = bucket_has(q, x);
    return found || bucket_open(q);
}

// Order bounds of a level: candidates x must satisfy lo < x < hi.
__device__ __forceinline__ void level_bounds(const XmLevel& L, const int32_t* m, int32_t& lo, int32_t& hi) {
    lo = -1;
    hi = INT_MAX;
    for (uint32_t a = L.lo_mask; a; a &= a - 1) lo = max(lo, m[__ffs(a) - 1]);
    for (uint32_t b = L.hi_mask; b; b &= b - 1) hi = min(hi, m[__ffs(b) - 1]);
}

// Operand lists of the first level for start node v: the driver (shortest
// list, ties to the first operand), the other list if any (the first level
// can only have an out- and an in-list of v), and the driver range cut by
// the order bounds.
__device__ __forceinline__ void first_level_lists(const XmPlanDev& P, const GraphDev& g, int32_t v, ListRef& drv,
                                                  ListRef& other, int& nother, int& c0, int& c1) {
    const XmLevel& L = P.lv[1];
    drv = op_list(g, L.op_dir[0], v);
    nother = 0;
    other = {nullptr, 0, 0, nullptr, 0};
    if (L.nops > 1) {
        ListRef r = op_list(g, L.op_dir[1], v);
        nother = 1;
        if (r.len < drv.len) { other = drv; drv = r; } else { other = r; }
    }
    int32_t lo = (L.lo_mask & 1u) ? v : -1;
    int32_t hi = (L.hi_mask & 1u) ? v : INT_MAX;
    c0 = 0;
    c1 = drv.len;
    if (drv.len > 0 && (nother == 0 || other.len > 0)) {
        if (lo >= 0) c0 = lbound(drv.p, 0, drv.len, lo + 1, false);
        if (hi != INT_MAX) c1 = lbound(drv.p, c0, drv.len, hi, false);
    } else {
        c1 = 0;
    }
    if (c1 < c0) c1 = c0;
}

__device__ __forceinline__ bool passes_degree(const GraphDev& g, int32_t x, int dmin_out, int dmin_in) {
    if (dmin_out > 0 && __ldg(g.out_off + x + 1) - __ldg(g.out_off + x) < dmin_out) return false;
    if (dmin_in > 0 && __ldg(g.in_off + x + 1) - __ldg(g.in_off + x) < dmin_in) return false;
    return true;
}

__device__ __forceinline__ bool list_has(const ListRef& r, int32_t x) {
    if (r.T) return hash_has(r.tab, r.T, x);
    const int q = lbound(r.p, 0, r.len, x, false);
    return q < r.len && __ldg(r.p + q) == x;
}

// Induced plans: x must lie in none of the level's difference lists. Inlined:
// as an out-of-line call its calling convention cost the matcher's count
// kernel registers (spills) once the product kernels also called it.
__device__ __forceinline__ bool passes_diffs(const XmLevel& L, const GraphDev& g, const int32_t* m, int32_t x) {
    for (int i = 0; i < L.ndiff; i++)
        if (list_has(op_list(g, L.diff_dir[i], m[L.diff_level[i]]), x)) return false;
    return true;
}

__device__ __forceinline__ int ceil_log2p1(int len) {  // ceil(log2(len + 1))
    return 32 - __clz(len);
}

// last index v in [0, n) with prefix[v] <= u (prefix is non-decreasing)
__device__ __forceinline__ int owner_of(const int32_t* __restrict__ prefix, int n, int u) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------ first-level candidate sets

__device__ __forceinline__ void plan_to_smem(XmPlanDev& P, const XmPlanDev* __restrict__ plan_g) {
    const int words = (int)(plan_bytes(__ldg(&plan_g->k)) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x)
        reinterpret_cast<int32_t*>(&P)[i] = reinterpret_cast<const int32_t*>(plan_g)[i];
    __syncthreads();
}

// Start node of index i (the root list, or the node itself).
__device__ __forceinline__ int32_t root_node(const RunArgs& ra, int i) {
    return ra.root_list ? __ldg(ra.root_list + i) : i;
}

#ifndef XM_BATCH_TU
// Chunks of the first-level driver list per start node (0 when the node
// fails the start vertex's degree filter or lies outside [r_lo, r_hi)).
__global__ void k_l1_chunks(const XmPlanDev* __restrict__ plan_g, RunArgs ra) {
    __shared__ __align__(16) unsigned char pbuf[plan_bytes(XM_MAXK)];
    XmPlanDev& P = *reinterpret_cast<XmPlanDev*>(pbuf);
    plan_to_smem(P, plan_g);
    const GraphDev& g = ra.g;
    const int ni = ra.n_idx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= ni; i += gridDim.x * blockDim.x) {
        int c = 0;
        const int v = i < ni ? root_node(ra, i) : -1;
        if (i < ni && v >= ra.r_lo && v < ra.r_hi && passes_degree(g, v, P.lv[0].dout_min, P.lv[0].din_min)) {
            ListRef d, o;
            int no, c0, c1;
            first_level_lists(P, g, v, d, o, no, c0, c1);
            c = (c1 - c0 + L1_CHUNK - 1) / L1_CHUNK;
        }
        ra.root_chunks[i] = c;
    }
}

// One warp per chunk: WRITE=false counts the chunk's survivors into
// chunk_cnt[c]; WRITE=true writes them at the scanned offset chunk_cnt[c].
template <bool WRITE, int MODE>
__global__ void __launch_bounds__(256) k_l1(const XmPlanDev* __restrict__ plan_g, RunArgs ra) {
    __shared__ __align__(16) unsigned char pbuf[plan_bytes(XM_MAXK)];
    XmPlanDev& P = *reinterpret_cast<XmPlanDev*>(pbuf);
    plan_to_smem(P, plan_g);
    const GraphDev& g = ra.g;
    const int ni = ra.n_idx;
    const int lane = threadIdx.x & 31;
    const int total = __ldg(ra.root_chunks + ni);
    const bool filter_deg = P.k > 2;
    const XmLevel& L1 = P.lv[1];
    unsigned long long st_bytes = 0;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // the entry after the last real chunk (the scan's terminal) gets a zero
    // count; the scan reads no further
    if (!WRITE && wid == 0 && lane == 0) ra.chunk_cnt[total] = 0;
    // warps take runs of consecutive chunks from a counter: a start node's
    // lists are fetched once per run, and the chunks of a hub still spread
    // over many warps
    constexpr int RUN = 4;
    unsigned long long* head = ra.ctl + CTL_L1_HEAD + (WRITE ? 1 : 0);
    int vi = -1, v = 0, no = 0, c0 = 0, c1 = 0;
    ListRef d{nullptr, 0, 0, nullptr, 0}, o{nullptr, 0, 0, nullptr, 0};
    for (;;) {
        int cb = 0;
        if (lane == 0) cb = (int)min((unsigned long long)total, atomicAdd(head, (unsigned long long)RUN));
        cb = __shfl_sync(FULL, cb, 0);
        if (cb >= total) break;
        const int ce = min(total, cb + RUN);
    for (int c = cb; c < ce; c++) {
        if (vi < 0 || c >= __ldg(ra.root_chunks + vi + 1)) {
            if (vi >= 0 && c < __ldg(ra.root_chunks + min(vi + 8, ni))) {
                do { vi++; } while (c >= __ldg(ra.root_chunks + vi + 1));
            } else {
                vi = owner_of(ra.root_chunks, ni, c);
            }
            v = root_node(ra, vi);
            first_level_lists(P, g, v, d, o, no, c0, c1);
        }
        const int j = c - __ldg(ra.root_chunks + vi);
        int pos = c0 + j * L1_CHUNK;
        const int end = min(c1, pos + L1_CHUNK);
        int plo = 0;
        int cnt = 0;
        int32_t* out = WRITE ? ra.l1set + ra.chunk_cnt[c] : nullptr;
        const bool filtered = no || L1.ndiff || (filter_deg && (L1.dout_min > 0 || L1.din_min > 0));
        // MODE_STATS (count pass only) adds the bytes of both passes: the
        // driver range and probes once, 8 B per degree check, 8 B per
        // candidate written with its owner, the offsets with a node's first
        // chunk
        if (!filtered) {
            // every driver id survives: count without reading, or copy
            if (WRITE) {
                int32_t* own = ra.l1root + (out - ra.l1set);
                for (int i = pos + lane; i < end; i += 32) {
                    out[i - pos] = __ldg(d.p + i);
                    own[i - pos] = vi;
                }
            } else if (lane == 0) {
                ra.chunk_cnt[c] = end - pos;
                if (MODE == MODE_STATS) st_bytes += (j == 0 ? 8ull : 0ull) + 12ull * (end - pos);
            }
            continue;
        }
        if (MODE == MODE_STATS && !WRITE && lane == 0) {
            const int run = end - pos;
            st_bytes += (j == 0 ? 8ull * (1 + no) : 0) + 4ull * run;
            if (no) st_bytes += 4ull * min((long long)o.len, (long long)run * ceil_log2p1(o.len));
        }
        for (; pos < end; pos += 32) {
            const int i = pos + lane;
            const bool valid = i < end;
            const int32_t x = valid ? __ldg(d.p + i) : INT_MAX;
            bool ok = valid;
            if (no) {
                if (o.T) {
                    ok = ok && hash_has(o.tab, o.T, x);
                } else {
                    const int q = lbound(o.p, plo, o.len, x, false);
                    ok = ok && q < o.len && __ldg(o.p + q) == x;
                    plo = __shfl_sync(FULL, q, min(31, end - 1 - pos));
                }
            }
            if (MODE == MODE_STATS && filter_deg && (L1.dout_min > 0 || L1.din_min > 0)) {
                const int checks = __popc(__ballot_sync(FULL, ok));
                if (lane == 0) st_bytes += 8ull * checks;
            }
            if (ok && filter_deg) ok = passes_degree(g, x, L1.dout_min, L1.din_min);
            if (ok && L1.ndiff) ok = passes_diffs(L1, g, &v, x);
            const unsigned mask = __ballot_sync(FULL, ok);
            if (WRITE && ok) {
                const int at = cnt + __popc(mask & ((1u << lane) - 1));
                out[at] = x;
                ra.l1root[ra.chunk_cnt[c] + at] = vi;
            }
            cnt += __popc(mask);
        }
        if (!WRITE && lane == 0) {
            ra.chunk_cnt[c] = cnt;
            if (MODE == MODE_STATS) st_bytes += 8ull * cnt;
        }
    }
    }
    if (MODE == MODE_STATS && !WRITE && lane == 0 && st_bytes) atomicAdd(ra.ctl + CTL_STATS + 5, st_bytes);
}

// Work units per start node: its first-level set cut into `unit` pieces.
__global__ void k_units(RunArgs ra) {
    const int n = ra.n_idx;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        int u = 0;
        if (v < n) {
            const int len = ra.chunk_cnt[ra.root_chunks[v + 1]] - ra.chunk_cnt[ra.root_chunks[v]];
            u = (len + ra.unit - 1) / ra.unit;
        }
        ra.units[v] = u;
    }
}

#endif
// ------------------------------------------------------ merge intersection
// Two sorted lists of similar length are intersected by streaming both
// (Alg. 2's A^{e.dest} cap Pi A^e when no list is much shorter than the
// other): every id is read once, in coalesced 16-byte loads, instead of one
// random hash-bucket sector per id of the shorter list.

// Chunk q (16 bytes, four ids) of the tile of list p that starts at the
// 16-byte boundary at or below position pos; *t0 receives the tile's first
// position. Ids at positions before pos read as -1 and at or after end as
// INT_MAX, so they sort before / after every node id and match nothing real.
// A 16-byte chunk that holds a position in [pos, end) lies inside the page of
// that position, so it is read whole; chunks entirely past end are not read.
__device__ __forceinline__ int4 merge_chunk(const int32_t* p, int pos, int end, int q, int& t0) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p + pos);
    t0 = pos - (int)((a & 15) >> 2);
    const int e = t0 + 4 * q;  // position of the chunk's first id
    int4 v = make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX);
    if (e < end) v = __ldg(reinterpret_cast<const int4*>(a & ~uintptr_t(15)) + q);
    if (e < pos) v.x = -1;
    if (e + 1 < pos) v.y = -1;
    if (e + 2 < pos) v.z = -1;
    if (e + 1 >= end) v.y = INT_MAX;
    if (e + 2 >= end) v.z = INT_MAX;
    if (e + 3 >= end) v.w = INT_MAX;
    return v;
}

__device__ __forceinline__ int32_t int4_at(const int4& v, int j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// Number of ids common to the ascending lists A[pa, ea) and B[pb, eb),
// leaving out the matched nodes m[j] for the bits j of neq (injectivity).
// Returns this lane's share; the warp's sum is the count. A is the shorter
// list. Each round loads a 128-id tile of A and a BV x 128-id tile of B
// (BV chosen from the length ratio, so that both tiles cover about the same
// id range and every load of the round is in flight at once), puts B's into
// `tile` (shared memory, MERGE_TILE ints of this warp), looks every id of
// A's tile up in it by binary search, and then advances both lists past the
// smaller of the two tiles' last ids (one tile is always used up): the
// merge-path step. The unused rest of the other tile is read again in the
// next round, from L1.
template <int BV>
__device__ unsigned merge_count_t(const int32_t* __restrict__ A, int pa, int ea, const int32_t* __restrict__ B,
                                  int pb, int eb, int32_t* tile, uint32_t neq, const int32_t* m, int lane) {
    constexpr int TB = 128 * BV;
    unsigned cnt = 0;
    while (pa < ea && pb < eb) {
        int ta, tb;
        const int4 va = merge_chunk(A, pa, ea, lane, ta);
        int4 vb[BV];
#pragma unroll
        for (int c = 0; c < BV; c++) vb[c] = merge_chunk(B, pb, eb, lane + 32 * c, tb);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < BV; c++) reinterpret_cast<int4*>(tile)[lane + 32 * c] = vb[c];
        __syncwarp();
        const int la = min(ea, ta + 128) - 1 - ta;  // tile index of A's last real id
        const int lb = min(eb, tb + TB) - 1 - tb;
        const int32_t lastA = __shfl_sync(FULL, int4_at(va, la & 3), la >> 2);
        const int32_t lim = min(lastA, tile[lb]);
        int na = 0, nb = 0;
#pragma unroll
        for (int c = 0; c < BV; c++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int32_t y = int4_at(vb[c], j);
                nb += __popc(__ballot_sync(FULL, y >= 0 && y <= lim));
            }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int32_t x = int4_at(va, j);
            const bool ok = x >= 0 && x <= lim;
            na += __popc(__ballot_sync(FULL, ok));
            if (ok) {
                int i = 0;  // number of tile ids below x (at most TB - 1)
#pragma unroll
                for (int s = TB / 2; s > 0; s >>= 1)
                    if (tile[i + s - 1] < x) i += s;
                bool f = tile[i] == x;
                for (uint32_t nm = neq; nm && f; nm &= nm - 1) f = x != m[__ffs(nm) - 1];
                cnt += f ? 1u : 0u;
            }
        }
        pa += na;
        pb += nb;
    }
    return cnt;
}

__device__ __forceinline__ unsigned merge_count(const int32_t* A, int pa, int ea, const int32_t* B, int pb, int eb,
                                                int32_t* tile, uint32_t neq, const int32_t* m, int lane) {
    const long long na = ea - pa, nb = eb - pb;
    if (nb >= 3 * na) return merge_count_t<4>(A, pa, ea, B, pb, eb, tile, neq, m, lane);
    if (nb >= 2 * na) return merge_count_t<2>(A, pa, ea, B, pb, eb, tile, neq, m, lane);
    return merge_count_t<1>(A, pa, ea, B, pb, eb, tile, neq, m, lane);
}

// ----------------------------------------------------------------- k_match

// Work and traffic counters of the instrumented (MODE_STATS) kernel, which
// takes exactly the code paths of the counting kernel.
//   bytes    algorithmic bytes: per list operand 8 B of offsets; 4 B per id
//            of a driver range scanned; for every other list the cheaper of
//            scanning it or probing it once per driver id by binary search,
//            4 B x min(|L|, run x ceil(log2(|L| + 1))), with |L| cut to the
//            driver range's ids where the kernel computes that cut; a bound
//            search in a list of L ids 4 B x ceil(log2(L + 1)); 8 B per
//            degree check.
//   touched  the bytes the kernel's chosen strategy moves at 32-byte-sector
//            granularity if nothing were cached: a merge both ranges, a
//            hash probe one sector, a binary search one sector per step
//            above the last sector, a list's offsets one sector.
struct Stats {
    unsigned long long bytes = 0, touched = 0, ext = 0, sets = 0, units = 0, leaf = 0;
};

__device__ __forceinline__ unsigned long long search_bytes(int len) { return 4ull * ceil_log2p1(len); }
__device__ __forceinline__ unsigned long long search_sectors(int len) {
    return (unsigned long long)max(1, ceil_log2p1(len) - 3);
}
__device__ __forceinline__ unsigned long long probe_bytes(long long cut_len, long long run, int len) {
    return 4ull * (unsigned long long)min(cut_len, run * ceil_log2p1(len));
}

// MODE_STATS, lane 0: a scan of `run` driver ids of set S against its probe
// lists (probe 0 cut to cut0 ids when cut0 >= 0).
template <int MODE>
__device__ __forceinline__ void account_scan(const LvState& S, long long run, Stats& st, int lane, long long cut0 = -1) {
    if (MODE != MODE_STATS || lane != 0 || run <= 0) return;
    if (!S.drv_shared) {
        st.bytes += 4ull * run;
        st.touched += 4ull * run;
    }
    for (int p = 0; p < S.nprobe; p++) {
        if ((S.probe_shared >> p) & 1) continue;
        const int len = S.phi[p];
        st.bytes += probe_bytes(p == 0 && cut0 >= 0 ? cut0 : len, run, len);
        st.touched += 32ull * run * (S.pT[p] ? 1ull : search_sectors(len));
    }
}

// Sets up level record L for the partial match in ws.m: operand lists (or a
// complete earlier set in their place), driver (the first shortest list),
// probes and the cut of the driver by the order bounds. MODE_STATS adds the
// offsets and bound searches to st, and with `whole` the scan of the whole
// cut range (levels that are always scanned whole).
template <int MODE>
__device__ void setup_lists(const XmLevel& L, const GraphDev& g, WarpSmem& ws, LvState& S, int lane, Stats& st,
                            bool whole) {
    int32_t lo, hi;
    level_bounds(L, ws.m, lo, hi);
    // lane i fetches operand i's list bounds and hash table, all in parallel;
    // the level's lists stay spread over the lanes (no per-thread array)
    ListRef mine{nullptr, 0, 0, nullptr, 0};
    if (lane < L.nops) mine = op_list(g, L.op_dir[lane], ws.m[L.op_level[lane]]);
    bool use_reuse = (L.reuse >= 1) && ws.st[L.reuse].complete;
    if (use_reuse && __popc(L.reuse_ops) == 1) {
        // a reused set that equals its single operand list adds nothing but
        // loses the list's hash index: take the list instead
        const int len_i = __shfl_sync(FULL, mine.len, __ffs(L.reuse_ops) - 1);
        if (len_i == ws.st[L.reuse].set_len) use_reuse = false;
    }
    // entries in order: the reused set (when used), then the operands it does
    // not cover; the driver is the first shortest entry
    const LvState& R = ws.st[use_reuse ? L.reuse : 0];
    const bool act = lane < L.nops && !(use_reuse && ((L.reuse_ops >> lane) & 1u));
    const unsigned amask = __ballot_sync(FULL, act);
    long long key = act ? (((long long)mine.len << 6) | (lane + 1)) : LLONG_MAX;
    for (int o = 16; o; o >>= 1) key = min(key, __shfl_xor_sync(FULL, key, o));
    if (use_reuse) key = min(key, (long long)R.set_len << 6);
    const int dord = (int)(key & 63);  // 0: the reused set; i + 1: operand i
    const int dlane = dord > 0 ? dord - 1 : 0;
    bool empty = __any_sync(FULL, act && mine.len == 0) || (use_reuse && R.set_len == 0);
    ListRef drv;
    drv.p = reinterpret_cast<const int32_t*>(__shfl_sync(FULL, reinterpret_cast<unsigned long long>(mine.p), dlane));
    drv.len = __shfl_sync(FULL, mine.len, dlane);
    drv.shared = 0;
    if (dord == 0) {
        drv.p = R.set_ptr;
        drv.len = R.set_len;
        drv.shared = R.set_shared;
    }
    int c0 = 0, c1 = drv.len;
    if (!empty) {
        if (lo >= 0) c0 = lbound(drv.p, 0, c1, lo + 1, drv.shared);
        if (hi != INT_MAX) c1 = lbound(drv.p, c0, c1, hi, drv.shared);
    }
    if (c0 >= c1) empty = true;
    // probes: the other entries, in order
    const bool reuse_probe = use_reuse && dord != 0;
    const unsigned pmask = amask & ~(dord > 0 ? 1u << dlane : 0u);
    if (act && !(dord > 0 && lane == dlane)) {
        const int np = (reuse_probe ? 1 : 0) + __popc(pmask & ((1u << lane) - 1u));
        S.probe[np] = mine.p;
        S.ptab[np] = mine.tab;
        S.pT[np] = mine.T;
        S.plo[np] = 0;
        S.phi[np] = mine.len;
    }
    if (lane == 0) {
        if (reuse_probe) {
            S.probe[0] = R.set_ptr;
            S.ptab[0] = nullptr;
            S.pT[0] = 0;
            S.plo[0] = 0;
            S.phi[0] = R.set_len;
        }
        S.drv = drv.p;
        S.drv_shared = drv.shared;
        S.nprobe = (reuse_probe ? 1 : 0) + __popc(pmask);
        S.probe_shared = reuse_probe && R.set_shared ? 1 : 0;
        S.c0 = c0;
        S.c1 = empty ? c0 : c1;
        S.drv_pos = c0;
        S.drv_end = empty ? c0 : c1;
        S.empty = empty;
        S.complete = 0;
        S.wcnt = S.wpos = S.it_hi = 0;
        if (MODE == MODE_STATS) {
            // offsets of every list entry (a shared set costs none), and the
            // driver's bound searches
            const int nlist = __popc(amask) + (use_reuse && !R.set_shared ? 1 : 0);
            st.bytes += 8ull * nlist;
            st.touched += 32ull * nlist;
            if (!drv.shared && drv.len > 0) {
                const int nsearch = (lo >= 0 ? 1 : 0) + (hi != INT_MAX ? 1 : 0);
                st.bytes += nsearch * search_bytes(drv.len);
                st.touched += 32ull * nsearch * search_sectors(drv.len);
            }
        }
    }
    __syncwarp();
    if (whole && !empty) account_scan<MODE>(S, c1 - c0, st, lane);
}

template <int MODE>
__device__ __forceinline__ void setup_level(const XmPlanDev& P, const GraphDev& g, WarpSmem& ws, int l, int lane,
                                            Stats& st, bool whole) {
    setup_lists<MODE>(P.lv[l], g, ws, ws.st[l], lane, st, whole);
}

// Runs the driver range [drv_pos, drv_end) of level l through probes and
// filters 32 ids at a time. With WINDOW the survivors are compacted into
// `win` (stopping when fewer than 32 slots are left); otherwise they are
// counted or emitted.
template <int MODE, bool WINDOW>
__device__ unsigned long long scan_level(const XmPlanDev& P, const XmLevel& L, const GraphDev& g, WarpSmem& ws,
                                         LvState& S, int l, int32_t* win, int W, int lane, const RunArgs& ra,
                                         Stats& st) {
    const bool dsh = S.drv_shared;
    const int np = S.nprobe;
    int32_t plo[XM_MAXOPS];
    for (int p = 0; p < np; p++) plo[p] = S.plo[p];
    int pos = S.drv_pos;
    const int end = S.drv_end;
    int wcnt = WINDOW ? S.wcnt : 0;
    unsigned long long leaf = 0;
    const int k = P.k;
    while (pos < end && (!WINDOW || wcnt + 32 <= W)) {
        const int i = pos + lane;
        const bool valid = i < end;
        const int32_t x = valid ? ld(S.drv, i, dsh) : INT_MAX;
        bool ok = valid;
        const int last_lane = min(31, end - 1 - pos);
        for (int p = 0; p < np; p++) {
            const uint32_t T = S.pT[p];
            if (T) {
                if (ok) ok = hash_has(S.ptab[p], T, x);
            } else {
                const bool psh = (S.probe_shared >> p) & 1;
                const int hi = S.phi[p];
                const int q = lbound(S.probe[p], plo[p], hi, x, psh);
                ok = ok && q < hi && ld(S.probe[p], q, psh) == x;
                plo[p] = __shfl_sync(FULL, q, last_lane);
            }
            if (__ballot_sync(FULL, ok) == 0) break;
        }
        if (ok) {
            for (uint32_t nm = L.neq_mask; nm; nm &= nm - 1)
                if (x == ws.m[__ffs(nm) - 1]) ok = false;
        }
        if (ok && L.ndiff) ok = passes_diffs(L, g, ws.m, x);
        if (WINDOW) {
            if (MODE == MODE_STATS && (L.dout_min > 0 || L.din_min > 0)) {
                const int checks = __popc(__ballot_sync(FULL, ok));
                if (lane == 0) {
                    st.bytes += 8ull * checks;
                    st.touched += 32ull * checks;
                }
            }
            if (ok) ok = passes_degree(g, x, L.dout_min, L.din_min);
        }
        const unsigned mask = __ballot_sync(FULL, ok);
        const int rank = __popc(mask & ((1u << lane) - 1));
        if (WINDOW) {
            if (ok) win[wcnt + rank] = x;
            wcnt += __popc(mask);
        } else if (MODE == MODE_EMIT) {
            const int c = __popc(mask);
            unsigned long long base = 0;
            if (lane == 0 && c) base = atomicAdd(ra.ctl + CTL_EMIT, (unsigned long long)c);
            base = __shfl_sync(FULL, base, 0);
            if (ok && base + rank < ra.capacity) {
                int32_t* o = ra.out + (base + rank) * (unsigned long long)k;
                for (int t = 0; t < l; t++) o[P.order[t]] = ws.m[t];
                o[P.order[l]] = x;
            }
            leaf += c;
        } else {
            leaf += __popc(mask);
        }
        pos += 32;
    }
    if (pos > end) pos = end;
    __syncwarp();
    if (lane == 0) {
        S.drv_pos = pos;
        for (int p = 0; p < np; p++) S.plo[p] = plo[p];
        if (WINDOW) S.wcnt = wcnt;
    }
    __syncwarp();
    return leaf;
}

// Last-level count when every probe list has a hash table: 128 driver ids
// per iteration (four per lane) with all four first-bucket probes issued
// before any is checked, so four sector reads per lane are in flight.
__device__ unsigned long long leaf_count_hashed(const XmLevel& L, WarpSmem& ws, LvState& S, int pos, int end,
                                                int lane) {
    const bool dsh = S.drv_shared;
    const int np = S.nprobe;
    unsigned long long cnt = 0;
    for (; pos < end; pos += 128) {
        int32_t x[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = pos + 32 * u + lane;
            ok[u] = i < end;
            x[u] = ok[u] ? ld(S.drv, i, dsh) : 0;
        }
        for (int p = 0; p < np; p++) {
            const int32_t* tab = S.ptab[p];
            const uint32_t T = S.pT[p];
            bool f[4], dn[4];
#pragma unroll
            for (int u = 0; u < 4; u++) dn[u] = ok[u] ? hash_first(tab, T, x[u], f[u]) : (f[u] = false, true);
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (ok[u]) ok[u] = dn[u] ? f[u] : hash_has(tab, T, x[u]);
            if (__ballot_sync(FULL, ok[0] || ok[1] || ok[2] || ok[3]) == 0) break;
        }
        for (uint32_t nm = L.neq_mask; nm; nm &= nm - 1) {
            const int32_t y = ws.m[__ffs(nm) - 1];
#pragma unroll
            for (int u = 0; u < 4; u++) ok[u] = ok[u] && x[u] != y;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) cnt += __popc(__ballot_sync(FULL, ok[u]));
    }
    return lane == 0 ? cnt : 0;
}

// Count (or emit) the candidates of level l's set S, already set up from
// record L, over the driver range [pos, end). The count is on lane 0.
// Counting with two lists (driver and one probe, no difference lists): the
// probe list is cut to the driver range's ids; when that cut is at most
// ra.merge_ratio times the driver range both are merged, else the driver's
// ids probe the list's hash table.
template <int MODE, bool LEAN = false>
__device__ unsigned long long leaf_tail(const XmPlanDev& P, const XmLevel& L, const GraphDev& g, WarpSmem& ws,
                                        LvState& S, int l, int lane, const RunArgs& ra, Stats& st, int pos, int end) {
    if (MODE == MODE_STATS && lane == 0) st.leaf += end - pos;
    if (MODE != MODE_EMIT && S.nprobe == 0 && L.ndiff == 0) {
        // A single list: its size, minus already matched nodes inside it.
        unsigned long long c = end - pos;
        for (uint32_t nm = L.neq_mask; nm; nm &= nm - 1) {
            const int32_t y = ws.m[__ffs(nm) - 1];
            const int q = lbound(S.drv, pos, end, y, S.drv_shared);
            if (q < end && ld(S.drv, q, S.drv_shared) == y) c--;
            if (MODE == MODE_STATS && lane == 0 && !S.drv_shared) {
                st.bytes += search_bytes(end - pos);
                st.touched += 32ull * search_sectors(end - pos);
            }
        }
        return lane == 0 ? c : 0;
    }
    const long long run = end - pos;
    if (MODE != MODE_EMIT && L.ndiff == 0) {
        const bool global = !S.drv_shared && S.probe_shared == 0;
        long long cut0 = -1;
        if (MODE == MODE_STATS && S.nprobe == 1 && global) {
            // accounting only: the probe list cut to the driver range's ids
            int pb, eb;
            warp_lbound2(S.probe[0], 0, S.phi[0], __ldg(S.drv + pos), 0, S.phi[0], __ldg(S.drv + end - 1) + 1, pb,
                         eb, lane);
            cut0 = eb - pb;
        }
        if (!LEAN && S.nprobe == 1 && global && ra.merge_ratio > 0 && run >= MERGE_MIN_RUN &&
            (long long)S.phi[0] <= (long long)ra.merge_ratio * run) {
            // the whole probe list is within the ratio: merged whole, no cut
            if (MODE == MODE_STATS && lane == 0) {
                st.bytes += 4ull * run + probe_bytes(cut0, run, S.phi[0]);
                st.touched += 4ull * (run + S.phi[0]) + 64;
            }
            unsigned c = merge_count(S.drv, pos, end, S.probe[0], 0, S.phi[0], ws.mtile, L.neq_mask, ws.m, lane);
            c = warp_sum(c);
            return lane == 0 ? c : 0;
        }
        account_scan<MODE>(S, run, st, lane, cut0);
        bool hashed = global;
        for (int p = 0; p < S.nprobe && hashed; p++) hashed = S.pT[p] != 0;
        if (hashed) return leaf_count_hashed(L, ws, S, pos, end, lane);
    } else {
        account_scan<MODE>(S, run, st, lane);
    }
    if (lane == 0) {
        S.drv_pos = pos;
        S.drv_end = end;
    }
    __syncwarp();
    unsigned long long r = scan_level<MODE, false>(P, L, g, ws, S, l, nullptr, 0, lane, ra, st);
    return lane == 0 ? r : 0;
}

// Count (or emit) the candidates of the last level l >= 2, optionally only
// the sub-range [c0 + ra_pos, c0 + ra_pos + ra_len) of its cut driver range.
template <int MODE, bool LEAN = false>
__device__ unsigned long long leaf_level(const XmPlanDev& P, const GraphDev& g, WarpSmem& ws, int l, int lane,
                                         const RunArgs& ra, Stats& st, int ra_pos = 0, int ra_len = -1) {
    setup_level<MODE>(P, g, ws, l, lane, st, false);
    LvState& S = ws.st[l];
    if (S.empty) return 0;
    const int pos = ra_len < 0 ? S.c0 : min(S.c1, S.c0 + ra_pos);
    const int end = ra_len < 0 ? S.c1 : min(S.c1, pos + ra_len);
    if (pos >= end) return 0;
    return leaf_tail<MODE, LEAN>(P, P.lv[l], g, ws, S, l, lane, ra, st, pos, end);
}

// Plans whose last level k - 1 intersects exactly two operand lists, one of
// a level before k - 2 (F, the same for every candidate of level k - 2) and
// one of level k - 2 itself (V, each candidate's own list), with no reuse and
// no difference lists, count their last level a batch of level-(k-2)
// candidates at a time (leaf_batch). Returns F's operand index, or -1.
__host__ __device__ inline int batch_leaf_fixed_op(const XmPlanDev& P) {
    if (P.k < 4) return -1;
    const XmLevel& L = P.lv[P.k - 1];
    const int l = P.k - 2;
    if (L.nops != 2 || L.ndiff != 0 || L.reuse >= 1) return -1;
    const bool v0 = L.op_level[0] == l, v1 = L.op_level[1] == l;
    if (v0 == v1) return -1;
    return v0 ? 1 : 0;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ const T* shfl_ptr(const T* p, int src) {
    return reinterpret_cast<const T*>(__shfl_sync(FULL, reinterpret_cast<unsigned long long>(p), src));
}

// The last level k - 1 of the nb <= 32 partial matches m_0..m_{l-1}, x_i
// (l = k - 2; lane i holds candidate x_i = cand[i]): each counts |F cap
// V(x_i)| within the order bounds, minus matched nodes, F being the batch's
// common operand list (cut once per batch) and V(x_i) lane i's own list (cut
// per lane). Pairs whose shorter range has at least MERGE_MIN_RUN ids and
// whose longer range is at most ra.merge_ratio times as long are merged, one
// pair at a time by the whole warp. The other pairs are counted together:
// the ids of their shorter ranges form one flattened index space that the
// lanes walk LEAF_PPL x 32 ids per round, each id probing the other list of
// its own pair (its hash table, or a binary search in a list too short for
// one) while the next round's ids are already being read, so a warp keeps
// its probes in flight however the ids are spread over the pairs. Returns
// the lane's share of the count.
template <int MODE>
__device__ unsigned long long leaf_batch(const XmPlanDev& P, const GraphDev& g, WarpSmem& ws, int iF,
                                         const int32_t* cand, bool cand_shared, int nb, int lane, const RunArgs& ra,
                                         Stats& st) {
    const int l = P.k - 2;
    const XmLevel& L = P.lv[P.k - 1];
    const int iV = 1 - iF;
    const uint32_t below = (1u << l) - 1;
    // the common list F and the order bounds of levels before l
    const ListRef F = op_list(g, L.op_dir[iF], ws.m[L.op_level[iF]]);
    int32_t lo = -1, hi = INT_MAX;
    for (uint32_t a = L.lo_mask & below; a; a &= a - 1) lo = max(lo, ws.m[__ffs(a) - 1]);
    for (uint32_t b = L.hi_mask & below; b; b &= b - 1) hi = min(hi, ws.m[__ffs(b) - 1]);
    int f0 = 0, f1 = F.len;
    if (F.len > 0 && lo >= 0) f0 = lbound(F.p, 0, f1, lo + 1, false);
    if (F.len > 0 && hi != INT_MAX) f1 = lbound(F.p, f0, f1, hi, false);
    const bool lx = (L.lo_mask >> l) & 1u, hx = (L.hi_mask >> l) & 1u;
    // lane i: candidate x_i, its list V and the cuts of both lists
    ListRef V{nullptr, 0, 0, nullptr, 0};
    int a0 = f0, a1 = f0, v0 = 0, v1 = 0, nsV = 0, nsF = 0;
    if (lane < nb && f0 < f1) {
        const int32_t x = ld(cand, lane, cand_shared);
        V = op_list(g, L.op_dir[iV], x);
        const int32_t lo_i = lx ? max(lo, x) : lo, hi_i = hx ? min(hi, x) : hi;
        nsV = (lo_i >= 0 ? 1 : 0) + (hi_i != INT_MAX ? 1 : 0);
        nsF = (lx && x > lo ? 1 : 0) + (hx && x < hi ? 1 : 0);
        v1 = V.len;
        if (v1 > 0 && lo_i >= 0) v0 = lbound(V.p, 0, v1, lo_i + 1, false);
        if (v0 < v1 && hi_i != INT_MAX) v1 = lbound(V.p, v0, v1, hi_i, false);
        a1 = f1;
        if (lx && x > lo) a0 = lbound(F.p, f0, f1, x + 1, false);
        if (hx && x < hi) a1 = lbound(F.p, a0, f1, x, false);
        if (v1 < v0) v1 = v0;
        if (a1 < a0) a1 = a0;
    }
    const int na = a1 - a0, nv = v1 - v0;
    const bool fdrv = na <= nv;                 // F's range drives, V is probed
    const int run = (na == 0 || nv == 0) ? 0 : min(na, nv);
    const int other = max(na, nv);
    const bool merge = ra.merge_ratio > 0 && run >= MERGE_MIN_RUN && (long long)other <= (long long)ra.merge_ratio * run;
    const uint32_t neq = L.neq_mask & below;    // x_i itself is never in its own list V(x_i)
    if (MODE == MODE_STATS) {
        // offsets of V (F's once), bound searches, the level's formula over the
        // cut ranges, and the bytes each pair's strategy moves
        unsigned long long b = 0, t = 0;
        if (lane < nb && f0 < f1) {
            b += 8 + nsV * search_bytes(V.len) + nsF * search_bytes(f1 - f0);
            t += 32 + 32ull * (nsV * search_sectors(V.len) + nsF * search_sectors(f1 - f0));
            if (run) {
                const int plen = fdrv ? V.len : F.len;
                b += 4ull * run + probe_bytes(other, run, plen);
                if (merge) t += 4ull * (na + nv) + 64;
                else t += 4ull * run + 32ull * run * ((fdrv ? V.T : F.T) ? 1ull : search_sectors(other));
            }
        }
        b = warp_sum64(b);
        t = warp_sum64(t);
        if (lane == 0) {
            const int nsF = (lo >= 0 ? 1 : 0) + (hi != INT_MAX ? 1 : 0);  // F's cut, once per batch
            st.bytes += b + 8 + nsF * search_bytes(F.len);
            st.touched += t + 32 + 32ull * nsF * search_sectors(F.len);
        }
        const unsigned long long e = warp_sum64(run);
        if (lane == 0) st.leaf += e;
    }
    unsigned long long cnt = 0;
    // long pairs of similar length: merged, the whole warp per pair
    for (unsigned mm = __ballot_sync(FULL, merge); mm; mm &= mm - 1) {
        const int i = __ffs(mm) - 1;
        const int32_t* Vp = shfl_ptr(V.p, i);
        const int b0 = __shfl_sync(FULL, v0, i), b1 = __shfl_sync(FULL, v1, i);
        const int c0 = __shfl_sync(FULL, a0, i), c1 = __shfl_sync(FULL, a1, i);
        if (c1 - c0 <= b1 - b0)
            cnt += merge_count(F.p, c0, c1, Vp, b0, b1, ws.mtile, neq, ws.m, lane);
        else
            cnt += merge_count(Vp, b0, b1, F.p, c0, c1, ws.mtile, neq, ws.m, lane);
    }
    // the rest: one flattened space of driver ids
    const int r = merge ? 0 : run;
    int pend = r;  // inclusive prefix of r over the lanes
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, pend, o);
        if (lane >= o) pend += y;
    }
    const int total = __shfl_sync(FULL, pend, 31);
    if (total == 0) return cnt;
    // driver ids of pair i: dptr[j], j = t - pre_i for flattened positions
    // t in [pre_i, pend_i); the probe: a hash table of ptn > 0 slots at ptab,
    // or -ptn ascending ids at ptab (binary search)
    const int pre = pend - r;
    const int32_t* dptr = fdrv ? F.p + a0 : V.p + v0;
    const int32_t* ptab;
    int ptn;
    if (fdrv) {
        ptab = V.T ? V.tab : V.p + v0;
        ptn = V.T ? (int)V.T : -nv;
    } else {
        ptab = F.T ? F.tab : F.p + a0;
        ptn = F.T ? (int)F.T : -na;
    }
    // Each lane walks the flattened positions lane, lane + 32, ... and keeps
    // the index of the pair its position falls in (pairs only ever advance),
    // reading a pair's pointers from the warp's shared table when it moves
    // on: no shuffles per probe.
    constexpr int PPL = LEAF_PPL;
    ws.lp[lane] = LeafPair{dptr - pre, ptab, pend, ptn};
    __syncwarp();
    int pi = 0, pe = ws.lp[0].end;
    // software pipeline: the driver ids of the next round are loaded before
    // this round's buckets, so the two dependent reads of a probe overlap
    // across rounds
    // the current pair's pointers stay in registers; the shared table is read
    // only when a lane moves on to the next pair
    const int32_t* cd = ws.lp[0].d;
    const int32_t* ctab = ws.lp[0].tab;
    int cn = ws.lp[0].n;
    int32_t xn[PPL];
    const int32_t* tn[PPL];
    int nn[PPL];
    bool okn[PPL];
#pragma unroll
    for (int u = 0; u < PPL; u++) {
        const int t = 32 * u + lane;
        okn[u] = t < total;
        xn[u] = -1;
        tn[u] = nullptr;
        nn[u] = 0;
        if (okn[u]) {
            if (pe <= t) {
                do { pe = ws.lp[++pi].end; } while (pe <= t);
                cd = ws.lp[pi].d;
                ctab = ws.lp[pi].tab;
                cn = ws.lp[pi].n;
            }
            xn[u] = __ldg(cd + t);
            tn[u] = ctab;
            nn[u] = cn;
        }
    }
    for (int t0 = 0; t0 < total; t0 += 32 * PPL) {
        int32_t x[PPL];
        const int32_t* tb[PPL];
        int nb_[PPL];
        bool ok[PPL];
#pragma unroll
        for (int u = 0; u < PPL; u++) {
            x[u] = xn[u];
            tb[u] = tn[u];
            nb_[u] = nn[u];
            ok[u] = okn[u];
            const int t = t0 + 32 * PPL + 32 * u + lane;
            okn[u] = t < total;
            if (okn[u]) {
                if (pe <= t) {
                    do { pe = ws.lp[++pi].end; } while (pe <= t);
                    cd = ws.lp[pi].d;
                    ctab = ws.lp[pi].tab;
                    cn = ws.lp[pi].n;
                }
                xn[u] = __ldg(cd + t);
                tn[u] = ctab;
                nn[u] = cn;
            }
        }
        bool f[PPL], dn[PPL];
#pragma unroll
        for (int u = 0; u < PPL; u++) {
            f[u] = false;
            dn[u] = true;
            if (ok[u]) {
                if (nb_[u] > 0) {
                    dn[u] = hash_first(tb[u], (uint32_t)nb_[u], x[u], f[u]);
                } else {
                    const int r0 = lbound(tb[u], 0, -nb_[u], x[u], false);
                    f[u] = r0 < -nb_[u] && __ldg(tb[u] + r0) == x[u];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < PPL; u++) {
            if (!dn[u]) f[u] = hash_has(tb[u], (uint32_t)nb_[u], x[u]);
            for (uint32_t nm = neq; nm && f[u]; nm &= nm - 1) f[u] = x[u] != ws.m[__ffs(nm) - 1];
            cnt += f[u] ? 1 : 0;
        }
    }
    __syncwarp();
    return cnt;
}

// The walk below a four-level plan's second level when its last level is a
// batched two-list level (explore's behaviour for that shape, without the
// deeper-level and other leaf paths): refill level 2's window from its
// driver range, count each batch of up to 32 candidates with leaf_batch.
template <int MODE>
__device__ bool walk_last2(const XmPlanDev& P, const GraphDev& g, WarpSmem& ws, int32_t* win, int W, int iF,
                           int lane, const RunArgs& ra, unsigned long long& acc, Stats& st, const Budget& budget) {
    LvState& S = ws.st[2];
    unsigned steps = 0;
    for (;;) {
        if ((++steps & 255u) == 0 && budget.expired(lane)) return false;
        if (S.wpos >= S.it_hi) {
            if (S.complete || S.drv_pos >= S.drv_end) return true;
            if (lane == 0) { S.wcnt = 0; S.wpos = 0; }
            __syncwarp();
            scan_level<MODE, true>(P, P.lv[2], g, ws, S, 2, win, W, lane, ra, st);
            if (lane == 0) S.it_hi = S.wcnt;
            __syncwarp();
            continue;
        }
        const int nb = min(32, S.it_hi - S.wpos);
        acc += leaf_batch<MODE>(P, g, ws, iF, S.it_ptr + S.wpos, S.it_shared, nb, lane, ra, st);
        if (MODE == MODE_STATS && lane == 0) {
            st.ext += nb;
            st.sets += nb;
        }
        __syncwarp();
        if (lane == 0) S.wpos += nb;
        __syncwarp();
    }
}

// Adds a 128-bit value on lane 0 to the lane's running count, or straight to
// the 128-bit counter when the 64-bit count would wrap.
__device__ __forceinline__ void add_count(unsigned long long& acc, unsigned __int128 v, unsigned long long* counter,
                                          int lane) {
    if (lane != 0 || v == 0) return;
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    if (hi == 0 && acc + lo >= acc) {
        acc += lo;
        return;
    }
    const unsigned long long old = atomicAdd(counter, lo);
    const unsigned long long carry = (old + lo < old) ? 1 : 0;
    if (hi + carry) atomicAdd(counter + 1, hi + carry);
}

// Leaf product at level l = prod_p (Sec. 5.3): the sizes of the product
// sets pv[] under the partial match m_0..m_{l-1}, combined into the number
// of tuples of pairwise distinct nodes (see XmPlanDev).
template <int MODE>
__device__ __noinline__ unsigned __int128 leaf_product(const XmPlanDev& P, const XmLevel* __restrict__ pv,
                                                       const GraphDev& g, WarpSmem& ws, int l, int lane,
                                                       const RunArgs& ra, Stats& st) {
    LvState& S = ws.st[l];
    auto size_of = [&](int i) -> unsigned long long {
        const XmLevel& V = pv[i];
        setup_lists<MODE>(V, g, ws, S, lane, st, false);
        unsigned long long c = 0;
        if (!S.empty) c = leaf_tail<MODE>(P, V, g, ws, S, l, lane, ra, st, S.c0, S.c1);
        return __shfl_sync(FULL, c, 0);
    };
    typedef unsigned __int128 u128;
    const int r = P.prod_r;
    if (P.prod_kind == XM_PROD_CHOOSE) {
        const unsigned long long c = size_of(0);
        if (c < (unsigned long long)r) return 0;
        // C(c, r) = prod_{i<r} (c - i) / (i + 1), exact after every step
        u128 t = 1;
        for (int i = 0; i < r; i++) t = t * (u128)(c - i) / (u128)(i + 1);
        return t;
    }
    if (r == 2) {
        const unsigned long long a = size_of(0);
        if (!a) return 0;
        const unsigned long long b = size_of(1);
        if (!b) return 0;
        const unsigned long long ab = size_of(2);
        return (u128)a * b - ab;
    }
    // r == 3; set s - 1 holds the intersection over the members in mask s
    const unsigned long long s1 = size_of(0);
    if (!s1) return 0;
    const unsigned long long s2 = size_of(1);
    if (!s2) return 0;
    const unsigned long long s4 = size_of(3);
    if (!s4) return 0;
    const unsigned long long s3 = size_of(2), s5 = size_of(4), s6 = size_of(5), s7 = size_of(6);
    return (u128)s1 * s2 * s4 - (u128)s3 * s4 - (u128)s5 * s2 - (u128)s6 * s1 + (u128)2 * s7;
}

// Sets up level nl and builds its first window `win`; false when empty.
template <int MODE>
__device__ bool descend(const XmPlanDev& P, const GraphDev& g, WarpSmem& ws, int32_t* win, int W, int nl, int lane,
                        const RunArgs& ra, Stats& st) {
    setup_level<MODE>(P, g, ws, nl, lane, st, true);
    if (MODE == MODE_STATS && lane == 0) st.sets++;
    LvState& N = ws.st[nl];
    if (N.empty) return false;
    scan_level<MODE, true>(P, P.lv[nl], g, ws, N, nl, win, W, lane, ra, st);
    if (lane == 0) {
        N.complete = N.drv_pos >= N.drv_end;
        N.it_ptr = win;
        N.it_shared = 1;
        N.wpos = 0;
        N.it_hi = N.wcnt;
        N.set_ptr = win;
        N.set_len = N.wcnt;
        N.set_shared = 1;
    }
    __syncwarp();
    return true;
}

// Depth-first extension below the first level (Alg. 2 Explore): level 1's
// iteration state is set; levels wl0.. use windows wins + (l - wl0) * W;
// the last level is counted (or emitted) into acc. With PROD (counting with
// a leaf product, sets ra.pv) the walk ends at level prod_p, which adds the
// product (values past 64 bits go straight to *counter).
template <int MODE, bool PROD, bool LEAN = false>
__device__ bool explore(const XmPlanDev& P, const GraphDev& g, WarpSmem& ws, int32_t* wins, int W, int wl0, int lane,
                        const RunArgs& ra, unsigned long long& acc, unsigned long long* counter, Stats& st,
                        const Budget& budget, int l0 = 1) {
    const int k = PROD ? P.prod_p + 1 : P.k;
    // two-list last levels are counted a batch of candidates at a time
    const int iF = (!PROD && !LEAN && MODE != MODE_EMIT) ? batch_leaf_fixed_op(P) : -1;
    int l = l0;
    unsigned steps = 0;
    while (l >= l0) {
        if ((++steps & 255u) == 0 && budget.expired(lane)) return false;
        LvState& S = ws.st[l];
        if (S.wpos >= S.it_hi) {
            if (S.complete || S.drv_pos >= S.drv_end) { l--; continue; }
            if (lane == 0) { S.wcnt = 0; S.wpos = 0; }
            __syncwarp();
            scan_level<MODE, true>(P, P.lv[l], g, ws, S, l, wins + (size_t)(l - wl0) * W, W, lane, ra, st);
            if (lane == 0) S.it_hi = S.wcnt;
            __syncwarp();
            continue;
        }
        if (iF >= 0 && l + 1 == k - 1) {
            const int nb = min(32, S.it_hi - S.wpos);
            acc += leaf_batch<MODE>(P, g, ws, iF, S.it_ptr + S.wpos, S.it_shared, nb, lane, ra, st);
            if (MODE == MODE_STATS && lane == 0) {
                st.ext += nb;
                st.sets += nb;
            }
            __syncwarp();
            if (lane == 0) S.wpos += nb;
            __syncwarp();
            continue;
        }
        const int32_t x = ld(S.it_ptr, S.wpos, S.it_shared);
        __syncwarp();
        if (lane == 0) { S.wpos++; ws.m[l] = x; }
        __syncwarp();
        if (MODE == MODE_STATS && lane == 0) st.ext++;
        if (l + 1 == k - 1) {
            if (PROD)
                add_count(acc, leaf_product<MODE>(P, ra.pv, g, ws, l + 1, lane, ra, st), counter, lane);
            else
                acc += leaf_level<MODE, LEAN>(P, g, ws, l + 1, lane, ra, st);
            if (MODE == MODE_STATS && lane == 0) st.sets++;
            continue;
        }
        if (descend<MODE>(P, g, ws, wins + (size_t)(l + 1 - wl0) * W, W, l + 1, lane, ra, st)) l++;
    }
    return true;
}

// 128-bit warp reduction of per-lane counts, added to counter[0..1].
__device__ __forceinline__ void flush_count(unsigned long long acc, unsigned long long* counter, int lane) {
    unsigned long long lo = acc, hi = 0;
    for (int off = 16; off; off >>= 1) {
        unsigned long long olo = __shfl_down_sync(FULL, lo, off);
        unsigned long long ohi = __shfl_down_sync(FULL, hi, off);
        unsigned long long s = lo + olo;
        hi += ohi + (s < lo ? 1 : 0);
        lo = s;
    }
    if (lane == 0 && (lo | hi)) {
        unsigned long long old = atomicAdd(counter, lo);
        unsigned long long carry = (old + lo < old) ? 1 : 0;
        if (hi + carry) atomicAdd(counter + 1, hi + carry);
    }
}

// Guided self-scheduling: lane 0 takes a batch of units proportional to
// what is left, at most maxb; returns [start, start + cnt) on every lane
// (cnt <= 0: done, or the budget is spent).
__device__ __forceinline__ void grab_units(unsigned long long* head, long long total, int nwarps, int lane,
                                           long long& start, int& cnt, const Budget& budget, int maxb = 64) {
    if (budget.expired(lane)) {
        start = total;
        cnt = 0;
        return;
    }
    long long s0 = 0;
    int c = 0;
    if (lane == 0) {
        unsigned long long seen = *((volatile unsigned long long*)head);
        long long left = total - (long long)seen;
        int batch = left > 0 ? (int)min((long long)maxb, max(1ll, left / (8ll * nwarps))) : 1;
        unsigned long long s = atomicAdd(head, (unsigned long long)batch);
        s0 = (long long)s >= total ? total : (long long)s;
        c = (int)min((long long)batch, total - s0);
    }
    start = __shfl_sync(FULL, s0, 0);
    cnt = __shfl_sync(FULL, c, 0);
}

// Start of start node i's first-level set in l1set.
__device__ __forceinline__ int set_start(const RunArgs& ra, int i) {
    return __ldg(ra.chunk_cnt + __ldg(ra.root_chunks + i));
}

// Second-level driver and its cut range for the partial match (m0, m1),
// computed by one thread exactly as setup_level does it for a warp: the
// same lists in the same order (the first level's complete set in place of
// the operands it covers, unless it equals its single operand list), the
// first shortest list as driver, the cut by the order bounds.
__device__ void level2_cut(const XmPlanDev& P, const GraphDev& g, int32_t m0, int32_t m1, const int32_t* set_ptr,
                           int set_len, int& c0, int& c1) {
    const XmLevel& L = P.lv[2];
    const int32_t m[2] = {m0, m1};
    int32_t lo = -1, hi = INT_MAX;
    for (uint32_t a = L.lo_mask; a; a &= a - 1) lo = max(lo, m[__ffs(a) - 1]);
    for (uint32_t b = L.hi_mask; b; b &= b - 1) hi = min(hi, m[__ffs(b) - 1]);
    bool use_reuse = L.reuse == 1;
    if (use_reuse && __popc(L.reuse_ops) == 1) {
        const int i = __ffs(L.reuse_ops) - 1;
        if (op_list(g, L.op_dir[i], m[L.op_level[i]]).len == set_len) use_reuse = false;
    }
    const int32_t* dp = nullptr;
    int dlen = INT_MAX;
    bool empty = false;
    if (use_reuse) {
        dp = set_ptr;
        dlen = set_len;
        if (set_len == 0) empty = true;
    }
    for (int i = 0; i < L.nops; i++) {
        if (use_reuse && ((L.reuse_ops >> i) & 1u)) continue;
        const ListRef r = op_list(g, L.op_dir[i], m[L.op_level[i]]);
        if (r.len == 0) empty = true;
        if (r.len < dlen) { dp = r.p; dlen = r.len; }
    }
    c0 = 0;
    c1 = dlen;
    if (!empty) {
        if (lo >= 0) c0 = lbound(dp, 0, c1, lo + 1, false);
        if (hi != INT_MAX) c1 = lbound(dp, c0, c1, hi, false);
    }
    if (empty || c1 < c0) c1 = c0;
}

// Second-level driver positions per work unit below the first-level node m1
// of start node m0, for a walk of ke levels: LEAF_UNIT when the second level
// is the last; for four levels whose last one intersects a list of node m0
// or m1 (the same for every leaf of the unit) with the leaf candidate's own
// list, fewer when that common list is longer than HEAVY_LIST ids -- each
// leaf costs about its length, and a hub's leaves would otherwise stay
// together in one warp; else `unit`.
__device__ __forceinline__ int l2_piece(const XmPlanDev& P, const GraphDev& g, int ke, int unit, int32_t m0,
                                        int32_t m1) {
    if (ke == 3) return LEAF_UNIT;
    if (ke == 4 && P.k == 4) {
        const int iF = batch_leaf_fixed_op(P);
        if (iF >= 0) {
            const XmLevel& L = P.lv[3];
            const int32_t v = L.op_level[iF] ? m1 : m0;
            const int32_t* off = L.op_dir[iF] == XM_DIR_OUT ? g.out_off : g.in_off;
            const long long len = __ldg(off + v + 1) - __ldg(off + v);
            if (len > HEAVY_LIST) return max(1, (int)((long long)unit * HEAVY_LIST / len));
        }
    }
    return unit;
}

// Work units per first-level candidate (patterns of three or more
// vertices): its second-level driver range cut into pieces (l2_piece), so
// the work below one hub is spread over many warps. One thread per
// candidate.
#ifndef XM_BATCH_TU
__global__ void k_l2_units(const XmPlanDev* __restrict__ plan_g, RunArgs ra) {
    __shared__ __align__(16) unsigned char pbuf[plan_bytes(XM_MAXK)];
    XmPlanDev& P = *reinterpret_cast<XmPlanDev*>(pbuf);
    plan_to_smem(P, plan_g);
    const int E = set_start(ra, ra.n_idx);
    const int ke = ra.pv ? P.prod_p + 1 : P.k;  // levels the count walks
    // the first-level candidates and a terminal zero: the scan reads no further
    if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<int32_t*>(ra.ctl + CTL_ELEN) = E;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= E; e += gridDim.x * blockDim.x) {
        int u = 0;
        if (e < E) {
            const int i = __ldg(ra.l1root + e);
            const int s0 = set_start(ra, i), s1 = set_start(ra, i + 1);
            const int32_t m0 = root_node(ra, i), m1 = __ldg(ra.l1set + e);
            int c0, c1;
            level2_cut(P, ra.g, m0, m1, ra.l1set + s0, s1 - s0, c0, c1);
            const int per = l2_piece(P, ra.g, ke, ra.unit, m0, m1);
            u = (c1 - c0 + per - 1) / per;
        }
        ra.e_units[e] = u;
    }
}
#endif

// Three-vertex plans, count mode: the last level of the partial match
// (m0, m1) over the driver piece [pos0, pos0 + per) of its cut range, with
// the lists in registers instead of a level state in shared memory (the
// general path's per-unit set-up dominated these kernels' shared-memory and
// local-memory traffic). Chooses the driver and cut exactly as setup_level
// and level2_cut do, so the pieces match the work units. With one probe
// list, the list is cut to the piece's ids and merged with the piece when
// the cut is at most ra.merge_ratio times the piece (else hashed probes).
// Returns false (nothing counted) when the level needs the general path:
// difference lists, more than two probe lists, or a probe without a hash
// table that is not merged. Survivors are counted per lane into acc.
template <int MODE, bool LEAN>
__device__ __forceinline__ bool leaf3_direct(const XmPlanDev& P, const GraphDev& g, int32_t m0, int32_t m1,
                                             const int32_t* set, int set_len, int pos0, int per, int lane,
                                             unsigned long long& acc, const RunArgs& ra, WarpSmem& ws, Stats& st) {
    const XmLevel& L = P.lv[2];
    if (L.ndiff) return false;
    ListRef mine{nullptr, 0, 0, nullptr, 0};
    if (lane < L.nops) mine = op_list(g, L.op_dir[lane], L.op_level[lane] ? m1 : m0);
    bool use_reuse = L.reuse == 1;
    if (use_reuse && __popc(L.reuse_ops) == 1) {
        const int len_i = __shfl_sync(FULL, mine.len, __ffs(L.reuse_ops) - 1);
        if (len_i == set_len) use_reuse = false;
    }
    // lists in setup_level's order: the reused set, then the remaining
    // operands; the driver is the first shortest
    int dsrc = -2, dlen = INT_MAX, nlists = 0;
    bool empty = false;
    if (use_reuse) {
        dsrc = -1;
        dlen = set_len;
        nlists = 1;
        empty = set_len == 0;
    }
    for (int i = 0; i < L.nops; i++) {
        if (use_reuse && ((L.reuse_ops >> i) & 1u)) continue;
        const int len = __shfl_sync(FULL, mine.len, i);
        nlists++;
        if (len == 0) empty = true;
        if (len < dlen) {
            dlen = len;
            dsrc = i;
        }
    }
    if (nlists > 3 || (use_reuse && dsrc != -1)) return false;  // > 2 probes, or the set as a probe
    // probes: the operands other than the driver
    const int32_t* tab[2] = {nullptr, nullptr};
    uint32_t T[2] = {0, 0};
    int plen[2] = {0, 0};
    int np = 0, psrc = -1;
    bool hashed = true;
    for (int i = 0; i < L.nops; i++) {
        if (i == dsrc || (use_reuse && ((L.reuse_ops >> i) & 1u))) continue;
        const uint32_t Ti = __shfl_sync(FULL, mine.T, i);
        const int32_t* ti =
            reinterpret_cast<const int32_t*>(__shfl_sync(FULL, reinterpret_cast<unsigned long long>(mine.tab), i));
        if (!Ti) hashed = false;
        if (np < 2) {
            tab[np] = ti;
            T[np] = Ti;
            plen[np] = __shfl_sync(FULL, mine.len, i);
        }
        if (np == 0) psrc = i;
        np++;
    }
    const bool try_merge = !LEAN && np == 1 && ra.merge_ratio > 0;
    if (!hashed && !try_merge) return false;
    const int32_t* dp =
        dsrc == -1 ? set
                   : reinterpret_cast<const int32_t*>(__shfl_sync(FULL, reinterpret_cast<unsigned long long>(mine.p), dsrc));
    if (MODE == MODE_STATS && lane == 0) {
        st.bytes += 8ull * (nlists - (use_reuse ? 1 : 0));
        st.touched += 32ull * (nlists - (use_reuse ? 1 : 0));
    }
    if (empty) return true;
    const int32_t m[2] = {m0, m1};
    int32_t lo, hi;
    level_bounds(L, m, lo, hi);
    int c0 = 0, c1 = dlen;
    if (lo >= 0) c0 = lbound(dp, 0, c1, lo + 1, false);
    if (hi != INT_MAX) c1 = lbound(dp, c0, c1, hi, false);
    if (MODE == MODE_STATS && lane == 0) {
        const int ns = (lo >= 0 ? 1 : 0) + (hi != INT_MAX ? 1 : 0);
        st.bytes += ns * search_bytes(dlen);
        st.touched += 32ull * ns * search_sectors(dlen);
    }
    const int pos = min(c1, c0 + pos0);
    const int end = min(c1, pos + per);
    if (pos >= end) return true;
    // matched nodes that may lie in the candidates (-1: none)
    const int32_t y0 = (L.neq_mask & 1u) ? m0 : -1;
    const int32_t y1 = (L.neq_mask & 2u) ? m1 : -1;
    const long long run = end - pos;
    if (MODE == MODE_STATS && lane == 0) st.leaf += run;
    if (np == 0) {
        if (lane == 0) {
            long long c = run;
            for (int32_t y : {y0, y1}) {
                if (y < 0) continue;
                const int q = lbound(dp, pos, end, y, false);
                if (q < end && __ldg(dp + q) == y) c--;
                if (MODE == MODE_STATS) {
                    st.bytes += search_bytes(end - pos);
                    st.touched += 32ull * search_sectors(end - pos);
                }
            }
            acc += c;
        }
        return true;
    }
    long long cut0 = -1;
    if (!LEAN && np == 1) {
        const int32_t* B = reinterpret_cast<const int32_t*>(
            __shfl_sync(FULL, reinterpret_cast<unsigned long long>(mine.p), psrc));
        const int blen = plen[0];
        if (MODE == MODE_STATS) {
            // accounting only: the probe list cut to the piece's ids
            int pb, eb;
            warp_lbound2(B, 0, blen, __ldg(dp + pos), 0, blen, __ldg(dp + end - 1) + 1, pb, eb, lane);
            cut0 = eb - pb;
        }
        if (try_merge && run >= MERGE_MIN_RUN && (long long)blen <= (long long)ra.merge_ratio * run) {
            // the whole probe list is within the ratio: merged whole, no cut
            if (MODE == MODE_STATS && lane == 0) {
                st.bytes += 4ull * run + probe_bytes(cut0, run, blen);
                st.touched += 4ull * (run + blen) + 64;
            }
            if (lane == 0) {
                ws.m[0] = m0;
                ws.m[1] = m1;
            }
            __syncwarp();
            acc += merge_count(dp, pos, end, B, 0, blen, ws.mtile, L.neq_mask & 3u, ws.m, lane);
            return true;
        }
    }
    if (!hashed) return false;
    if (MODE == MODE_STATS && lane == 0) {
        st.bytes += 4ull * run;
        st.touched += 4ull * run;
        for (int p = 0; p < np && p < 2; p++) {
            st.bytes += probe_bytes(p == 0 && cut0 >= 0 ? cut0 : plen[p], run, plen[p]);
            st.touched += 32ull * run;
        }
    }
    unsigned cnt = 0;
    for (int base = pos; base < end; base += 128) {
        int32_t x[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = base + 32 * u + lane;
            ok[u] = i < end;
            x[u] = ok[u] ? __ldg(dp + i) : 0;
        }
        for (int p = 0; p < np; p++) {
            const int32_t* tb = tab[p];
            const uint32_t Tp = T[p];
            bool f[4], dn[4];
#pragma unroll
            for (int u = 0; u < 4; u++) dn[u] = ok[u] ? hash_first(tb, Tp, x[u], f[u]) : (f[u] = false, true);
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (ok[u]) ok[u] = dn[u] ? f[u] : hash_has(tb, Tp, x[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) cnt += (ok[u] && x[u] != y0 && x[u] != y1) ? 1u : 0u;
    }
    acc += cnt;
    return true;
}

// Three-vertex plans whose last level needs no intersection per partial
// match (leaf_kind, chosen on the host by leaf_closed_form_kind):
//   1: the last level's candidates are the first level's set itself (reuse
//      of all its operands): the count for the candidate at index i follows
//      from i and the set's cut by the start node's bounds;
//   2: the last level is one list of the start node: its cut length, minus
//      the first-level node when injectivity demands and it lies inside.
// One lane per first-level candidate of the unit [a, b); returns the lane's
// count.
template <int MODE>
__device__ unsigned long long leaf_closed_form(const XmPlanDev& P, const GraphDev& g, int kind, int32_t m0,
                                               const int32_t* set, int set_len, int a, int b, int lane, Stats& st) {
    const XmLevel& L = P.lv[2];
    const int32_t lo0 = (L.lo_mask & 1u) ? m0 : -1;
    const int32_t hi0 = (L.hi_mask & 1u) ? m0 : INT_MAX;
    const int32_t* list = set;
    int len = set_len;
    if (kind == 2) {
        const ListRef r = op_list(g, L.op_dir[0], m0);
        list = r.p;
        len = r.len;
    }
    const int c0 = lo0 >= 0 ? lbound(list, 0, len, lo0 + 1, false) : 0;
    const int c1 = hi0 != INT_MAX ? lbound(list, c0, len, hi0, false) : len;
    if (MODE == MODE_STATS && lane == 0) {
        const int ns = (lo0 >= 0 ? 1 : 0) + (hi0 != INT_MAX ? 1 : 0);
        st.bytes += (kind == 2 ? 8ull : 0ull) + ns * search_bytes(len);
        st.touched += (kind == 2 ? 32ull : 0ull) + 32ull * ns * search_sectors(len);
    }
    const int per_cand = kind == 1 ? 0 : ((L.lo_mask & 2u) ? 1 : 0) + ((L.hi_mask & 2u) ? 1 : 0) + ((L.neq_mask & 2u) ? 1 : 0);
    unsigned long long acc = 0, nc = 0;
    for (int i = a + lane; i < b; i += 32) {
        const int32_t m1 = __ldg(set + i);
        int lo = c0, hi = c1;
        nc++;
        if (kind == 1) {
            // positions in the set are the candidates' own indices
            if (L.lo_mask & 2u) lo = max(lo, i + 1);
            if (L.hi_mask & 2u) hi = min(hi, i);
            long long c = hi > lo ? hi - lo : 0;
            if ((L.neq_mask & 2u) && i >= lo && i < hi) c--;
            acc += c;
        } else {
            if (L.lo_mask & 2u) lo = max(lo, lbound(list, lo, hi, m1 + 1, false));
            if (L.hi_mask & 2u) hi = min(hi, lbound(list, lo, hi, m1, false));
            long long c = hi > lo ? hi - lo : 0;
            if ((L.neq_mask & 2u) && c > 0) {
                // the first-level node itself is not a candidate
                const int q = lbound(list, lo, hi, m1, false);
                if (q < hi && __ldg(list + q) == m1) c--;
            }
            acc += c;
        }
    }
    if (MODE == MODE_STATS && per_cand) {
        // every candidate's bound searches over the cut list
        const unsigned long long s = warp_sum((unsigned)nc);
        if (lane == 0) {
            st.bytes += s * per_cand * search_bytes(c1 - c0);
            st.touched += 32ull * s * per_cand * search_sectors(c1 - c0);
        }
    }
    return acc;
}

// With ra.root_counts (count mode) the count of every unit goes to the
// 128-bit counter of its start-node index i (the position in the root list,
// or the node id without one), ra.root_counts[2 i .. 2 i + 1]. (A run-time
// switch: a third template flag for it made ptxas fail on the product
// kernel.)
// MINB: resident 512-thread blocks the register budget must allow -- 3 (40
// registers a thread, 48 warps an SM) for three-level plans, whose probe
// loops are latency-bound and want warps; 2 (64 registers) for deeper
// plans, whose batched last level needs the registers.
// Resident blocks of 512 threads the matcher's register budget is cut for
// (2: 64 registers per thread).
#ifndef XM_BATCH_TU
#ifndef XM_MATCH_MINB
#define XM_MATCH_MINB 2
#endif
template <int MODE, bool PROD, int MINB = XM_MATCH_MINB, bool B4 = false>
__global__ void __launch_bounds__(512, MINB) k_match(const XmPlanDev* __restrict__ plan_g, RunArgs ra) {
    // the three-level build leaves out the batched last level and the
    // merges (their registers would spill into its probe loops)
    constexpr bool LEAN = MINB >= 3;
    const bool ROOTS = MODE == MODE_COUNT && ra.root_counts != nullptr;
    extern __shared__ __align__(16) unsigned char smem[];
    XmPlanDev& P = *reinterpret_cast<XmPlanDev*>(smem);
    plan_to_smem(P, plan_g);

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int k = P.k;
    // counting with a leaf product walks levels 0..prod_p only (ke levels)
    constexpr bool prod = PROD;
    const int ke = prod ? P.prod_p + 1 : k;
    const int W = ra.window;
    const bool tile = !LEAN && ra.merge_ratio > 0;
    const size_t warp_bytes = match_warp_bytes(k, W, tile);
    unsigned char* wbase = smem + plan_bytes(k) + (size_t)wib * warp_bytes;
    WarpSmem& ws = *reinterpret_cast<WarpSmem*>(wbase);
    int32_t* wins = reinterpret_cast<int32_t*>(wbase + warp_state_bytes(k));  // level l >= 2 at (l-2)*W
    if (lane == 0) ws.mtile = tile ? wins + (size_t)n_windows(k) * W : nullptr;
    __syncwarp();
    const GraphDev& g = ra.g;
    // B4: four-level plans counted through units below the first level, whose
    // last level is a batched two-list level (the launch checks the shape)
    const bool two_level = B4 ? false : !ra.l2_units;
    // unit index space: pieces of a start node's first-level set, or pieces
    // of a first-level candidate's second-level driver range
    const int32_t* uprefix = two_level ? ra.units : ra.e_units;
    const int nidx = two_level ? ra.n_idx : set_start(ra, ra.n_idx);
    // a work-unit scan that overflowed int32 left wrapped prefixes: walk
    // nothing (the host sees the status bit and retries with larger units)
    if (*((volatile unsigned long long*)(ra.ctl + CTL_STATUS)) & STATUS_OVERFLOW) return;
    const int total = uprefix[nidx];
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    // walks of four or more levels: the units of one heavy start node lie
    // next to each other and cost far more than the average, so warps take
    // them two at a time (a batch of them would end up in one warp)
    const int maxb = ke >= 4 ? 2 : 64;

    unsigned long long acc = 0;
    Stats st;
    Budget budget;
    budget.start(ra.ctl, ra.budget_ns, lane);
    int owner = -1;
    int acc_root = -1;  // ROOTS: start-node index the running count belongs to
    unsigned long long* counter = ra.ctl + CTL_COUNT_LO;
    if (MODE == MODE_STATS && lane == 0) atomicCAS(ra.ctl + CTL_W_START, 0ull, global_ns());
    for (;;) {
        long long start;
        int cnt;
        grab_units(ra.ctl + CTL_HEAD, total, nwarps, lane, start, cnt, budget, maxb);
        if (cnt <= 0) break;
        bool stop = false;
        for (int u = (int)start; u < (int)start + cnt && !stop; u++) {
            if (owner < 0 || u < __ldg(uprefix + owner) || u >= __ldg(uprefix + owner + 1)) {
                // consecutive units usually belong to the next owners: step a
                // few ahead before searching
                int o = owner;
                bool found = false;
                if (o >= 0 && u >= __ldg(uprefix + o))
                    for (int t = 0; t < 4 && o + 1 < nidx; t++) {
                        o++;
                        if (u < __ldg(uprefix + o + 1)) { found = u >= __ldg(uprefix + o); break; }
                    }
                owner = found ? o : owner_of(uprefix, nidx, u);
            }
            const int chunk = u - __ldg(uprefix + owner);
            if (ROOTS) {
                const int rt = two_level ? owner : __ldg(ra.l1root + owner);
                if (rt != acc_root) {
                    if (acc_root >= 0) flush_count(acc, counter, lane);
                    acc = 0;
                    acc_root = rt;
                    counter = ra.root_counts + 2 * (size_t)rt;
                }
            }
            if (MODE == MODE_STATS && lane == 0) st.units++;
            if (!B4 && two_level && ke > 2) {
                // unit = (start node, a piece of its first-level set)
                const int root = owner;
                const int s0 = set_start(ra, root), s1 = set_start(ra, root + 1);
                const int32_t* base = ra.l1set + s0;
                const int a = chunk * ra.unit;
                const int b = min(s1 - s0, a + ra.unit);
                if (MODE == MODE_STATS && lane == 0) {
                    st.bytes += 4ull * (b - a);
                    st.touched += 4ull * (b - a);
                }
                if (MODE != MODE_EMIT && ra.leaf_kind) {
                    acc += leaf_closed_form<MODE>(P, g, ra.leaf_kind, root_node(ra, root), base, s1 - s0, a, b, lane,
                                                  st);
                    continue;
                }
                if (lane == 0) {
                    ws.m[0] = root_node(ra, root);
                    LvState& S1 = ws.st[1];
                    S1.it_ptr = base;
                    S1.it_shared = 0;
                    S1.wpos = a;
                    S1.it_hi = b;
                    S1.set_ptr = base;
                    S1.set_len = s1 - s0;
                    S1.set_shared = 0;
                    S1.complete = 1;
                    S1.drv_pos = S1.drv_end = 0;
                }
                __syncwarp();
                if (!explore<MODE, PROD, LEAN>(P, g, ws, wins, W, 2, lane, ra, acc, counter, st, budget, 1))
                    stop = true;
                continue;
            }
            if (!B4 && two_level) {
                // the first level is the last: every candidate is a match
                const int root = owner;
                const int s0 = set_start(ra, root), s1 = set_start(ra, root + 1);
                const int32_t* base = ra.l1set + s0;
                const int a = chunk * ra.unit;
                const int b = min(s1 - s0, a + ra.unit);
                const int32_t rnode = root_node(ra, root);
                if (MODE == MODE_EMIT) {
                    for (int p = a; p < b; p += 32) {
                        const bool ok = p + lane < b;
                        const unsigned mask = __ballot_sync(FULL, ok);
                        unsigned long long o = 0;
                        if (lane == 0) o = atomicAdd(ra.ctl + CTL_EMIT, (unsigned long long)__popc(mask));
                        o = __shfl_sync(FULL, o, 0) + lane;
                        if (ok && o < ra.capacity) {
                            ra.out[o * 2 + P.order[0]] = rnode;
                            ra.out[o * 2 + P.order[1]] = __ldg(base + p + lane);
                        }
                    }
                }
                if (lane == 0) acc += b - a;
                continue;
            }
            // unit = (start node, one first-level candidate, a piece of the
            // second level's driver range)
            const int e = owner;
            const int root = __ldg(ra.l1root + e);
            const int s0 = set_start(ra, root), s1 = set_start(ra, root + 1);
            const int per2 = l2_piece(P, g, ke, ra.unit, root_node(ra, root), __ldg(ra.l1set + e));
            if (MODE == MODE_STATS && lane == 0) {
                st.bytes += 4;
                st.touched += 4;
            }
            if (!B4 && MODE != MODE_EMIT && ke == 3 &&
                leaf3_direct<MODE, LEAN>(P, g, root_node(ra, root), __ldg(ra.l1set + e), ra.l1set + s0, s1 - s0,
                                   chunk * per2, per2, lane, acc, ra, ws, st))
                continue;
            if (lane == 0) {
                ws.m[0] = root_node(ra, root);
                ws.m[1] = __ldg(ra.l1set + e);
                LvState& S1 = ws.st[1];
                S1.set_ptr = ra.l1set + s0;
                S1.set_len = s1 - s0;
                S1.set_shared = 0;
                S1.complete = 1;
                S1.wpos = S1.it_hi = 0;
                S1.drv_pos = S1.drv_end = 0;
            }
            __syncwarp();
            if (MODE == MODE_STATS && lane == 0) st.ext++;
            if (!B4 && ke == 3) {
                acc += leaf_level<MODE, LEAN>(P, g, ws, 2, lane, ra, st, chunk * per2, per2);
                if (MODE == MODE_STATS && lane == 0) st.sets++;
                continue;
            }
            setup_level<MODE>(P, g, ws, 2, lane, st, false);
            if (MODE == MODE_STATS && lane == 0) st.sets++;
            LvState& S2 = ws.st[2];
            if (S2.empty) continue;
            const int pos = min(S2.c1, S2.c0 + chunk * per2);
            const int end = min(S2.c1, pos + per2);
            if (pos >= end) continue;
            account_scan<MODE>(S2, end - pos, st, lane);
            const bool whole = pos == S2.c0 && end == S2.c1;
            if (lane == 0) {
                S2.drv_pos = pos;
                S2.drv_end = end;
            }
            __syncwarp();
            int32_t* win = wins;  // level 2's window
            scan_level<MODE, true>(P, P.lv[2], g, ws, S2, 2, win, W, lane, ra, st);
            if (lane == 0) {
                S2.complete = whole && S2.drv_pos >= S2.drv_end;
                S2.it_ptr = win;
                S2.it_shared = 1;
                S2.wpos = 0;
                S2.it_hi = S2.wcnt;
                S2.set_ptr = win;
                S2.set_len = S2.wcnt;
                S2.set_shared = 1;
            }
            __syncwarp();
            if (B4) {
                if (!walk_last2<MODE>(P, g, ws, win, W, batch_leaf_fixed_op(P), lane, ra, acc, st, budget))
                    stop = true;
                continue;
            }
            if (!explore<MODE, PROD, LEAN>(P, g, ws, wins, W, 2, lane, ra, acc, counter, st, budget, 2)) stop = true;
        }
        if (stop) break;
    }
    if (!ROOTS || acc_root >= 0) flush_count(acc, counter, lane);
    if (MODE == MODE_STATS && lane == 0) {
        atomicAdd(ra.ctl + CTL_STATS + 0, st.bytes);
        atomicAdd(ra.ctl + CTL_STATS + 1, st.ext);
        atomicAdd(ra.ctl + CTL_STATS + 2, st.sets);
        atomicAdd(ra.ctl + CTL_STATS + 3, st.units);
        atomicAdd(ra.ctl + CTL_STATS + 4, st.leaf);
        atomicAdd(ra.ctl + CTL_STATS + 6, st.touched);
        // load balance of the persistent grid: when each warp ran out of work
        const unsigned long long t = global_ns();
        const unsigned long long t0 = *((volatile unsigned long long*)(ra.ctl + CTL_W_START));
        atomicMax(ra.ctl + CTL_W_FIRST, ~t);
        atomicMax(ra.ctl + CTL_W_LAST, t);
        atomicAdd(ra.ctl + CTL_W_SUM, t - t0);
        atomicAdd(ra.ctl + CTL_W_COUNT, 1ull);
    }
}

#endif
#ifdef XM_BATCH_TU
// Batched matcher: many (plan, graph) pairs in one persistent launch. A
// work unit is a block of `root_block` consecutive start nodes of one pair;
// each warp keeps its own copy of the current pair's plan. The first level
// is built per start node in a shared-memory window (the graphs are small),
// then the same Explore() recursion runs, ending in the plan's leaf product
// when it has one; counts go to the pair's counter. Compiled only in the
// batch translation unit (xm_batch_kernel.cu). 64 registers: at 40 the
// product walk spilled 896 bytes and the configured batch ran 16 % slower.
__global__ void __launch_bounds__(512, 2) k_match_batch(BatchDev b) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int W = b.window;
    const size_t warp_bytes = batch_warp_bytes_impl(b.kmax, W);
    unsigned char* wbase = smem + (size_t)wib * warp_bytes;
    XmPlanDev& P = *reinterpret_cast<XmPlanDev*>(wbase);
    WarpSmem& ws = *reinterpret_cast<WarpSmem*>(wbase + plan_bytes(b.kmax));
    int32_t* wins = reinterpret_cast<int32_t*>(wbase + plan_bytes(b.kmax) + warp_state_bytes(b.kmax));
    if (lane == 0) ws.mtile = wins + (size_t)(b.kmax > 2 ? b.kmax - 2 : 0) * W;
    __syncwarp();
    const long long total = __ldg(b.unit_prefix + b.npairs);
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    RunArgs ra{};  // count mode: no emission buffer
    ra.window = W;
    ra.merge_ratio = b.merge_ratio;
    GraphDev g{};
    Stats st;
    Budget budget;
    budget.start(b.ctl, b.budget_ns, lane);
    int cur = -1;
    unsigned long long acc = 0;
    bool stop = false;
    Budget pair_budget;  // per-pair budgets: the current pair's
    for (; !stop;) {
        long long start;
        int cnt;
        grab_units(b.ctl + CTL_HEAD, total, nwarps, lane, start, cnt, budget);
        if (cnt <= 0) break;
        for (long long u = start; u < start + cnt; u++) {
            // pair owning unit u: last p with unit_prefix[p] <= u
            int lo = 0, hi = b.npairs;
            if (cur >= 0 && u >= __ldg(b.unit_prefix + cur) && u < __ldg(b.unit_prefix + cur + 1)) {
                lo = cur;
            } else {
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (__ldg(b.unit_prefix + mid) <= u) lo = mid; else hi = mid;
                }
            }
            if (lo != cur) {
                if (cur >= 0) flush_count(acc, b.counts + 2 * (size_t)cur, lane);
                acc = 0;
                cur = lo;
                const int2 pg = b.pairs[cur];
                __syncwarp();
                for (int i = lane; i < (int)(plan_bytes(__ldg(&b.plans[pg.x].k)) / 4); i += 32)
                    reinterpret_cast<int32_t*>(&P)[i] = reinterpret_cast<const int32_t*>(b.plans + pg.x)[i];
                g = b.graphs[pg.y];
                // counts with a leaf product (Sec. 5.3) read its sets from the
                // device plan in global memory (the shared copy holds levels only)
                ra.pv = P.prod_r > 0 ? b.plans[pg.x].pv : nullptr;
                __syncwarp();
            }
            // per-pair budgets count from the start of each unit, so that time a
            // pair's units spend queued behind other pairs' units in a warp's
            // grab is not charged to it; once one unit of a pair runs out, the
            // pair's remaining units are skipped
            if (b.pair_budget_ns) {
                pair_budget.start_unit(b.pair_status + cur, b.pair_budget_ns, lane);
                if (pair_budget.expired(lane)) continue;
            }
            const int r0 = (int)(u - __ldg(b.unit_prefix + cur)) * b.root_block;
            const int r1 = min(r0 + b.root_block, g.n);
            const int k = P.k;
            const Budget& bud = b.pair_budget_ns ? pair_budget : budget;
            for (int v = r0; v < r1; v++) {
                if (!passes_degree(g, v, P.lv[0].dout_min, P.lv[0].din_min)) continue;
                if (lane == 0) ws.m[0] = v;
                __syncwarp();
                if (k == 2) {
                    acc += leaf_level<MODE_COUNT>(P, g, ws, 1, lane, ra, st);
                    continue;
                }
                if (!descend<MODE_COUNT>(P, g, ws, wins, W, 1, lane, ra, st)) continue;
                const bool done =
                    ra.pv ? explore<MODE_COUNT, true>(P, g, ws, wins, W, 1, lane, ra, acc, b.counts + 2 * (size_t)cur,
                                                      st, bud)
                          : explore<MODE_COUNT, false>(P, g, ws, wins, W, 1, lane, ra, acc,
                                                       b.counts + 2 * (size_t)cur, st, bud);
                if (!done) {
                    stop = !b.pair_budget_ns;  // a pair's budget ends that pair only
                    break;
                }
            }
            if (stop) break;
        }
    }
    if (cur >= 0) flush_count(acc, b.counts + 2 * (size_t)cur, lane);
}

#endif
#ifndef XM_BATCH_TU
// ------------------------------------------------------ cut-vertex split
// sum over nodes v of prod_{i < t} cnt_i(v), mod 2^128, where cnt_i(v) is
// the 128-bit counter cnt[i * 2n + 2v .. + 1]; added to out[0..1].
__global__ void k_root_product(const unsigned long long* __restrict__ cnt, int t, int n, unsigned long long* out) {
    typedef unsigned __int128 u128;
    u128 sum = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        u128 prod = 1;
        for (int i = 0; i < t && prod; i++) {
            const unsigned long long* c = cnt + (size_t)i * 2 * n + 2 * (size_t)v;
            prod *= ((u128)__ldg(c + 1) << 64) | __ldg(c);
        }
        sum += prod;
    }
    unsigned long long lo = (unsigned long long)sum, hi = (unsigned long long)(sum >> 64);
    for (int off = 16; off; off >>= 1) {
        const unsigned long long olo = __shfl_down_sync(FULL, lo, off);
        const unsigned long long ohi = __shfl_down_sync(FULL, hi, off);
        const unsigned long long s = lo + olo;
        hi += ohi + (s < lo ? 1 : 0);
        lo = s;
    }
    if ((threadIdx.x & 31) == 0 && (lo | hi)) {
        const unsigned long long old = atomicAdd(out, lo);
        const unsigned long long carry = (old + lo < old) ? 1 : 0;
        if (hi + carry) atomicAdd(out + 1, hi + carry);
    }
}

// ------------------------------------------------------------------- scan
// Exclusive scan of an int32 array in place, in three passes over tiles of
// SCAN_TILE elements (tile sums, one-block scan of the sums, tile scans).

__device__ __forceinline__ long long block_sum(long long x) {
    __shared__ long long wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) x += __shfl_down_sync(FULL, x, o);
    if (lane == 0) wsum[w] = x;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x < 32) {
        t = (threadIdx.x < (blockDim.x >> 5)) ? wsum[threadIdx.x] : 0;
        for (int o = 16; o; o >>= 1) t += __shfl_down_sync(FULL, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// The scans' tiles: a grid-stride loop over the tiles that hold elements
// (with `last`: up to the terminal element only), so a capacity-sized array
// of which little is used costs a few blocks, not one block per tile.
__global__ void k_scan_reduce(const int32_t* __restrict__ v, int64_t len, int64_t* __restrict__ sums,
                              const int32_t* __restrict__ last) {
    if (last) len = min(len, (int64_t)__ldg(last) + 1);
    const int64_t ntiles = (len + SCAN_TILE - 1) / SCAN_TILE;
    for (int64_t b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const int64_t base = b * SCAN_TILE;
        long long s = 0;
        for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
            if (base + i < len) s += v[base + i];
        s = block_sum(s);
        if (threadIdx.x == 0) sums[b] = s;
        __syncthreads();  // block_sum's shared words are reused by the next tile
    }
}
template <typename T>
__device__ void block_exclusive_scan(T* vals, int per, T carry_in, T& total) {
    __shared__ T wtot[32];
    __shared__ T wpre[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T t = 0;
    for (int j = 0; j < per; j++) t += vals[j];
    T inc = t;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wtot[w] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T run = 0;
        for (int i = 0; i < nw; i++) { wpre[i] = run; run += wtot[i]; }
        wtot[0] = run;
    }
    __syncthreads();
    T pre = carry_in + wpre[w] + inc - t;
    total = wtot[0];
    for (int j = 0; j < per; j++) {
        T x = vals[j];
        vals[j] = pre;
        pre += x;
    }
    __syncthreads();
}

__global__ void k_scan_top(int64_t* sums, int64_t nb, unsigned long long* __restrict__ status,
                           const int32_t* __restrict__ last) {
    if (last) nb = min(nb, ((int64_t)__ldg(last) + SCAN_TILE) / SCAN_TILE);  // tiles holding v[0..*last]
    const int per = 8;
    long long carry = 0;
    for (int64_t base = 0; base < nb; base += (int64_t)blockDim.x * per) {
        long long vals[per];
        for (int j = 0; j < per; j++) {
            int64_t i = base + (int64_t)threadIdx.x * per + j;
            vals[j] = i < nb ? sums[i] : 0;
        }
        long long tot;
        block_exclusive_scan<long long>(vals, per, carry, tot);
        for (int j = 0; j < per; j++) {
            int64_t i = base + (int64_t)threadIdx.x * per + j;
            if (i < nb) sums[i] = vals[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && carry > INT_MAX) atomicOr(status, (unsigned long long)STATUS_OVERFLOW);
}

__global__ void k_scan_down(int32_t* __restrict__ v, int64_t len, const int64_t* __restrict__ sums,
                            const int32_t* __restrict__ last) {
    if (last) len = min(len, (int64_t)__ldg(last) + 1);
    const int64_t ntiles = (len + SCAN_TILE - 1) / SCAN_TILE;
    const int per = SCAN_TILE / 1024;  // launched with 1024 threads
    for (int64_t b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const int64_t base = b * SCAN_TILE;
        long long vals[per];
        for (int j = 0; j < per; j++) {
            int64_t i = base + (int64_t)threadIdx.x * per + j;
            vals[j] = i < len ? v[i] : 0;
        }
        long long tot;
        block_exclusive_scan<long long>(vals, per, sums[b], tot);
        for (int j = 0; j < per; j++) {
            int64_t i = base + (int64_t)threadIdx.x * per + j;
            if (i < len) v[i] = (int32_t)vals[j];
        }
        __syncthreads();  // the scan's shared words are reused by the next tile
    }
}
cudaError_t scan_in_place(int32_t* v, int64_t len, const RunArgs& a, cudaStream_t stream,
                          const int32_t* last = nullptr) {
    const int64_t nb = (len + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > a.n_block_sums) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // two 1024-thread blocks per SM walk the tiles
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)nsm * 2));
    k_scan_reduce<<<grid, 1024, 0, stream>>>(v, len, a.block_sums, last);
    k_scan_top<<<1, 1024, 0, stream>>>(a.block_sums, nb, a.ctl + CTL_STATUS, last);
    k_scan_down<<<grid, 1024, 0, stream>>>(v, len, a.block_sums, last);
    return cudaGetLastError();
}

#endif
}  // namespace

#ifdef XM_BATCH_TU
size_t batch_warp_bytes(int kmax, int window) { return batch_warp_bytes_impl(kmax, window); }

cudaError_t launch_batch(const BatchDev& b, int warps_per_block, int blocks_per_sm, cudaStream_t stream) {
    cudaError_t err;
    int dev = 0, nsm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    const size_t smem = batch_warp_bytes_impl(b.kmax, b.window) * warps_per_block;
    if ((err = cudaFuncSetAttribute((const void*)k_match_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)) != cudaSuccess)
        return err;
    int occ = 0;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_match_batch, warps_per_block * 32,
                                                             smem)) != cudaSuccess)
        return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
    k_match_batch<<<nsm * bps, warps_per_block * 32, smem, stream>>>(b);
    return cudaGetLastError();
}
#else
cudaError_t scan_int32_in_place(int32_t* v, int64_t len, const RunArgs& a, cudaStream_t stream) {
    return scan_in_place(v, len, a, stream);
}

size_t match_smem_bytes(int k, int window, int warps, bool merge) {
    return plan_bytes(k) + match_warp_bytes(k, window, merge) * warps;
}

int64_t chunk_capacity(int32_t n, int64_t m) { return (int64_t)n + (m + L1_CHUNK - 1) / L1_CHUNK; }


cudaError_t launch_root_product(const unsigned long long* cnt, int t, int32_t n, unsigned long long* out,
                                cudaStream_t stream) {
    cudaError_t err;
    int dev = 0, nsm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), stream)) != cudaSuccess) return err;
    const int grid = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)nsm * 8);
    k_root_product<<<std::max(grid, 1), 256, 0, stream>>>(cnt, t, n, out);
    return cudaGetLastError();
}

int leaf_closed_form_kind(const XmPlanDev& P) {
    if (P.k != 3) return 0;
    const XmLevel& L = P.lv[2];
    if (L.ndiff) return 0;
    if ((L.lo_mask | L.hi_mask | L.neq_mask) & ~3u) return 0;
    if (L.reuse == 1 && __builtin_popcount(L.reuse_ops) == L.nops) return 1;
    if (L.reuse < 1 && L.nops == 1 && L.op_level[0] == 0) return 2;
    return 0;
}

bool use_l2_units(const XmPlanDev& P, bool counting) {
    // a leaf product at level 2 takes whole first-level candidates: units
    // per start node; deeper products split below the first level
    if (counting && P.prod_r > 0) return P.prod_p >= 3;
    if (P.k < 3) return false;
    if (P.k > 3) return true;
    // three vertices: split below the first level only when the last level
    // intersects lists (a single list is counted in O(log) per candidate)
    const XmLevel& L = P.lv[2];
    const int lists = (L.reuse >= 1 ? 1 : 0) + L.nops - (L.reuse >= 1 ? __builtin_popcount(L.reuse_ops) : 0);
    return lists + L.ndiff > 1;
}

cudaError_t launch_match(int mode, const XmPlanDev& P, const XmPlanDev* plan_dev, const RunArgs& a,
                         int warps_per_block, int blocks_per_sm, cudaStream_t stream, cudaEvent_t* ev) {
    cudaError_t err;
    const int64_t len = (int64_t)a.n_idx + 1;
    int dev = 0, nsm = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if (a.pv) return cudaErrorInvalidValue;  // set here only
    RunArgs b = a;
    // counting passes evaluate the plan's leaf product from the device copy
    if (mode != MODE_EMIT && P.prod_r > 0)
        b.pv = reinterpret_cast<const XmLevel*>(reinterpret_cast<const unsigned char*>(plan_dev) +
                                                offsetof(XmPlanDev, pv));
    if (ev && (err = cudaEventRecord(ev[0], stream)) != cudaSuccess) return err;
    const int grid_nodes = (int)std::min<int64_t>((len + 255) / 256, (int64_t)nsm * 16);
    // 1. first-level candidate sets
    k_l1_chunks<<<grid_nodes, 256, 0, stream>>>(plan_dev, b);
    if ((err = scan_in_place(b.root_chunks, len, b, stream)) != cudaSuccess) return err;
    const int grid_chunks = nsm * 8;  // 256-thread blocks: 8 warps each
    if (mode == MODE_STATS)
        k_l1<false, MODE_STATS><<<grid_chunks, 256, 0, stream>>>(plan_dev, b);
    else
        k_l1<false, MODE_COUNT><<<grid_chunks, 256, 0, stream>>>(plan_dev, b);
    if ((err = scan_in_place(b.chunk_cnt, (int64_t)b.cmax + 1, b, stream, b.root_chunks + b.n_idx)) != cudaSuccess)
        return err;
    k_l1<true, MODE_COUNT><<<grid_chunks, 256, 0, stream>>>(plan_dev, b);
    // 2. work units: per start node for two-vertex patterns, else per
    // first-level candidate (pieces of the second level's driver range)
    if (!b.l2_units) {
        k_units<<<grid_nodes, 256, 0, stream>>>(b);
        if ((err = scan_in_place(b.units, len, b, stream)) != cudaSuccess) return err;
    } else {
        const int grid_e = (int)std::min<int64_t>(((int64_t)b.emax + 256) / 256, (int64_t)nsm * 16);
        k_l2_units<<<grid_e, 256, 0, stream>>>(plan_dev, b);
        if ((err = scan_in_place(b.e_units, (int64_t)b.emax + 1, b, stream,
                                 reinterpret_cast<const int32_t*>(b.ctl + CTL_ELEN))) != cudaSuccess)
            return err;
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // 3. persistent matcher
    const bool prod = b.pv != nullptr;
    const bool roots = b.root_counts != nullptr;
    if (roots && mode != MODE_COUNT) return cudaErrorInvalidValue;
    // three-level counts (the last level probed from registers) run the
    // 40-register build, which never merges
    const bool three = mode == MODE_COUNT && !prod && P.k == 3;
    // four-level plans whose last level is a batched two-list level run a
    // build without the other level and leaf paths (fewer registers spilled,
    // less code for the instruction cache)
    const bool b4 = mode == MODE_COUNT && !prod && P.k == 4 && b.l2_units && batch_leaf_fixed_op(P) >= 0;
    const size_t smem = match_smem_bytes(P.k, b.window, warps_per_block, b.merge_ratio > 0 && !three);
    const void* fn = mode == MODE_STATS  ? (prod ? (const void*)k_match<MODE_STATS, true>
                                                 : (const void*)k_match<MODE_STATS, false>)
                     : mode == MODE_EMIT ? (const void*)k_match<MODE_EMIT, false>
                     : prod              ? (const void*)k_match<MODE_COUNT, true>
                     : three             ? (const void*)k_match<MODE_COUNT, false, 3>
                     : b4                ? (const void*)k_match<MODE_COUNT, false, XM_MATCH_MINB, true>
                                         : (const void*)k_match<MODE_COUNT, false>;
    if ((err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return err;
    int occ = 0;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, warps_per_block * 32, smem)) != cudaSuccess)
        return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
    dim3 grid(nsm * bps), block(warps_per_block * 32);
    if (ev && (err = cudaEventRecord(ev[1], stream)) != cudaSuccess) return err;
    if (mode == MODE_STATS && prod)
        k_match<MODE_STATS, true><<<grid, block, smem, stream>>>(plan_dev, b);
    else if (mode == MODE_STATS)
        k_match<MODE_STATS, false><<<grid, block, smem, stream>>>(plan_dev, b);
    else if (mode == MODE_EMIT)
        k_match<MODE_EMIT, false><<<grid, block, smem, stream>>>(plan_dev, b);
    else if (prod)
        k_match<MODE_COUNT, true><<<grid, block, smem, stream>>>(plan_dev, b);
    else if (three)
        k_match<MODE_COUNT, false, 3><<<grid, block, smem, stream>>>(plan_dev, b);
    else if (b4)
        k_match<MODE_COUNT, false, XM_MATCH_MINB, true><<<grid, block, smem, stream>>>(plan_dev, b);
    else
        k_match<MODE_COUNT, false><<<grid, block, smem, stream>>>(plan_dev, b);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (ev && (err = cudaEventRecord(ev[2], stream)) != cudaSuccess) return err;
    return cudaSuccess;
}

#endif

}  // namespace xm
