// Host-side pattern compiler: constraint inclusion (Sec. 4.1), pattern
// reduction (Alg. 1), plan generation (Sec. 5.1) with candidate-set reuse
// (Sec. 5.2), symmetry-breaking conditions, lowered to the flat plan IR.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "xm_internal.h"

namespace xm {

namespace {

struct Pat {
    int k = 0, e = 0;
    std::vector<int> s, d;  // arc i: s[i] -> d[i]
    uint32_t outb[XM_MAXK] = {0}, inb[XM_MAXK] = {0};
    int dout[XM_MAXK] = {0}, din[XM_MAXK] = {0}, deg[XM_MAXK] = {0};
    bool arc(int u, int v) const { return (outb[u] >> v) & 1u; }
    bool incident(int ed, int v) const { return s[ed] == v || d[ed] == v; }
    int other(int ed, int v) const { return s[ed] == v ? d[ed] : s[ed]; }
};

inline uint64_t bit(int i) { return 1ull << i; }
inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

// ------------------------------------------------------------ Aut(P) ---

void automorphisms(const Pat& P, std::vector<std::vector<int>>& out) {
    std::vector<int> p(P.k);
    for (int i = 0; i < P.k; i++) p[i] = i;
    do {
        bool ok = true;
        for (int i = 0; i < P.e && ok; i++) ok = P.arc(p[P.s[i]], p[P.d[i]]);
        if (ok) out.push_back(p);
    } while (std::next_permutation(p.begin(), p.end()));
}

// ------------------------------------------- constraint inclusion (4.1) ---
// incl[e] = set of edges e' with e' included in e (the matches of e' are a
// subset of those of e under the shared context). Only the degree is a
// vertex constraint, so a vertex with a larger pattern degree is the more
// constrained one: x is included in y (same context) when deg(x) >= deg(y).

std::vector<uint64_t> inclusion_sets(const Pat& P) {
    std::vector<uint64_t> incl(P.e, 0);
    // Neighbour grouping (Thm. 2.1): edges sharing a destination are
    // related through their sources, edges sharing a source through their
    // destinations.
    for (int a = 0; a < P.e; a++)
        for (int b = 0; b < P.e; b++) {
            if (a == b) continue;
            if (P.d[a] == P.d[b] && P.deg[P.s[a]] >= P.deg[P.s[b]]) incl[b] |= bit(a);
            if (P.s[a] == P.s[b] && P.deg[P.d[a]] >= P.deg[P.d[b]]) incl[b] |= bit(a);
        }
    // Path closure (Thm. 2.2): if e1 is included in e3, an edge e2 that
    // continues e1 is included in an edge e4 that continues e3 the same way
    // (leaving the heads, or entering the tails), when e2's far endpoint is
    // at least as constrained. Repeat to a fixpoint.
    bool changed = true;
    while (changed) {
        changed = false;
        for (int e3 = 0; e3 < P.e; e3++)
            for (int e1 = 0; e1 < P.e; e1++) {
                if (!(incl[e3] & bit(e1))) continue;
                for (int e2 = 0; e2 < P.e; e2++)
                    for (int e4 = 0; e4 < P.e; e4++) {
                        if (e2 == e4 || (incl[e4] & bit(e2))) continue;
                        bool fwd = P.s[e2] == P.d[e1] && P.s[e4] == P.d[e3] && P.deg[P.d[e2]] >= P.deg[P.d[e4]];
                        bool bwd = P.d[e2] == P.s[e1] && P.d[e4] == P.s[e3] && P.deg[P.s[e2]] >= P.deg[P.s[e4]];
                        if (fwd || bwd) { incl[e4] |= bit(e2); changed = true; }
                    }
            }
    }
    return incl;
}

// --------------------------------------------------- reduction (Alg. 1) ---

struct Reduction {
    int start = 0;
    std::vector<int> split;       // explored edges, in order
    std::vector<int> covered_by;  // per edge: the edge that covers it, or -1
    std::vector<int> from;        // per split edge: the vertex it was explored from
};

struct Reducer {
    const Pat& P;
    const std::vector<uint64_t>& incl;
    bool reduce;
    uint64_t unvisited;
    Reduction R;

    Reducer(const Pat& p, const std::vector<uint64_t>& in, bool red) : P(p), incl(in), reduce(red) {
        unvisited = (P.e == 64) ? ~0ull : (bit(P.e) - 1);
        R.covered_by.assign(P.e, -1);
        R.from.assign(P.e, -1);
    }

    bool has_unvisited_at(int v) const {
        for (int ed = 0; ed < P.e; ed++)
            if ((unvisited & bit(ed)) && P.incident(ed, v)) return true;
        return false;
    }

    // findMaxECoverage: the unvisited edge at v whose inclusion set covers the
    // most unvisited edges (ties: lowest edge index).
    int find_max_coverage(int v) const {
        int best = -1, best_cov = -1;
        for (int ed = 0; ed < P.e; ed++) {
            if (!(unvisited & bit(ed)) || !P.incident(ed, v)) continue;
            int cov = reduce ? popc64(incl[ed] & unvisited) : 0;
            if (cov > best_cov) { best = ed; best_cov = cov; }
        }
        return best;
    }

    // updateVInclusion: after edge ec (explored from v) materialises w, the
    // unvisited edges it includes that hang off v the same way (v -> x when
    // ec = v -> w, x -> v when ec = w -> v) are covered: x is materialised
    // from w's candidates, and the covering recurses from x.
    void update_inclusion(int ec, int v) {
        if (!reduce) return;
        bool out_of_v = P.s[ec] == v;
        for (int ed = 0; ed < P.e; ed++) {
            if (!(unvisited & bit(ed)) || !(incl[ec] & bit(ed))) continue;
            bool same_role = out_of_v ? (P.s[ed] == v) : (P.d[ed] == v);
            if (!same_role) continue;
            unvisited &= ~bit(ed);
            R.covered_by[ed] = ec;
            update_inclusion(ed, v);
        }
    }

    // Neighbor_MaxDegree: the neighbour of w with the highest degree that
    // still has unvisited edges (ties: lowest id); -1 when none.
    int neighbor_max_degree(int w) const {
        if (w < 0) return -1;
        int best = -1;
        for (int x = 0; x < P.k; x++) {
            if (x == w || !(P.arc(w, x) || P.arc(x, w)) || !has_unvisited_at(x)) continue;
            if (best < 0 || P.deg[x] > P.deg[best]) best = x;
        }
        return best;
    }

    void search_split(int u) {
        int v = u;
        while (v >= 0) {
            int w = -1;
            while (has_unvisited_at(v)) {
                int mec = find_max_coverage(v);
                unvisited &= ~bit(mec);
                R.split.push_back(mec);
                R.from[mec] = v;
                w = P.other(mec, v);
                update_inclusion(mec, v);
            }
            v = neighbor_max_degree(w);
        }
    }

    void run(int forced_start = -1) {
        int start = 0;
        for (int v = 1; v < P.k; v++)
            if (P.deg[v] > P.deg[start]) start = v;  // maxDegree, ties: lowest id
        if (forced_start >= 0) start = forced_start;  // rooted plans start at their root
        R.start = start;
        search_split(start);
        while (unvisited) {
            int ed = __builtin_ctzll(unvisited);
            int u = (P.deg[P.s[ed]] <= P.deg[P.d[ed]]) ? P.d[ed] : P.s[ed];
            search_split(u);
        }
    }
};

// -------------------------------------------- plan generation (Sec. 5.1) ---
// Materialisation order: the start vertex, then the vertices reached by the
// explored edges in queue order, each followed by the vertices materialised
// from it through covered edges.

std::vector<int> materialisation_order(const Pat& P, const Reduction& R) {
    std::vector<int> order{R.start};
    uint32_t placed = 1u << R.start;
    std::vector<int> pending(R.split.begin(), R.split.end());
    auto place_covered = [&](auto&& self, int ed) -> void {
        for (int c = 0; c < P.e; c++) {
            if (R.covered_by[c] != ed) continue;
            for (int x : {P.s[c], P.d[c]})
                if (!(placed >> x & 1u) && (placed >> P.other(c, x) & 1u)) {
                    order.push_back(x);
                    placed |= 1u << x;
                }
            self(self, c);
        }
    };
    bool progress = true;
    while (!pending.empty() && progress) {
        progress = false;
        for (size_t i = 0; i < pending.size(); i++) {
            int ed = pending[i];
            bool ps = placed >> P.s[ed] & 1u, pd = placed >> P.d[ed] & 1u;
            if (!ps && !pd) continue;
            const uint32_t before = placed;
            const size_t g0 = order.size();
            if (!ps || !pd) {
                int x = ps ? P.d[ed] : P.s[ed];
                order.push_back(x);
                placed |= 1u << x;
            }
            place_covered(place_covered, ed);
            // Vertices materialised in one step are explored smallest set
            // first (Alg. 2 iterates the endpoint with fewer matchings): more
            // arcs to the vertices placed before the step, then higher degree.
            auto ties = [&](int x) { return __builtin_popcount((P.outb[x] | P.inb[x]) & before) +
                                            __builtin_popcount(P.outb[x] & P.inb[x] & before); };
            std::stable_sort(order.begin() + (long)g0, order.end(), [&](int a, int b) {
                if (ties(a) != ties(b)) return ties(a) > ties(b);
                return P.deg[a] > P.deg[b];
            });
            pending.erase(pending.begin() + (long)i);
            progress = true;
            break;
        }
    }
    // anything left (not reachable through the queue): adjacent, highest degree first
    while ((int)order.size() < P.k) {
        int best = -1;
        for (int x = 0; x < P.k; x++) {
            if (placed >> x & 1u) continue;
            if (!((P.outb[x] | P.inb[x]) & placed)) continue;
            if (best < 0 || P.deg[x] > P.deg[best]) best = x;
        }
        order.push_back(best);
        placed |= 1u << best;
    }
    return order;
}

// ---------------------------------------------- symmetry-breaking conditions
// Grochow-Kellis: walking the vertices in plan order, require m(v) < m(w)
// for every other w in v's orbit under the current group, then keep only the
// stabiliser of v. Exactly one embedding per Aut-orbit satisfies them all.
// less[v] = bitmask of vertices w with the condition m(v) < m(w).

void symmetry_conditions(int k, const std::vector<int>& order, std::vector<std::vector<int>> G,
                         uint32_t less[XM_MAXK]) {
    for (int i = 0; i < k; i++) less[i] = 0;
    for (int v : order) {
        if (G.size() <= 1) break;
        uint32_t orbit = 0;
        for (auto& g : G) orbit |= 1u << g[v];
        orbit &= ~(1u << v);
        less[v] |= orbit;
        std::vector<std::vector<int>> H;
        for (auto& g : G)
            if (g[v] == v) H.push_back(g);
        G.swap(H);
    }
}

// ----------------------------------------------------- leaf products (5.3)
// Sec. 5.3 counts by multiplying the sizes of the candidate sets of the
// vertices that are still open once the active nodes are matched. Here such
// vertices form a set I of pattern vertices with no arc between them and a
// weakly connected rest: with I at the end of the order, every vertex of I
// is constrained by earlier levels only. A count is then exact when
//   - no symmetry condition relates two vertices of I (inclusion-exclusion
//     over the sets removes tuples that repeat a node), r = |I| <= 3; or
//   - the conditions order I totally and all of I have the same operands
//     and bounds against the rest (one set C): C(|C|, r) increasing tuples.

struct ProductChoice {
    int r = 0;
    int kind = XM_PROD_NONE;
    std::vector<int> order;
};

// Order of the vertices outside `drop` (which never holds base[0]): each
// vertex after the first is the earliest vertex of `base` adjacent to one
// already placed. Empty when the rest is not weakly connected.
std::vector<int> prefix_order(const Pat& P, const std::vector<int>& base, uint32_t drop) {
    std::vector<int> out;
    uint32_t placed = 0;
    const int want = P.k - __builtin_popcount(drop);
    while ((int)out.size() < want) {
        int pick = -1;
        for (int v : base) {
            if ((drop >> v & 1u) || (placed >> v & 1u)) continue;
            if (placed && !((P.outb[v] | P.inb[v]) & placed)) continue;
            pick = v;
            break;
        }
        if (pick < 0) return {};
        out.push_back(pick);
        placed |= 1u << pick;
    }
    return out;
}

ProductChoice choose_product(const Pat& P, const std::vector<int>& base, const std::vector<std::vector<int>>& aut,
                             bool symmetry) {
    const int k = P.k;
    std::vector<int> pos(k);
    for (int i = 0; i < k; i++) pos[base[i]] = i;
    ProductChoice best;
    long best_score = -1;
    for (uint32_t I = 1; I < (1u << k); I++) {
        const int r = __builtin_popcount(I);
        if (r < 2 || r > k - 2) continue;
        if (I >> base[0] & 1u) continue;  // the start vertex stays Alg. 1's maxDegree choice
        bool independent = true;
        for (int v = 0; v < k && independent; v++)
            if ((I >> v & 1u) && ((P.outb[v] | P.inb[v]) & I)) independent = false;
        if (!independent) continue;
        std::vector<int> order = prefix_order(P, base, I);
        if (order.empty()) continue;
        std::vector<int> mem;
        for (int v : base)
            if (I >> v & 1u) mem.push_back(v);
        order.insert(order.end(), mem.begin(), mem.end());
        uint32_t less[XM_MAXK] = {0};
        if (symmetry) symmetry_conditions(k, order, aut, less);
        // direct conditions among I, and their transitive closure
        uint32_t rel[XM_MAXK] = {0};
        int direct = 0;
        for (int a : mem)
            for (int b : mem)
                if (less[a] >> b & 1u) { rel[a] |= 1u << b; direct++; }
        for (int it = 0; it < r; it++)
            for (int a : mem)
                for (int b : mem)
                    if (rel[a] >> b & 1u) rel[a] |= rel[b];
        int kind = XM_PROD_NONE;
        if (direct == 0) {
            if (r <= 3) kind = XM_PROD_IE;
        } else {
            bool total = true;
            for (int a : mem)
                for (int b : mem)
                    if (a != b && !((rel[a] >> b & 1u) || (rel[b] >> a & 1u))) total = false;
            bool same = true;
            const uint32_t rest = ((1u << k) - 1) & ~I;
            for (int b : mem)
                for (int w = 0; w < k; w++) {
                    if (!(rest >> w & 1u)) continue;
                    const int a = mem[0];
                    if (P.arc(w, a) != P.arc(w, b) || P.arc(a, w) != P.arc(b, w) ||
                        ((less[w] >> a) & 1u) != ((less[w] >> b) & 1u) || ((less[a] >> w) & 1u) != ((less[b] >> w) & 1u))
                        same = false;
                }
            if (total && same) kind = XM_PROD_CHOOSE;
        }
        if (kind == XM_PROD_NONE) continue;
        // more product vertices first, then one common set, then the set
        // whose vertices come latest in the reduction's order
        long late = 0;
        for (int v : mem) late += pos[v];
        const long score = (long)r * 10000 + (kind == XM_PROD_CHOOSE ? 1000 : 0) + late;
        if (score > best_score) {
            best_score = score;
            best.r = r;
            best.kind = kind;
            best.order = order;
        }
    }
    return best;
}

// ------------------------------------------------- cut-vertex decomposition

// Weakly connected parts of the pattern without vertex c (vertex masks).
std::vector<uint32_t> parts_without(const Pat& P, int c) {
    uint32_t left = ((1u << P.k) - 1) & ~(1u << c);
    std::vector<uint32_t> parts;
    while (left) {
        uint32_t comp = left & (~left + 1), frontier = comp;
        while (frontier) {
            uint32_t nxt = 0;
            for (int v = 0; v < P.k; v++)
                if (frontier >> v & 1u) nxt |= P.outb[v] | P.inb[v];
            nxt &= left & ~comp;
            comp |= nxt;
            frontier = nxt;
        }
        parts.push_back(comp);
        left &= ~comp;
    }
    return parts;
}

// Isomorphism-invariant key of a pattern on k <= 8 vertices: the smallest
// 64-bit adjacency matrix over all relabellings (with fix0, over the
// relabellings that keep vertex 0: a key of the pattern rooted at 0).
uint64_t canonical_key(int k, const std::vector<std::pair<int, int>>& arcs, bool fix0 = false) {
    std::vector<int> p(k);
    for (int i = 0; i < k; i++) p[i] = i;
    uint64_t best = ~0ull;
    do {
        uint64_t key = 0;
        for (auto& a : arcs) key |= 1ull << (p[a.first] * 8 + p[a.second]);
        best = std::min(best, key);
    } while (std::next_permutation(p.begin() + (fix0 ? 1 : 0), p.end()));
    return best;
}

constexpr int kMaxQuotientPartitions = 4096;

// Picks a cut vertex (most parts, then the smallest largest part, then the
// lowest id) and builds out.decomp: rooted plans of the parts and the
// quotient patterns with their multiplicities. Leaves out.decomp null when
// the pattern has no cut vertex or too many quotients.
// With `start_fixed` (every automorphism fixes the plan's start vertex) and
// the cut vertex chosen equal to that start vertex, every quotient is also
// compiled rooted at the cut vertex, for counts restricted to start nodes.
int decompose(const Pat& P, int flags, Plan& out, std::string& err, bool start_fixed) {
    const int k = P.k;
    int cut = -1, best_big = 0;
    std::vector<uint32_t> best_parts;
    for (int c = 0; c < k; c++) {
        std::vector<uint32_t> parts = parts_without(P, c);
        if (parts.size() < 2) continue;
        int big = 0;
        for (uint32_t m : parts) big = std::max(big, __builtin_popcount(m));
        if (cut < 0 || parts.size() > best_parts.size() || (parts.size() == best_parts.size() && big < best_big)) {
            cut = c;
            best_parts = parts;
            best_big = big;
        }
    }
    if (cut < 0) return XM_OK;
    const int sub_flags = flags & (XM_NO_REDUCE | XM_NO_PRODUCT | XM_NO_SPLIT);
    auto d = std::make_shared<Decomp>();
    d->cut = cut;
    d->rooted = start_fixed && cut == out.start;
    int part_of[XM_MAXK];
    for (int v = 0; v < k; v++) part_of[v] = -1;
    for (size_t i = 0; i < best_parts.size(); i++) {
        std::vector<int> verts{cut};
        for (int v = 0; v < k; v++)
            if (best_parts[i] >> v & 1u) { verts.push_back(v); part_of[v] = (int)i; }
        int lab[XM_MAXK];
        for (size_t j = 0; j < verts.size(); j++) lab[verts[j]] = (int)j;
        const uint32_t mask = best_parts[i] | (1u << cut);
        std::vector<int32_t> s, t;
        for (int a = 0; a < P.e; a++)
            if ((mask >> P.s[a] & 1u) && (mask >> P.d[a] & 1u)) {
                s.push_back(lab[P.s[a]]);
                t.push_back(lab[P.d[a]]);
            }
        Plan sub;
        int rc = compile_pattern((int)verts.size(), (int)s.size(), s.data(), t.data(),
                                 sub_flags | XM_NO_PRODUCT | XM_NO_SPLIT, sub, err, 0);
        if (rc) return rc;
        d->part_factor *= sub.stab_size;
        d->part_vertices.push_back(verts);
        d->parts.push_back(std::move(sub));
    }
    // partitions of V \ {c} whose blocks hold at most one vertex of a part
    std::vector<int> vs;
    for (int v = 0; v < k; v++)
        if (v != cut) vs.push_back(v);
    std::vector<int> block(vs.size());
    std::vector<uint32_t> block_parts;
    std::vector<uint64_t> keys;
    int n_partitions = 0;
    bool too_many = false;
    auto emit = [&]() -> int {
        if (block_parts.size() == vs.size()) return XM_OK;  // the finest: P itself
        if (++n_partitions > kMaxQuotientPartitions) { too_many = true; return XM_OK; }
        int lab[XM_MAXK];
        lab[cut] = 0;
        for (size_t i = 0; i < vs.size(); i++) lab[vs[i]] = block[i] + 1;
        const int qk = (int)block_parts.size() + 1;
        uint64_t seen = 0;
        std::vector<std::pair<int, int>> arcs;
        for (int a = 0; a < P.e; a++) {
            const int u = lab[P.s[a]], v = lab[P.d[a]];
            if (seen >> (u * 8 + v) & 1ull) continue;
            seen |= 1ull << (u * 8 + v);
            arcs.push_back({u, v});
        }
        // counts rooted at the cut vertex (label 0) group only quotients that
        // are isomorphic by a map keeping the cut vertex: two quotients
        // isomorphic by a map that moves it have different rooted counts
        const uint64_t key = canonical_key(qk, arcs, d->rooted);
        for (size_t j = 0; j < keys.size(); j++)
            if (keys[j] == key && d->quots[j].k == qk) { d->quot_mult[j]++; return XM_OK; }
        std::vector<int32_t> s, t;
        for (auto& a : arcs) { s.push_back(a.first); t.push_back(a.second); }
        Plan q;
        int rc = compile_pattern(qk, (int)s.size(), s.data(), t.data(), sub_flags, q, err);
        if (rc) return rc;
        if (d->rooted) {
            // the quotient rooted at the cut vertex (label 0): its rooted
            // matches at node v times |Stab(0)| are its embeddings mapping c to v.
            // Compiled without reduction: the reduced rooted plans probe
            // reused first-level sets (no hash table) by binary search
            Plan qr;
            rc = compile_pattern(qk, (int)s.size(), s.data(), t.data(), sub_flags | XM_NO_SPLIT | XM_NO_REDUCE, qr,
                                 err, 0);
            if (rc) return rc;
            d->rquots.push_back(std::move(qr));
        }
        keys.push_back(key);
        d->quots.push_back(std::move(q));
        d->quot_mult.push_back(1);
        return XM_OK;
    };
    auto rec = [&](auto&& self, size_t i) -> int {
        if (too_many) return XM_OK;
        if (i == vs.size()) return emit();
        const uint32_t pb = 1u << part_of[vs[i]];
        for (size_t b = 0; b <= block_parts.size(); b++) {
            if (b < block_parts.size() && (block_parts[b] & pb)) continue;
            block[i] = (int)b;
            const bool fresh = b == block_parts.size();
            if (fresh) block_parts.push_back(pb); else block_parts[b] |= pb;
            int rc = self(self, i + 1);
            if (fresh) block_parts.pop_back(); else block_parts[b] &= ~pb;
            if (rc) return rc;
        }
        return XM_OK;
    };
    int rc = rec(rec, 0);
    if (rc) return rc;
    if (too_many) return XM_OK;
    out.decomp = d;
    return XM_OK;
}

}  // namespace

// --------------------------------------------------------------- compile ---

int compile_pattern(int32_t k, int32_t e, const int32_t* psrc, const int32_t* pdst, int flags, Plan& out,
                    std::string& err, int root) {
    if (k < 2 || k > XM_MAXK) { err = "k must be in [2, 8]"; return XM_EINVAL; }
    if (e < 1 || e > k * (k - 1)) { err = "arc count out of range"; return XM_EINVAL; }
    if (!psrc || !pdst) { err = "NULL arc array"; return XM_EINVAL; }
    if (flags & ~(XM_NO_REDUCE | XM_EMBEDDINGS | XM_INDUCED | XM_NO_PRODUCT | XM_NO_SPLIT)) {
        err = "unknown flag";
        return XM_EINVAL;
    }
    if (root >= k) { err = "root out of range"; return XM_EINVAL; }
    Pat P;
    P.k = k;
    P.e = e;
    for (int i = 0; i < e; i++) {
        int u = psrc[i], v = pdst[i];
        if (u < 0 || u >= k || v < 0 || v >= k) { err = "pattern vertex id out of range"; return XM_EINVAL; }
        if (u == v) { err = "pattern self-loop"; return XM_EINVAL; }
        if (P.arc(u, v)) { err = "repeated pattern arc"; return XM_EINVAL; }
        P.outb[u] |= 1u << v;
        P.inb[v] |= 1u << u;
        P.s.push_back(u);
        P.d.push_back(v);
    }
    // weak connectivity
    uint32_t seen = 1, frontier = 1;
    while (frontier) {
        uint32_t nxt = 0;
        for (int v = 0; v < k; v++)
            if (frontier >> v & 1u) nxt |= P.outb[v] | P.inb[v];
        frontier = nxt & ~seen;
        seen |= nxt;
    }
    if (seen != (1u << k) - 1) { err = "pattern is not weakly connected"; return XM_EINVAL; }
    for (int v = 0; v < k; v++) {
        P.dout[v] = __builtin_popcount(P.outb[v]);
        P.din[v] = __builtin_popcount(P.inb[v]);
        P.deg[v] = P.dout[v] + P.din[v];
    }

    const bool reduce = !(flags & XM_NO_REDUCE);
    std::vector<std::vector<int>> aut;
    automorphisms(P, aut);
    // a rooted plan maps the root to a given node: its symmetry conditions
    // come from the automorphisms that fix the root
    std::vector<std::vector<int>> sym;
    for (auto& g : aut)
        if (root < 0 || g[root] == root) sym.push_back(g);
    std::vector<uint64_t> incl = reduce ? inclusion_sets(P) : std::vector<uint64_t>(e, 0);
    Reducer red(P, incl, reduce);
    red.run(root);
    const Reduction& R = red.R;
    std::vector<int> order = materialisation_order(P, R);
    ProductChoice pc;
    if (!(flags & (XM_INDUCED | XM_NO_PRODUCT)) && k >= 4 && root < 0) {
        pc = choose_product(P, order, aut, !(flags & XM_EMBEDDINGS));
        if (pc.r) order = pc.order;
    }

    uint32_t less[XM_MAXK];
    if (flags & XM_EMBEDDINGS)
        for (int i = 0; i < k; i++) less[i] = 0;
    else
        symmetry_conditions(k, order, sym, less);
    // transitive closure of the "<" conditions (used to check reuse bounds)
    uint32_t lt[XM_MAXK];
    for (int i = 0; i < k; i++) lt[i] = less[i];
    for (int it = 0; it < k; it++)
        for (int i = 0; i < k; i++)
            for (int j = 0; j < k; j++)
                if (lt[i] >> j & 1u) lt[i] |= lt[j];

    int level_of[XM_MAXK];
    for (int l = 0; l < k; l++) level_of[order[l]] = l;

    XmPlanDev D;
    memset(&D, 0, sizeof D);
    D.k = k;
    for (int l = 0; l < k; l++) D.order[l] = order[l];
    int n_reuse = 0;
    for (int l = 0; l < k; l++) {
        int v = order[l];
        XmLevel& L = D.lv[l];
        L.reuse = -1;
        L.dout_min = P.dout[v];
        L.din_min = P.din[v];
        uint32_t adj_levels = 0;
        static_assert(XM_MAXOPS >= 2 * (XM_MAXK - 1), "operand arrays too small");
        for (int j = 0; j < l; j++) {
            int u = order[j];
            if (P.arc(u, v)) { L.op_level[L.nops] = j; L.op_dir[L.nops] = XM_DIR_OUT; L.nops++; adj_levels |= 1u << j; }
            if (P.arc(v, u)) { L.op_level[L.nops] = j; L.op_dir[L.nops] = XM_DIR_IN; L.nops++; adj_levels |= 1u << j; }
            if (less[u] >> v & 1u) L.lo_mask |= 1u << j;  // m(u) < m(v)
            if (less[v] >> u & 1u) L.hi_mask |= 1u << j;  // m(v) < m(u)
        }
        if (l > 0 && L.nops == 0) { err = "internal: plan level without an operand list"; return XM_EINVAL; }
        if (flags & XM_INDUCED) {
            // induced matching: every missing pattern arc to an earlier level
            // becomes a list the candidate must not be in
            for (int j = 0; j < l; j++) {
                int u = order[j];
                if (!P.arc(u, v)) { L.diff_level[L.ndiff] = j; L.diff_dir[L.ndiff] = XM_DIR_OUT; L.ndiff++; }
                if (!P.arc(v, u)) { L.diff_level[L.ndiff] = j; L.diff_dir[L.ndiff] = XM_DIR_IN; L.ndiff++; }
            }
        }
        L.neq_mask = ((1u << l) - 1) & ~adj_levels & ~L.lo_mask & ~L.hi_mask;
    }
    // Candidate-set reuse (Sec. 5.2): level l starts from the stored set of an
    // earlier level r when (i) every operand list of r is also an operand of
    // l, (ii) the edge joining l to a shared operand is included in the edge
    // joining r to it (Sec. 4.1 inclusion), (iii) r's order bounds are
    // implied at l (degree thresholds are reconciled below). Among valid
    // sources take the most operands, then the nearest level ("initialise
    // e_i from e_j rather than e_k").
    if (reduce) {
        auto edge_index = [&](int a, int b) {
            for (int i = 0; i < e; i++)
                if (P.s[i] == a && P.d[i] == b) return i;
            return -1;
        };
        for (int l = 2; l < k; l++) {
            XmLevel& L = D.lv[l];
            int v = order[l];
            int best = -1, best_ops = 0;
            uint32_t best_mask = 0;
            for (int r = 1; r < l; r++) {
                const XmLevel& Rl = D.lv[r];
                int w = order[r];
                uint32_t mask = 0;
                bool subset = true, included = false;
                for (int i = 0; i < Rl.nops && subset; i++) {
                    int found = -1;
                    for (int q = 0; q < L.nops; q++)
                        if (L.op_level[q] == Rl.op_level[i] && L.op_dir[q] == Rl.op_dir[i]) found = q;
                    if (found < 0) { subset = false; break; }
                    mask |= 1u << found;
                    int u = order[Rl.op_level[i]];
                    int el = Rl.op_dir[i] == XM_DIR_OUT ? edge_index(u, v) : edge_index(v, u);
                    int er = Rl.op_dir[i] == XM_DIR_OUT ? edge_index(u, w) : edge_index(w, u);
                    if (el >= 0 && er >= 0 && (incl[er] & bit(el))) included = true;
                }
                if (!subset || !included || Rl.nops == 0) continue;
                // a reused set was filtered by its own difference lists: they
                // must all be differences of the reusing level too
                bool diffs_ok = true;
                for (int i = 0; i < Rl.ndiff && diffs_ok; i++) {
                    bool found = false;
                    for (int q = 0; q < L.ndiff; q++)
                        if (L.diff_level[q] == Rl.diff_level[i] && L.diff_dir[q] == Rl.diff_dir[i]) found = true;
                    diffs_ok = found;
                }
                if (!diffs_ok) continue;
                bool bounds_ok = true;
                for (int j = 0; j < r && bounds_ok; j++) {
                    int u = order[j];
                    if ((Rl.lo_mask >> j & 1u) && !(lt[u] >> v & 1u)) bounds_ok = false;
                    if ((Rl.hi_mask >> j & 1u) && !(lt[v] >> u & 1u)) bounds_ok = false;
                }
                if (!bounds_ok) continue;
                if (Rl.nops > best_ops || (Rl.nops == best_ops && r > best)) {
                    best = r;
                    best_ops = Rl.nops;
                    best_mask = mask;
                }
            }
            if (best >= 0) {
                L.reuse = best;
                L.reuse_ops = best_mask;
                n_reuse++;
            }
        }
        // A reused set must keep every candidate its reusers need, so the
        // degree filter of a reuse source is weakened to the componentwise
        // minimum of its own thresholds and its reusers' (the degree filter
        // only prunes; weakening it never changes results). Walking down the
        // levels carries the minimum along reuse chains.
        for (int l = k - 1; l >= 2; l--) {
            const XmLevel& L = D.lv[l];
            if (L.reuse < 1) continue;
            XmLevel& Rl = D.lv[L.reuse];
            Rl.dout_min = std::min(Rl.dout_min, L.dout_min);
            Rl.din_min = std::min(Rl.din_min, L.din_min);
        }
    }
    // A candidate drawn from the out-lists of `nout` earlier matched nodes
    // (distinct by injectivity) has at least nout in-arcs, and likewise for
    // in-lists: thresholds those lists already guarantee are dropped, so
    // the kernels only gather degrees that can still prune.
    for (int l = 1; l < k; l++) {
        XmLevel& L = D.lv[l];
        int nout = 0, nin = 0;
        for (int i = 0; i < L.nops; i++) (L.op_dir[i] == XM_DIR_OUT ? nout : nin)++;
        if (L.din_min <= nout) L.din_min = 0;
        if (L.dout_min <= nin) L.dout_min = 0;
    }

    // Leaf-product sets: each is a level over the prefix p = k - r, with the
    // operands, order bounds (against the prefix) of its member levels and
    // injectivity against the prefix nodes no operand or bound excludes.
    // It may start from a complete prefix set (Sec. 5.2) whose operands it
    // contains, whose bounds hold for it and whose degree thresholds every
    // member's candidates meet.
    if (pc.r) {
        const int p = k - pc.r;
        const uint32_t prefix = (1u << p) - 1;
        D.prod_p = p;
        D.prod_r = pc.r;
        D.prod_kind = pc.kind;
        D.prod_nv = pc.kind == XM_PROD_CHOOSE ? 1 : (1 << pc.r) - 1;
        for (int si = 0; si < D.prod_nv; si++) {
            const uint32_t members = (uint32_t)si + 1;
            XmLevel& V = D.pv[si];
            memset(&V, 0, sizeof V);
            V.reuse = -1;
            uint32_t adj = 0, mverts = 0;
            int dmax_out = 0, dmax_in = 0;
            for (int j = 0; j < pc.r; j++) {
                if (!(members >> j & 1u)) continue;
                const XmLevel& M = D.lv[p + j];
                const int v = order[p + j];
                mverts |= 1u << v;
                for (int i = 0; i < M.nops; i++) {
                    bool have = false;
                    for (int q = 0; q < V.nops; q++)
                        if (V.op_level[q] == M.op_level[i] && V.op_dir[q] == M.op_dir[i]) have = true;
                    if (!have) {
                        V.op_level[V.nops] = M.op_level[i];
                        V.op_dir[V.nops] = M.op_dir[i];
                        V.nops++;
                    }
                    adj |= 1u << M.op_level[i];
                }
                V.lo_mask |= M.lo_mask & prefix;
                V.hi_mask |= M.hi_mask & prefix;
                dmax_out = std::max(dmax_out, P.dout[v]);
                dmax_in = std::max(dmax_in, P.din[v]);
            }
            V.neq_mask = prefix & ~adj & ~V.lo_mask & ~V.hi_mask;
            if (!reduce) continue;
            int best = -1, best_ops = 0;
            uint32_t best_mask = 0;
            for (int r = 1; r < p; r++) {
                const XmLevel& Rl = D.lv[r];
                if (Rl.nops == 0 || Rl.ndiff) continue;
                if (Rl.dout_min > dmax_out || Rl.din_min > dmax_in) continue;
                uint32_t mask = 0;
                bool subset = true;
                for (int i = 0; i < Rl.nops && subset; i++) {
                    int found = -1;
                    for (int q = 0; q < V.nops; q++)
                        if (V.op_level[q] == Rl.op_level[i] && V.op_dir[q] == Rl.op_dir[i]) found = q;
                    if (found < 0) subset = false; else mask |= 1u << found;
                }
                if (!subset) continue;
                bool bounds_ok = true;
                for (int j = 0; j < r && bounds_ok; j++) {
                    const int u = order[j];
                    bool lo_implied = false, hi_implied = false;
                    for (int v = 0; v < k; v++) {
                        if (!(mverts >> v & 1u)) continue;
                        if (lt[u] >> v & 1u) lo_implied = true;
                        if (lt[v] >> u & 1u) hi_implied = true;
                    }
                    if ((Rl.lo_mask >> j & 1u) && !lo_implied) bounds_ok = false;
                    if ((Rl.hi_mask >> j & 1u) && !hi_implied) bounds_ok = false;
                }
                if (!bounds_ok) continue;
                if (Rl.nops > best_ops || (Rl.nops == best_ops && r > best)) {
                    best = r;
                    best_ops = Rl.nops;
                    best_mask = mask;
                }
            }
            if (best >= 0) {
                V.reuse = best;
                V.reuse_ops = best_mask;
            }
        }
    }

    out.dev = D;
    out.k = k;
    out.e = e;
    out.flags = flags;
    out.aut_size = (int)aut.size();
    out.stab_size = (int)sym.size();
    out.n_reuse = n_reuse;
    out.start = R.start;
    out.split = R.split;
    out.covered_by = R.covered_by;
    out.psrc.assign(psrc, psrc + e);
    out.pdst.assign(pdst, pdst + e);
    out.decomp.reset();
    // Counting by a cut vertex, when the plan still walks three or more
    // levels (a product at level 2 is cheaper than any split).
    if (root < 0 && k >= 4 && !(flags & (XM_INDUCED | XM_NO_SPLIT)) && (D.prod_r == 0 || D.prod_p >= 3)) {
        bool start_fixed = true;
        for (auto& g : aut)
            if (g[out.start] != out.start) start_fixed = false;
        int rc = decompose(P, flags, out, err, start_fixed);
        if (rc) return rc;
    }
    return XM_OK;
}

std::string describe_plan(const Plan& p) {
    std::string s;
    char buf[256];
    snprintf(buf, sizeof buf, "k=%d e=%d |Aut|=%d start=%d reuse_levels=%d flags=%d\n", p.k, p.e, p.aut_size,
             p.start, p.n_reuse, p.flags);
    s += buf;
    s += "split:";
    for (int ed : p.split) {
        snprintf(buf, sizeof buf, " (%d,%d)", p.psrc[ed], p.pdst[ed]);
        s += buf;
    }
    s += "\ncovered:";
    for (int ed = 0; ed < p.e; ed++)
        if (p.covered_by[ed] >= 0) {
            int c = p.covered_by[ed];
            snprintf(buf, sizeof buf, " (%d,%d)<=(%d,%d)", p.psrc[ed], p.pdst[ed], p.psrc[c], p.pdst[c]);
            s += buf;
        }
    s += "\n";
    const XmPlanDev& D = p.dev;
    for (int l = 0; l < D.k; l++) {
        const XmLevel& L = D.lv[l];
        snprintf(buf, sizeof buf, "L%d v%d deg>=(%d,%d) ops:", l, D.order[l], L.dout_min, L.din_min);
        s += buf;
        for (int i = 0; i < L.nops; i++) {
            snprintf(buf, sizeof buf, " %s(L%d)", L.op_dir[i] == XM_DIR_OUT ? "out" : "in", L.op_level[i]);
            s += buf;
        }
        snprintf(buf, sizeof buf, " reuse=%d/0x%x lo=0x%x hi=0x%x neq=0x%x", L.reuse, L.reuse_ops, L.lo_mask,
                 L.hi_mask, L.neq_mask);
        s += buf;
        for (int i = 0; i < L.ndiff; i++) {
            snprintf(buf, sizeof buf, " not-%s(L%d)", L.diff_dir[i] == XM_DIR_OUT ? "out" : "in", L.diff_level[i]);
            s += buf;
        }
        s += "\n";
    }
    if (D.prod_r) {
        snprintf(buf, sizeof buf, "product: level %d r=%d kind=%s sets=%d\n", D.prod_p, D.prod_r,
                 D.prod_kind == XM_PROD_CHOOSE ? "choose" : "incl-excl", D.prod_nv);
        s += buf;
        for (int i = 0; i < D.prod_nv; i++) {
            const XmLevel& V = D.pv[i];
            snprintf(buf, sizeof buf, "P%d ops:", i + 1);
            s += buf;
            for (int q = 0; q < V.nops; q++) {
                snprintf(buf, sizeof buf, " %s(L%d)", V.op_dir[q] == XM_DIR_OUT ? "out" : "in", V.op_level[q]);
                s += buf;
            }
            snprintf(buf, sizeof buf, " reuse=%d/0x%x lo=0x%x hi=0x%x neq=0x%x\n", V.reuse, V.reuse_ops, V.lo_mask,
                     V.hi_mask, V.neq_mask);
            s += buf;
        }
    }
    if (p.decomp) {
        snprintf(buf, sizeof buf, "cut-vertex split: cut %d, %d parts, %d quotients, start-node subsets %s\n",
                 p.decomp->cut, (int)p.decomp->parts.size(), (int)p.decomp->quots.size(),
                 p.decomp->rooted ? "split" : "walked");
        s += buf;
    }
    return s;
}

}  // namespace xm
