/*
 * CPU oracle for directed subgraph matching (test infrastructure only).
 *
 * This file is test infrastructure: only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark load it. The product path never
 * does, and it shares no code with the GPU library.
 *
 * It computes the plain definition of the matching problem of the XMiner
 * paper (Sec. 2, Def. 2.1 digraph, Def. 2.2 pattern graph, the vertex/edge
 * constraints that follow it):
 *   - the data graph G = (V, E) is a digraph; repeated arcs and self-loops
 *     of the input arc list are dropped;
 *   - an embedding of a pattern P = (V_P, E_P) is an injective map
 *     m: V_P -> V with (m(u), m(v)) in E for every pattern arc (u, v)
 *     (non-induced: further arcs among matched nodes are allowed);
 *   - a match (a distinct matched subgraph) is an orbit of embeddings under
 *     the automorphism group Aut(P); the matches are the embeddings that are
 *     lexicographically smallest within their orbit, and
 *     #matches = #embeddings / |Aut(P)|.
 * Induced variant (the induced-subgraph reading of "isomorphic and oriented
 * the same", Sec. 2): additionally, for every ordered pair of pattern
 * vertices (u, v) WITHOUT a pattern arc, (m(u), m(v)) must NOT be an arc;
 * a match is then a node set whose induced subgraph is isomorphic to P.
 * The matcher is single-threaded backtracking over the original (unreduced)
 * pattern, visiting pattern vertices in breadth-first order from a chosen
 * root vertex, checking every pattern arc to an already matched vertex by
 * binary search in a sorted out-list, and injectivity by a scan.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    int64_t m;
    int64_t *out_off; /* n + 1 */
    int32_t *out_adj; /* m, each out-list ascending */
    int64_t *in_off;
    int32_t *in_adj;  /* m, each in-list ascending */
} og_graph;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Bucket the arcs by one endpoint, sort each bucket and drop repeats. */
static int build_side(int32_t n, int64_t m, const int32_t *key, const int32_t *val,
                      int64_t **off_out, int32_t **adj_out) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!off || !adj || !fill) { free(off); free(adj); free(fill); return -1; }
    for (int64_t i = 0; i < m; i++)
        if (key[i] != val[i]) off[key[i] + 1]++;
    for (int32_t v = 0; v < n; v++) off[v + 1] += off[v];
    memcpy(fill, off, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < m; i++)
        if (key[i] != val[i]) adj[fill[key[i]]++] = val[i];
    /* sort and deduplicate each list, compacting in place */
    int64_t w = 0;
    for (int32_t v = 0; v < n; v++) {
        int64_t lo = off[v], hi = off[v + 1];
        qsort(adj + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_i32);
        off[v] = w;
        for (int64_t i = lo; i < hi; i++)
            if (i == lo || adj[i] != adj[i - 1]) adj[w++] = adj[i];
    }
    off[n] = w;
    free(fill);
    *off_out = off;
    *adj_out = adj;
    return 0;
}

og_graph *og_build(int32_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    if (n < 0 || m < 0) return NULL;
    for (int64_t i = 0; i < m; i++)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return NULL;
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    if (!g) return NULL;
    g->n = n;
    if (build_side(n, m, src, dst, &g->out_off, &g->out_adj) ||
        build_side(n, m, dst, src, &g->in_off, &g->in_adj)) {
        free(g->out_off); free(g->out_adj); free(g->in_off); free(g->in_adj); free(g);
        return NULL;
    }
    g->m = g->out_off[n];
    return g;
}

void og_free(og_graph *g) {
    if (!g) return;
    free(g->out_off); free(g->out_adj); free(g->in_off); free(g->in_adj);
    free(g);
}

int64_t og_num_arcs(const og_graph *g) { return g->m; }

/* Copies the deduplicated out-CSR (offsets n+1, adjacency m) to the caller. */
void og_out_csr(const og_graph *g, int64_t *off, int32_t *adj) {
    memcpy(off, g->out_off, ((size_t)g->n + 1) * sizeof(int64_t));
    memcpy(adj, g->out_adj, (size_t)g->m * sizeof(int32_t));
}

/* Is (u, v) an arc? Binary search in u's sorted out-list. */
static int has_arc(const og_graph *g, int32_t u, int32_t v) {
    int64_t lo = g->out_off[u], hi = g->out_off[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->out_adj[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < g->out_off[u + 1] && g->out_adj[lo] == v;
}

int og_has_arc(const og_graph *g, int32_t u, int32_t v) { return has_arc(g, u, v); }

/* ------------------------------------------------------------ Aut(P) ---- */

#define OG_MAXK 8

static int pattern_arc(int k, int e, const int32_t *ps, const int32_t *pd, int u, int v) {
    (void)k;
    for (int i = 0; i < e; i++)
        if (ps[i] == u && pd[i] == v) return 1;
    return 0;
}

/* All permutations s of {0..k-1} that map the arc set onto itself. Writes
 * them (k entries each) into perms when it is not NULL and returns |Aut|. */
int og_aut(int k, int e, const int32_t *ps, const int32_t *pd, int32_t *perms) {
    if (k < 1 || k > OG_MAXK) return -1;
    int p[OG_MAXK], used[OG_MAXK] = {0}, depth = 0, count = 0;
    int next[OG_MAXK + 1];
    next[0] = 0;
    /* iterative depth-first generation of permutations */
    while (depth >= 0) {
        if (depth == k) {
            int ok = 1;
            for (int i = 0; i < e && ok; i++)
                ok = pattern_arc(k, e, ps, pd, p[ps[i]], p[pd[i]]);
            if (ok) {
                if (perms) memcpy(perms + (size_t)count * k, p, k * sizeof(int32_t));
                count++;
            }
            depth--;
            if (depth >= 0) used[p[depth]] = 0;
            continue;
        }
        int c = next[depth];
        while (c < k && used[c]) c++;
        if (c >= k) {
            depth--;
            if (depth >= 0) used[p[depth]] = 0;
            continue;
        }
        p[depth] = c;
        used[c] = 1;
        next[depth] = c + 1;
        depth++;
        next[depth] = 0;
    }
    return count;
}

/* ------------------------------------------------------- backtracking --- */

typedef struct {
    const og_graph *g;
    int k, e;
    const int32_t *ps, *pd;
    int order[OG_MAXK];        /* pattern vertex visited at each depth */
    int pos[OG_MAXK];          /* depth of each pattern vertex */
    int parent[OG_MAXK];       /* earlier pattern neighbour used to draw candidates, or -1 */
    int parent_out[OG_MAXK];   /* 1: arc parent -> v (scan parent's out-list), 0: arc v -> parent */
    int32_t m[OG_MAXK];        /* m[v] = data node matched to pattern vertex v */
    int32_t r_lo, r_hi;        /* allowed data nodes for the root vertex */
    int induced;               /* 1: non-arcs of the pattern must be non-arcs of G */
    /* match output */
    int unique_only;
    int naut;
    const int32_t *aut;
    unsigned __int128 count;
    int32_t *out;
    int64_t capacity;
    /* work cap: candidates examined so far, the cap (0: none), set when hit */
    uint64_t steps, max_steps;
    int gave_up;
} og_search;

/* breadth-first order over the undirected pattern from `root`, neighbours by
 * ascending id; unreached vertices (disconnected pattern) follow in id order */
static void bfs_order(og_search *s, int root) {
    int seen[OG_MAXK] = {0}, head = 0, tail = 0;
    s->order[tail++] = root;
    seen[root] = 1;
    for (;;) {
        while (head < tail) {
            int u = s->order[head++];
            for (int v = 0; v < s->k; v++)
                if (!seen[v] && (pattern_arc(s->k, s->e, s->ps, s->pd, u, v) ||
                                 pattern_arc(s->k, s->e, s->ps, s->pd, v, u))) {
                    seen[v] = 1;
                    s->order[tail++] = v;
                }
        }
        if (tail == s->k) break;
        for (int v = 0; v < s->k; v++)
            if (!seen[v]) { seen[v] = 1; s->order[tail++] = v; break; }
    }
    for (int d = 0; d < s->k; d++) s->pos[s->order[d]] = d;
    for (int d = 0; d < s->k; d++) {
        int v = s->order[d];
        s->parent[v] = -1;
        for (int j = 0; j < d && s->parent[v] < 0; j++) {
            int u = s->order[j];
            if (pattern_arc(s->k, s->e, s->ps, s->pd, u, v)) { s->parent[v] = u; s->parent_out[v] = 1; }
            else if (pattern_arc(s->k, s->e, s->ps, s->pd, v, u)) { s->parent[v] = u; s->parent_out[v] = 0; }
        }
    }
}

/* Does candidate x for pattern vertex v (at depth d) satisfy injectivity and
 * every pattern arc to the vertices matched before it? */
static int consistent(const og_search *s, int d, int v, int32_t x) {
    for (int j = 0; j < d; j++)
        if (s->m[s->order[j]] == x) return 0;
    for (int i = 0; i < s->e; i++) {
        int a = s->ps[i], b = s->pd[i];
        if (a == v && s->pos[b] < d && !has_arc(s->g, x, s->m[b])) return 0;
        if (b == v && s->pos[a] < d && !has_arc(s->g, s->m[a], x)) return 0;
    }
    if (s->induced) {
        for (int j = 0; j < d; j++) {
            int u = s->order[j];
            if (!pattern_arc(s->k, s->e, s->ps, s->pd, u, v) && has_arc(s->g, s->m[u], x)) return 0;
            if (!pattern_arc(s->k, s->e, s->ps, s->pd, v, u) && has_arc(s->g, x, s->m[u])) return 0;
        }
    }
    return 1;
}

/* Is the embedding m the lexicographically smallest tuple of its orbit
 * {(m[s(0)], ..., m[s(k-1)]) : s in Aut(P)}? */
static int is_orbit_min(const og_search *s) {
    for (int a = 0; a < s->naut; a++) {
        const int32_t *sg = s->aut + (size_t)a * s->k;
        for (int i = 0; i < s->k; i++) {
            int32_t t = s->m[sg[i]];
            if (t < s->m[i]) return 0;
            if (t > s->m[i]) break;
        }
    }
    return 1;
}

static void record(og_search *s) {
    if (s->unique_only && !is_orbit_min(s)) return;
    if (s->out && (int64_t)s->count < s->capacity)
        memcpy(s->out + (size_t)s->count * s->k, s->m, s->k * sizeof(int32_t));
    s->count++;
}

/* One more candidate examined; 1 when the work cap is exceeded. */
static int over_cap(og_search *s) {
    s->steps++;
    if (s->max_steps && s->steps > s->max_steps) s->gave_up = 1;
    return s->gave_up;
}

static void extend(og_search *s, int d) {
    if (d == s->k) { record(s); return; }
    int v = s->order[d];
    if (d == 0) {
        for (int32_t x = s->r_lo; x < s->r_hi && !s->gave_up; x++) {
            s->m[v] = x;
            extend(s, 1);
        }
        return;
    }
    int u = s->parent[v];
    if (u < 0) { /* no matched neighbour: every node is a candidate */
        for (int32_t x = 0; x < s->g->n && !over_cap(s); x++)
            if (consistent(s, d, v, x)) { s->m[v] = x; extend(s, d + 1); }
        return;
    }
    const og_graph *g = s->g;
    int32_t mu = s->m[u];
    const int32_t *list = s->parent_out[v] ? g->out_adj + g->out_off[mu] : g->in_adj + g->in_off[mu];
    int64_t len = s->parent_out[v] ? g->out_off[mu + 1] - g->out_off[mu] : g->in_off[mu + 1] - g->in_off[mu];
    for (int64_t i = 0; i < len && !over_cap(s); i++) {
        int32_t x = list[i];
        if (consistent(s, d, v, x)) { s->m[v] = x; extend(s, d + 1); }
    }
}

static int setup(og_search *s, const og_graph *g, int k, int e, const int32_t *ps, const int32_t *pd,
                 int root, int32_t r_lo, int32_t r_hi, int induced) {
    if (k < 1 || k > OG_MAXK || root < 0 || root >= k) return -1;
    memset(s, 0, sizeof *s);
    s->induced = induced;
    s->g = g; s->k = k; s->e = e; s->ps = ps; s->pd = pd;
    s->r_lo = r_lo < 0 ? 0 : r_lo;
    s->r_hi = r_hi > g->n ? g->n : r_hi;
    bfs_order(s, root);
    return 0;
}

/* Number of embeddings whose root pattern vertex maps into [r_lo, r_hi), as
 * a 128-bit value (lo, hi). */
int og_count_embeddings(const og_graph *g, int k, int e, const int32_t *ps, const int32_t *pd, int root,
                        int32_t r_lo, int32_t r_hi, int induced, uint64_t *lo, uint64_t *hi) {
    og_search s;
    if (setup(&s, g, k, e, ps, pd, root, r_lo, r_hi, induced)) return -1;
    extend(&s, 0);
    *lo = (uint64_t)s.count;
    *hi = (uint64_t)(s.count >> 64);
    return 0;
}

/* og_count_embeddings that gives up after examining max_steps candidates
 * (summed over all levels of the walk): returns 1 (no count) when it gave
 * up, 0 with the exact count otherwise. */
int og_count_embeddings_capped(const og_graph *g, int k, int e, const int32_t *ps, const int32_t *pd, int root,
                               int32_t r_lo, int32_t r_hi, int induced, uint64_t max_steps, uint64_t *lo,
                               uint64_t *hi) {
    og_search s;
    if (setup(&s, g, k, e, ps, pd, root, r_lo, r_hi, induced)) return -1;
    s.max_steps = max_steps;
    extend(&s, 0);
    if (s.gave_up) return 1;
    *lo = (uint64_t)s.count;
    *hi = (uint64_t)(s.count >> 64);
    return 0;
}

/* Number of matches (embeddings that are the smallest of their Aut-orbit). */
int og_count_matches(const og_graph *g, int k, int e, const int32_t *ps, const int32_t *pd, int induced,
                     uint64_t *lo, uint64_t *hi) {
    og_search s;
    if (setup(&s, g, k, e, ps, pd, 0, 0, g->n, induced)) return -1;
    int32_t *aut = (int32_t *)malloc(40320 * OG_MAXK * sizeof(int32_t));
    if (!aut) return -1;
    s.naut = og_aut(k, e, ps, pd, aut);
    s.aut = aut;
    s.unique_only = 1;
    extend(&s, 0);
    free(aut);
    *lo = (uint64_t)s.count;
    *hi = (uint64_t)(s.count >> 64);
    return 0;
}

/* Writes up to `capacity` matches (k node ids each, in pattern-vertex order,
 * each the orbit-smallest embedding) in search order; returns the total
 * number of matches. */
int64_t og_enumerate(const og_graph *g, int k, int e, const int32_t *ps, const int32_t *pd, int induced,
                     int32_t *out, int64_t capacity) {
    og_search s;
    if (setup(&s, g, k, e, ps, pd, 0, 0, g->n, induced)) return -1;
    int32_t *aut = (int32_t *)malloc(40320 * OG_MAXK * sizeof(int32_t));
    if (!aut) return -1;
    s.naut = og_aut(k, e, ps, pd, aut);
    s.aut = aut;
    s.unique_only = 1;
    s.out = out;
    s.capacity = capacity;
    extend(&s, 0);
    free(aut);
    return (int64_t)s.count;
}

/* Writes up to `capacity` embeddings whose root pattern vertex maps into
 * [r_lo, r_hi) (k node ids each, in pattern-vertex order) in search order;
 * returns how many there are. Every embedding is written, not one per orbit. */
int64_t og_enumerate_embeddings(const og_graph *g, int k, int e, const int32_t *ps, const int32_t *pd, int root,
                                int32_t r_lo, int32_t r_hi, int induced, int32_t *out, int64_t capacity) {
    og_search s;
    if (setup(&s, g, k, e, ps, pd, root, r_lo, r_hi, induced)) return -1;
    s.out = out;
    s.capacity = capacity;
    extend(&s, 0);
    return (int64_t)s.count;
}

/* |a ∩ b| of two ascending lists: each id of the shorter looked up in the
 * longer by binary search. */
static uint64_t common_ids(const int32_t *a, int64_t na, const int32_t *b, int64_t nb) {
    if (na > nb) { const int32_t *t = a; a = b; b = t; int64_t tn = na; na = nb; nb = tn; }
    uint64_t c = 0;
    for (int64_t i = 0; i < na; i++) {
        int64_t lo = 0, hi = nb;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (b[mid] < a[i]) lo = mid + 1; else hi = mid;
        }
        if (lo < nb && b[lo] == a[i]) c++;
    }
    return c;
}

/* Triangle sums over the arcs (u, w) whose source u lies in [u_lo, u_hi):
 *   *ffl = sum |N_out(u) ∩ N_in(w)|: the nodes x with u -> x -> w besides
 *          u -> w, i.e. the feed-forward triangles whose source is in the
 *          range; over all u this is sum(A o A^2);
 *   *cyc = sum |N_out(w) ∩ N_in(u)|: the closed walks u -> w -> x -> u
 *          starting with such an arc; over all u this is tr(A^3), three
 *          times the number of directed 3-cycles.
 * (No self-loops, so x differs from u and w in both sums.) */
void og_triangle_sums(const og_graph *g, int32_t u_lo, int32_t u_hi, uint64_t *ffl, uint64_t *cyc) {
    uint64_t f = 0, c = 0;
    if (u_lo < 0) u_lo = 0;
    if (u_hi > g->n) u_hi = g->n;
    for (int32_t u = u_lo; u < u_hi; u++) {
        const int32_t *ou = g->out_adj + g->out_off[u], *iu = g->in_adj + g->in_off[u];
        const int64_t nou = g->out_off[u + 1] - g->out_off[u], niu = g->in_off[u + 1] - g->in_off[u];
        for (int64_t j = 0; j < nou; j++) {
            const int32_t w = ou[j];
            f += common_ids(ou, nou, g->in_adj + g->in_off[w], g->in_off[w + 1] - g->in_off[w]);
            c += common_ids(g->out_adj + g->out_off[w], g->out_off[w + 1] - g->out_off[w], iu, niu);
        }
    }
    *ffl = f;
    *cyc = c;
}

/* Replaces each k-tuple (an embedding written in pattern-vertex order) by the
 * lexicographically smallest tuple of its Aut-orbit. */
void og_canonicalize(int k, int naut, const int32_t *aut, int64_t ntup, const int32_t *in, int32_t *out) {
    for (int64_t t = 0; t < ntup; t++) {
        const int32_t *m = in + (size_t)t * k;
        int32_t best[OG_MAXK];
        memcpy(best, m, k * sizeof(int32_t));
        for (int a = 0; a < naut; a++) {
            const int32_t *sg = aut + (size_t)a * k;
            int cmp = 0;
            for (int i = 0; i < k && cmp == 0; i++) {
                int32_t x = m[sg[i]];
                cmp = (x < best[i]) ? -1 : (x > best[i]) ? 1 : 0;
            }
            if (cmp < 0)
                for (int i = 0; i < k; i++) best[i] = m[sg[i]];
        }
        memcpy(out + (size_t)t * k, best, k * sizeof(int32_t));
    }
}
