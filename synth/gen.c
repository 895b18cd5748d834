/*
 * Seeded synthetic inputs for directed subgraph matching.
 *
 * This module only draws inputs: arc lists of data digraphs and arc lists of
 * pattern digraphs. It holds none of the matching arithmetic, so both the
 * CPU oracle and the GPU path can read the very same inputs.
 *
 * Random numbers come from two published generators:
 *   - splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 *     generators", OOPSLA 2014) turns a 64-bit seed into state words;
 *   - xoshiro256** (Blackman, Vigna, "Scrambled linear pseudorandom number
 *     generators", ACM TOMS 2021) draws the stream.
 * Bulk generators work in fixed blocks of arcs, each block seeding its own
 * xoshiro256** state from (seed, block index), so the output does not depend
 * on the number of threads.
 *
 * Graph families:
 *   - directed Erdos-Renyi G(n, m): exactly m distinct arcs drawn uniformly
 *     from the n(n-1) ordered pairs u != v (rejection of repeats/self-loops);
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): 2^scale nodes,
 *     edge_factor * 2^scale arcs, each arc picks one quadrant per level with
 *     probabilities a, b, c, d = 1-a-b-c; no noise, no relabelling.
 *     Repeated arcs and self-loops are left in: loaders drop them.
 *   - random patterns: k vertices, each ordered pair kept with probability
 *     rho, redrawn until weakly connected.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xoshiro256ss;

static inline uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

static inline uint64_t xo_next(xoshiro256ss *g) {
    uint64_t *s = g->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static inline void xo_seed(xoshiro256ss *g, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ULL);
    for (int i = 0; i < 4; i++) g->s[i] = splitmix64_next(&x);
}

/* uniform double in [0, 1) from the top 53 bits */
static inline double xo_uniform(xoshiro256ss *g) {
    return (double)(xo_next(g) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, bound) by Lemire's multiply-shift with rejection */
static inline uint64_t xo_below(xoshiro256ss *g, uint64_t bound) {
    for (;;) {
        uint64_t r = xo_next(g);
        unsigned __int128 p = (unsigned __int128)r * bound;
        uint64_t lo = (uint64_t)p;
        if (lo >= bound || lo >= (uint64_t)(-bound) % bound) return (uint64_t)(p >> 64);
    }
}

/* ---------------------------------------------------------------- ER ---- */

/* open-addressing set of 64-bit keys (key 0 reserved as empty; we store
 * key+1) */
typedef struct { uint64_t *t; uint64_t mask; } u64set;

static int set_init(u64set *h, uint64_t cap) {
    uint64_t sz = 16;
    while (sz < cap * 2) sz <<= 1;
    h->t = (uint64_t *)calloc(sz, sizeof(uint64_t));
    h->mask = sz - 1;
    return h->t ? 0 : -1;
}

static int set_insert(u64set *h, uint64_t key) { /* 1 if newly inserted */
    uint64_t k = key + 1;
    uint64_t i = (k * 0x9E3779B97F4A7C15ULL) >> 7;
    for (;;) {
        i &= h->mask;
        if (h->t[i] == 0) { h->t[i] = k; return 1; }
        if (h->t[i] == k) return 0;
        i++;
    }
}

/* Directed G(n, m): m distinct arcs, no self-loops. Returns 0, or -1 when
 * m exceeds n(n-1) or memory runs out. */
int synth_er(int32_t n, int64_t m, uint64_t seed, int32_t *src, int32_t *dst) {
    if (n < 2 || m < 0 || (double)m > (double)n * (double)(n - 1)) return -1;
    xoshiro256ss g;
    xo_seed(&g, seed, 0);
    u64set h;
    if (set_init(&h, (uint64_t)m + 1)) return -1;
    int64_t got = 0;
    while (got < m) {
        uint64_t u = xo_below(&g, (uint64_t)n), v = xo_below(&g, (uint64_t)n);
        if (u == v) continue;
        if (!set_insert(&h, (u << 32) | v)) continue;
        src[got] = (int32_t)u;
        dst[got] = (int32_t)v;
        got++;
    }
    free(h.t);
    return 0;
}

/* -------------------------------------------------------------- R-MAT --- */

#define RMAT_BLOCK 4096

/* Writes edge_factor * 2^scale arcs (repeats and self-loops included). */
int synth_rmat(int scale, int64_t n_arcs, double a, double b, double c, uint64_t seed,
               int32_t *src, int32_t *dst) {
    if (scale < 1 || scale > 30 || n_arcs < 0) return -1;
    const double ab = a + b, abc = a + b + c;
    const int64_t nblocks = (n_arcs + RMAT_BLOCK - 1) / RMAT_BLOCK;
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nblocks; blk++) {
        xoshiro256ss g;
        xo_seed(&g, seed, (uint64_t)blk + 1);
        int64_t lo = blk * RMAT_BLOCK, hi = lo + RMAT_BLOCK;
        if (hi > n_arcs) hi = n_arcs;
        for (int64_t e = lo; e < hi; e++) {
            uint32_t u = 0, v = 0;
            for (int l = 0; l < scale; l++) {
                double r = xo_uniform(&g);
                uint32_t bu, bv;
                if (r < a) { bu = 0; bv = 0; }
                else if (r < ab) { bu = 0; bv = 1; }
                else if (r < abc) { bu = 1; bv = 0; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            src[e] = (int32_t)u;
            dst[e] = (int32_t)v;
        }
    }
    return 0;
}

/* Keeps the first n_keep node ids of an arc list: arcs with an endpoint at or
 * above n_keep are dropped. Returns the number of arcs kept (compacted in
 * place). Used to trim an R-MAT graph of 2^ceil(log2 n) nodes to n nodes. */
int64_t synth_trim(int64_t m, int32_t n_keep, int32_t *src, int32_t *dst) {
    int64_t w = 0;
    for (int64_t i = 0; i < m; i++) {
        if (src[i] < n_keep && dst[i] < n_keep) { src[w] = src[i]; dst[w] = dst[i]; w++; }
    }
    return w;
}

/* ---------------------------------------------------------- patterns ---- */

static int weakly_connected(int k, const uint8_t *adj /* k*k */) {
    int seen = 1, stack[16], top = 0;
    stack[top++] = 0;
    while (top) {
        int u = stack[--top];
        for (int v = 0; v < k; v++) {
            if (!(seen >> v & 1) && (adj[u * k + v] || adj[v * k + u])) {
                seen |= 1 << v;
                stack[top++] = v;
            }
        }
    }
    return seen == (1 << k) - 1;
}

/* One random weakly connected pattern with k vertices: every ordered pair
 * (u, v), u != v, is an arc with probability rho; redrawn until weakly
 * connected. Arcs are written in (u, v) lexicographic order. Returns the
 * number of arcs, or -1 on bad arguments. `stream` selects an independent
 * draw for the same seed. */
int synth_pattern(int k, double rho, uint64_t seed, uint64_t stream, int32_t *psrc, int32_t *pdst) {
    if (k < 2 || k > 8 || !(rho > 0.0) || rho > 1.0) return -1;
    xoshiro256ss g;
    xo_seed(&g, seed, stream);
    uint8_t adj[64];
    for (int attempt = 0; attempt < 1000000; attempt++) {
        memset(adj, 0, sizeof adj);
        for (int u = 0; u < k; u++)
            for (int v = 0; v < k; v++)
                if (u != v && xo_uniform(&g) < rho) adj[u * k + v] = 1;
        if (!weakly_connected(k, adj)) continue;
        int e = 0;
        for (int u = 0; u < k; u++)
            for (int v = 0; v < k; v++)
                if (adj[u * k + v]) { psrc[e] = u; pdst[e] = v; e++; }
        return e;
    }
    return -1;
}

/* Plain uniform doubles / integers for Python-side recipes (sizes, degrees). */
void synth_uniform(uint64_t seed, uint64_t stream, int64_t count, double *out) {
    xoshiro256ss g;
    xo_seed(&g, seed, stream);
    for (int64_t i = 0; i < count; i++) out[i] = xo_uniform(&g);
}
