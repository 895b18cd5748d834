/*
 * xm.h -- C ABI of the B300 directed subgraph matcher.
 *
 * Method: XMiner, "Efficient Directed Subgraph Matching with Pattern
 * Reduction" (Yuan, Wang, Ma, He, Liu; arXiv 2404.11105).
 *
 * Problem (Sec. 2, Defs. 2.1-2.2 and the vertex/edge constraints after
 * them): a data digraph G = (V, E) and a weakly connected pattern digraph
 * P = (V_P, E_P) given by its arc list (Sec. 5.4: users state a pattern by
 * listing its edges). An embedding is an injective map m: V_P -> V with
 * (m(u), m(v)) in E for every pattern arc (u, v); further arcs among the
 * matched nodes are allowed (non-induced). A match is a distinct matched
 * subgraph, i.e. an orbit of embeddings under Aut(P); results are unique
 * (Sec. 5.3). By default the library counts/enumerates matches; with
 * XM_EMBEDDINGS it counts every embedding (= |Aut(P)| x matches).
 *
 * Conventions for every entry point:
 *   - Return value: XM_OK (0) or an XM_E* status. Nothing is thrown across
 *     the ABI. On error the output arguments are left untouched unless the
 *     function says otherwise; xm_strerror() names the status and
 *     xm_last_error() gives a one-line detail for the calling thread.
 *   - Ownership: handles (xm_graph, xm_plan) belong to the library until
 *     the matching *_free call. Input arrays are borrowed for the duration
 *     of the call and copied. Output buffers belong to the caller.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that
 *     run kernels enqueue them on `stream` and return after the results
 *     they report have been copied back (they synchronise `stream`).
 *   - Node ids are int32 in [0, n). Data graphs need fewer than 2^31 arcs
 *     after deduplication. Counts are 128-bit, returned as (lo, hi) halves.
 *   - A graph handle owns one set of device scratch buffers; calls that use
 *     the same graph handle must not overlap in time (serialise them on one
 *     stream). Different graph handles are independent.
 */
#ifndef XM_H
#define XM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    XM_OK = 0,
    XM_EINVAL = 1,    /* bad argument: ids out of range, bad pattern, ... */
    XM_ENOMEM = 2,    /* host or device allocation failed */
    XM_EOVERFLOW = 3, /* enumeration buffer too small; *total is still exact */
    XM_ECUDA = 4,     /* a CUDA runtime call failed (no device, launch error) */
    XM_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    XM_EBUSY = 6      /* resource in use */
};

/* ------------------------------------------------------ pattern flags */
enum {
    XM_REDUCE = 0,     /* default: plan from the reduced pattern (Alg. 1, Sec. 5.1-5.2) */
    XM_NO_REDUCE = 1,  /* plan over the original pattern, no reuse of candidate sets
                          (the "XMiner without reduction" variant of Sec. 6.3) */
    XM_EMBEDDINGS = 2, /* count every embedding; no symmetry-breaking conditions */
    XM_INDUCED = 4,    /* induced matching: a pair of pattern vertices without an arc must map to a
                          pair of nodes without that arc (DIFF operands); the paper defines only
                          edge and degree constraints, so this is an extension */
    XM_NO_PRODUCT = 8, /* count by walking every level: no leaf products (see xm_plan_product) */
    XM_NO_SPLIT = 16   /* count with the whole pattern: no cut-vertex decomposition (see xm_plan_split) */
};

typedef struct xm_graph_s *xm_graph;
typedef struct xm_plan_s *xm_plan;

/* Name of a status code (static string). */
const char *xm_strerror(int status);

/* Detail of the last error raised on the calling thread (static per-thread
 * buffer, "" when none). */
const char *xm_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int xm_version(void);

/*
 * xm_fault_inject -- host-side fault injection, for tests of the error
 * paths (no GPU fault is ever involved). spec: "alloc:N" makes the N-th
 * device allocation of the library from now on fail as if the device were
 * out of memory (the call reports XM_ENOMEM and releases what it had
 * allocated); "compile:N" makes the N-th xm_compile_pattern from now on fail
 * with XM_ENOMEM; several items comma-separated; "none" clears both. The
 * environment variable XM_FAULT, read when the library loads, takes the same
 * spec. Errors: XM_EINVAL for a malformed spec (nothing changes).
 */
int xm_fault_inject(const char *spec);

/* Device memory currently held by the library (all handles), in bytes. */
uint64_t xm_device_bytes_live(void);

/* ------------------------------------------------------------- graphs */

/*
 * xm_load_graph -- build the data digraph on the current CUDA device.
 *
 * Def. 2.1 (digraph); the per-node out_arcs / in_arcs lists that plan
 * execution reads (Alg. 2, its two initialisation branches).
 *
 *   n          number of nodes; ids are [0, n). 1 <= n < 2^31.
 *   m          number of input arcs (src[i] -> dst[i]), m >= 0.
 *   src, dst   arc endpoints, m int32 each, host or device memory (detected
 *              with cudaPointerGetAttributes). Repeated arcs and
 *              self-loops are dropped.
 *   flags      reserved, pass 0.
 *   stream     stream for the uploads.
 *   out        receives the handle.
 *
 * Builds a dual sorted CSR (out-lists and in-lists, each ascending, int32
 * offsets) on the device, in memory owned by the handle: host arcs are
 * uploaded, the arcs are packed into 64-bit (src, dst) keys, radix-sorted,
 * and repeats and self-loops are dropped; the in-lists come from the keys
 * with their halves swapped and sorted again. Then come the handle's scratch
 * buffers (about 12 bytes per node and 12 bytes per arc) and a hash index of
 * the lists of at least 32 ids (up to 16 bytes per arc, built one thread
 * per list entry). The build's temporaries (about 16 bytes per input arc
 * for the keys, plus the uploaded arcs) are freed before the call returns.
 * Synchronises `stream`.
 * Errors: XM_EINVAL for n/m out of range or an id outside [0, n), or more
 * than 2^31-1 arcs after deduplication; XM_ENOMEM; XM_ECUDA.
 */
int xm_load_graph(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int flags, void *stream,
                  xm_graph *out);

/* Node count and arc count after deduplication. */
int xm_graph_info(xm_graph g, int32_t *n, int64_t *m);

/*
 * Device pointers of the dual CSR (read-only views owned by the handle):
 * out_off/in_off have n+1 int32 entries, out_adj/in_adj have m.
 */
int xm_graph_csr(xm_graph g, const int32_t **out_off, const int32_t **out_adj, const int32_t **in_off,
                 const int32_t **in_adj);

/* Frees the handle and its device memory. NULL is a no-op. */
void xm_graph_free(xm_graph g);

/* ----------------------------------------------------------- patterns */

/*
 * xm_compile_pattern -- host-only pattern compiler.
 *
 * Follows Sec. 4 and Sec. 5.1-5.2:
 *   1. constraint inclusion among pattern edges and vertices (Thm. 2.1,
 *      Thm. 2.2, the neighbour grouping of Sec. 4.1, closed to a fixpoint);
 *   2. pattern reduction by the greedy constraint cover of Alg. 1 (start at
 *      the highest-degree vertex; repeatedly take the adjacent edge of
 *      highest coverage; mark included edges as covered);
 *   3. plan generation (Sec. 5.1): a materialisation order of the pattern
 *      vertices, and for each vertex the lists it intersects (out-lists of
 *      matched in-neighbours, in-lists of matched out-neighbours), the
 *      earlier candidate set it reuses (Sec. 5.2), degree thresholds, and
 *      symmetry-breaking order conditions (Sec. 7 mentions symmetry
 *      destruction without a mechanism; the library uses the stabiliser-
 *      chain conditions of Grochow and Kellis, RECOMB 2007).
 *
 *   k          pattern vertices, 2 <= k <= 8 (vertices are 0..k-1).
 *   e          pattern arcs, 1 <= e <= k(k-1).
 *   psrc, pdst arc endpoints (host memory), e int32 each.
 *   flags      XM_REDUCE (0) | XM_NO_REDUCE | XM_EMBEDDINGS | XM_INDUCED |
 *              XM_NO_PRODUCT | XM_NO_SPLIT.
 *   out        receives the plan handle.
 * Errors: XM_EINVAL for a self-loop, a repeated arc, an id outside [0, k),
 * k or e out of range, or a pattern that is not weakly connected.
 */
int xm_compile_pattern(int32_t k, int32_t e, const int32_t *psrc, const int32_t *pdst, int flags,
                       xm_plan *out);

/*
 * xm_plan_info -- summary of a compiled plan (any pointer may be NULL).
 *   k         pattern vertices;
 *   aut_size  |Aut(P)|;
 *   n_levels  levels of the plan (= k);
 *   n_reuse   levels whose candidate set starts from an earlier level's
 *             set (Sec. 5.2 reuse); 0 with XM_NO_REDUCE;
 *   start     the pattern vertex matched first (Alg. 1 maxDegree).
 */
int xm_plan_info(xm_plan p, int32_t *k, int32_t *aut_size, int32_t *n_levels, int32_t *n_reuse,
                 int32_t *start);

/*
 * xm_plan_order -- the plan's materialisation order: order[l] is the
 * pattern vertex matched at level l (k entries, caller-owned).
 */
int xm_plan_order(xm_plan p, int32_t *order);

/*
 * xm_plan_describe -- human-readable plan (levels, operand lists, reuse,
 * filters, reduction queue), NUL-terminated, truncated to cap bytes.
 * Returns the length the full text needs (excluding the NUL) or -XM_EINVAL.
 */
int xm_plan_describe(xm_plan p, char *buf, int32_t cap);

/*
 * xm_plan_level -- the flat plan IR record of one level (for inspection and
 * tests). Level l matches pattern vertex `vertex`; its candidates are the
 * intersection of the operand lists i < nops: the out-list (op_dir 0) or
 * in-list (op_dir 1) of the node matched at level op_level[i]. With
 * reuse >= 1 the operands in bit set reuse_ops may be replaced by level
 * `reuse`'s stored candidate set (Sec. 5.2). Filters: x > m(j) for bits j of
 * lo_mask, x < m(j) for hi_mask, x != m(j) for neq_mask; outdeg(x) >=
 * dout_min and indeg(x) >= din_min. Errors: XM_EINVAL for a bad level.
 */
typedef struct {
    int32_t vertex;
    int32_t nops;
    int32_t op_level[14];
    int32_t op_dir[14];
    int32_t reuse;
    uint32_t reuse_ops;
    int32_t dout_min;
    int32_t din_min;
    uint32_t lo_mask;
    uint32_t hi_mask;
    uint32_t neq_mask;
    int32_t ndiff;          /* induced plans: lists the candidate must NOT be in */
    int32_t diff_level[14];
    int32_t diff_dir[14];
} xm_level_info;

int xm_plan_level(xm_plan p, int32_t level, xm_level_info *out);

/*
 * xm_plan_product -- the plan's leaf product (Sec. 5.3: when only the count
 * is wanted, the sizes of the candidate sets of the vertices left once the
 * active nodes are matched are multiplied instead of enumerated).
 *
 * Unless XM_NO_PRODUCT or XM_INDUCED is given, the compiler looks for 2..3
 * pattern vertices (up to k-2 when they are interchangeable) that share no
 * arc and whose removal leaves the pattern weakly connected, and moves them
 * to the end of the materialisation order. Their candidate sets then depend
 * only on the nodes matched before them, so xm_count stops at the first of
 * them (level `level`) and adds, for each partial match, the number of
 * ways to pick pairwise distinct nodes from the r sets:
 *   kind 1 (choose): one common set C and a total order imposed by the
 *     symmetry conditions: C(|C|, r);
 *   kind 2 (inclusion-exclusion, r <= 3): |C_0||C_1| - |C_0 & C_1| for
 *     r = 2, and the alternating sum over set partitions for r = 3. The
 *     paper multiplies the set sizes without correcting for nodes that lie
 *     in several sets; the correction keeps matches injective.
 * xm_enumerate ignores the product and walks all k levels.
 *
 *   level, r, kind  product level p, number of product vertices r (0: no
 *                   product), kind (0 none, 1 choose, 2 inclusion-exclusion);
 *   n_sets          records readable with xm_plan_product_set: 1 for kind 1,
 *                   2^r - 1 for kind 2.
 * Any pointer may be NULL. Errors: XM_EINVAL for a NULL plan.
 */
int xm_plan_product(xm_plan p, int32_t *level, int32_t *r, int32_t *kind, int32_t *n_sets);

/*
 * xm_plan_product_set -- set record i of the leaf product, in the layout of
 * xm_plan_level (vertex = -1; operands, bounds and injectivity refer to
 * levels < p only; no degree thresholds). Kind 1: record 0 is the common
 * set. Kind 2: record s - 1 is the intersection of the sets of the product
 * vertices in bit mask s (bit j = level p + j).
 * Errors: XM_EINVAL for a NULL plan or i outside [0, n_sets).
 */
int xm_plan_product_set(xm_plan p, int32_t i, xm_level_info *out);

/*
 * xm_plan_split -- the plan's cut-vertex decomposition, used by xm_count.
 *
 * When the pattern has a cut vertex c (a vertex whose removal splits it into
 * parts A_1..A_t, t >= 2) and the plan would walk three or more levels,
 * xm_count counts with the parts instead of the whole pattern: for each
 * node v the embeddings of every A_i + c that map c to v are counted
 * (rooted plans, one launch per part), their products are summed over v
 * (one more kernel), and the embeddings of the quotient patterns -- the
 * pattern with vertices of different parts identified, which the products
 * also count -- are subtracted (each counted by its own plan, recursively).
 * This extends the paper's count-by-multiplication (Sec. 5.3) from single
 * vertices to whole parts; the subtraction keeps matches injective. Cut
 * vertex choice: most parts, then the smallest largest part, then the
 * lowest id. Not with XM_INDUCED or XM_NO_SPLIT, nor when a leaf product
 * already stops the walk at level 2, nor beyond 4096 quotient partitions.
 * xm_count_range, xm_count_roots, xm_count_stats, the enumerations, batches,
 * the server and xm_count_noalloc always walk the plan itself.
 *
 *   cut          the cut vertex, or -1 when the plan has no decomposition;
 *   n_parts      t;  n_quotients  distinct quotient patterns (up to
 *                isomorphism);
 *   part_factor  product over the parts of the automorphisms of A_i + c
 *                that fix c (rooted plans count one embedding per orbit).
 * Any pointer may be NULL. Errors: XM_EINVAL for a NULL plan.
 */
int xm_plan_split(xm_plan p, int32_t *cut, int32_t *n_parts, int32_t *n_quotients, int64_t *part_factor);

/*
 * xm_plan_split_part -- part i of the decomposition as a pattern A_i + c
 * with its vertices relabelled 0..k-1, c being 0: k, e arcs psrc/pdst
 * (caller arrays of >= 56 entries), vertices[j] = the original pattern
 * vertex of label j (>= 8 entries), stab = automorphisms of A_i + c fixing
 * c. Any output pointer may be NULL.
 * Errors: XM_EINVAL for a NULL plan, no decomposition or i out of range.
 */
int xm_plan_split_part(xm_plan p, int32_t i, int32_t *k, int32_t *e, int32_t *psrc, int32_t *pdst,
                       int32_t *vertices, int32_t *stab);

/*
 * xm_plan_split_quotient -- quotient pattern i (k vertices, e arcs into
 * caller arrays of >= 56 entries; the cut vertex is 0) and mult, the number
 * of identifications of vertices across parts that yield it. Any output
 * pointer may be NULL.
 * Errors: XM_EINVAL for a NULL plan, no decomposition or i out of range.
 */
int xm_plan_split_quotient(xm_plan p, int32_t i, int32_t *k, int32_t *e, int32_t *psrc, int32_t *pdst,
                           int64_t *mult);

/* Frees a plan. NULL is a no-op. */
void xm_plan_free(xm_plan p);

/* ------------------------------------------------------------- tuning */

/*
 * Launch parameters of the matcher (0 = library default):
 *   window           candidate-window capacity per plan level, in node
 *                    ids (multiple of 32, 64..4096);
 *   unit             positions of the first level's candidate list handed
 *                    out as one work unit (1..65536);
 *   warps_per_block  1..16;
 *   blocks_per_sm    resident blocks per SM to launch (persistent grid);
 *   budget_ms        work budget: when the matcher has run this long (GPU
 *                    global timer) every warp stops at its next check and
 *                    the call returns XM_ETIMEOUT with no count (0 = none).
 *                    The kernel always finishes and the context stays
 *                    usable;
 *   merge_ratio      intersection strategy of counted last levels with two
 *                    lists (Alg. 2's A^{e.dest} cap Pi A^e): the longer list,
 *                    cut to the shorter one's id range, is merged with it
 *                    (both streamed in coalesced 16-byte loads) when it is at
 *                    most merge_ratio times as long, and otherwise probed
 *                    once per id of the shorter list (hash table, or binary
 *                    search for lists under 32 ids). 1..1024; 0 = default
 *                    (8); -1 = never merge. Counts never depend on it.
 */
typedef struct {
    int32_t window;
    int32_t unit;
    int32_t warps_per_block;
    int32_t blocks_per_sm;
    int32_t budget_ms;  /* device-time budget of one call's matcher kernel, 0 = none */
    int32_t merge_ratio;
} xm_tuning;

/* Sets the tuning used by later calls with this plan (copied). */
int xm_plan_set_tuning(xm_plan p, const xm_tuning *t);
/* Reads back the effective tuning. */
int xm_plan_get_tuning(xm_plan p, xm_tuning *t);

/*
 * xm_plan_tune -- autotuner for one (plan, graph) pair: runs xm_count once
 * per candidate to warm up, then `reps` times, timed with the graph's CUDA
 * events (xm_graph_last_timing); keeps the fastest candidate as the plan's
 * tuning and reports it. Every candidate must give the same count (else
 * XM_EINVAL). Synchronises `stream`.
 */
int xm_plan_tune(xm_graph g, xm_plan p, const xm_tuning *cand, int32_t ncand, int32_t reps, xm_tuning *best,
                 float *best_ms, void *stream);

/*
 * xm_plan_tune_roots -- xm_plan_tune on the counts of a start-node list
 * (xm_count_roots; roots: host array of nroots node ids, as there), for
 * workloads that count a sample of the start nodes.
 */
int xm_plan_tune_roots(xm_graph g, xm_plan p, const int32_t *roots, int64_t nroots, const xm_tuning *cand,
                       int32_t ncand, int32_t reps, xm_tuning *best, float *best_ms, void *stream);

/* ------------------------------------------------------------ matching */

/*
 * xm_count -- number of matches of plan p in graph g (Alg. 2 plan
 * execution with count-only result generation, Sec. 5.3).
 * Uses the plan's leaf product (xm_plan_product) and, for the whole graph,
 * its cut-vertex decomposition (xm_plan_split: several launches and host
 * steps, per-node counters of 16 B x n per part allocated with the graph
 * on first use). Writes the 128-bit count as (*lo, *hi). Synchronises
 * `stream`.
 * Errors: XM_EINVAL (NULL handle/output), XM_ETIMEOUT (tuning budget spent
 * in one of the launches), XM_ENOMEM, XM_ECUDA.
 */
int xm_count(xm_graph g, xm_plan p, uint64_t *lo, uint64_t *hi, void *stream);

/*
 * xm_count_range -- as xm_count, restricted to the matches whose start
 * vertex (xm_plan_info's `start`) is mapped to a node in [root_lo, root_hi)
 * (Alg. 2 parallelises over the start vertex's candidates). Counts over a
 * partition of [0, n) add up to xm_count. Ranges are clipped to [0, n).
 * Uses the leaf product, and the cut-vertex decomposition when its cut
 * vertex is the start vertex and every automorphism of the pattern fixes
 * it (xm_plan_describe: "start-node subsets split"): then all embeddings of
 * a match map the cut vertex to the same node, so the per-node form of the
 * split identity holds, with the quotient patterns counted rooted at the
 * cut vertex over the same start nodes. Otherwise the plan is walked.
 */
int xm_count_range(xm_graph g, xm_plan p, int64_t root_lo, int64_t root_hi, uint64_t *lo, uint64_t *hi,
                   void *stream);

/*
 * Work and traffic counters of one instrumented run (xm_count_stats). The
 * instrumented kernels take exactly the code paths of the counting kernels
 * (same driver ranges, leaf shortcuts, merge-or-probe choices), so the
 * bytes describe the timed work.
 *   alg_bytes     algorithmic bytes of the persistent matcher (the kernel
 *                 xm_graph_last_timing reports as match_ms): per list operand
 *                 8 B of offsets; 4 B per driver id scanned; for every other
 *                 list the cheaper of scanning it or probing it once per
 *                 driver id, 4 B x min(|L|, |C| x ceil(log2(|L|+1))) with
 *                 |L| cut to the driver range's ids where the kernel computes
 *                 that cut (two-list last levels); 4 B x ceil(log2(L+1)) per
 *                 bound search in a list of L ids; 8 B per degree check;
 *   extensions    partial matches created (descents into a level);
 *   set_ops       candidate sets computed (level set-ups);
 *   units         work units executed;
 *   leaf_elems    driver elements examined at the last level;
 *   l1_bytes      algorithmic bytes of the first-level pass (prep_ms): 16 B
 *                 per start node checked, the first level's lists as above,
 *                 8 B per first-level candidate written with its owner;
 *   touched_bytes bytes the matcher's chosen strategies move at 32-byte-sector
 *                 granularity if nothing were cached (a merge reads both
 *                 ranges, a hash probe one sector, a binary search one sector
 *                 per step above the last sector, offsets one sector);
 *   warp_exit_first_ns / _mean_ns / _last_ns
 *                 load balance of the instrumented matcher's persistent grid:
 *                 when its warps ran out of work (earliest, mean, latest), in
 *                 ns of the GPU global timer after the first warp started.
 */
typedef struct {
    uint64_t alg_bytes;
    uint64_t extensions;
    uint64_t set_ops;
    uint64_t units;
    uint64_t leaf_elems;
    uint64_t l1_bytes;
    uint64_t touched_bytes;
    uint64_t warp_exit_first_ns;
    uint64_t warp_exit_mean_ns;
    uint64_t warp_exit_last_ns;
} xm_stats;

/*
 * xm_count_stats -- xm_count_range with the counters above (a separately
 * compiled, slower kernel; for measurement, not for timing). Through a
 * cut-vertex split the counters are summed over the instrumented passes of
 * the parts and rooted quotients (load-balance times: the last pass's).
 */
int xm_count_stats(xm_graph g, xm_plan p, int64_t root_lo, int64_t root_hi, uint64_t *lo, uint64_t *hi,
                   xm_stats *stats, void *stream);

/*
 * xm_enumerate -- materialise the matches (Sec. 5.3 result generation).
 *
 *   dev_out   caller-owned device buffer of capacity * k int32; match i is
 *             written at dev_out[i*k .. i*k+k-1] in pattern-vertex order
 *             (entry v is the node matched to pattern vertex v).
 *   capacity  number of matches dev_out can hold.
 *   total     receives the exact number of matches (always).
 *   written   receives min(total, capacity).
 * One embedding per match is written (the one meeting the plan's
 * symmetry-breaking conditions; every embedding with XM_EMBEDDINGS).
 * The order of matches is unspecified. Returns XM_EOVERFLOW when total >
 * capacity (the first `capacity` slots are filled, total stays exact).
 */
int xm_enumerate(xm_graph g, xm_plan p, int32_t *dev_out, uint64_t capacity, uint64_t *total,
                 uint64_t *written, void *stream);

/*
 * xm_count_roots / xm_enumerate_roots -- as xm_count / xm_enumerate,
 * restricted to the matches whose start vertex is mapped to one of the
 * given nodes (the paper's runs from a given percentage of start nodes,
 * Sec. 6.4). roots: host array of nroots node ids in [0, n) (copied; sorted
 * and deduplicated by the call). Counts over a partition of the nodes add
 * up to xm_count. Errors: XM_EINVAL for an id outside [0, n) or nroots > n.
 */
int xm_count_roots(xm_graph g, xm_plan p, const int32_t *roots, int64_t nroots, uint64_t *lo, uint64_t *hi,
                   void *stream);
int xm_enumerate_roots(xm_graph g, xm_plan p, const int32_t *roots, int64_t nroots, int32_t *dev_out,
                       uint64_t capacity, uint64_t *total, uint64_t *written, void *stream);
/*
 * xm_count_roots_each -- per-start-node counts: counts[2i], counts[2i+1]
 * (host, caller-owned, 2 * nroots uint64) receive the 128-bit count (lo,
 * hi) of the matches whose start vertex is mapped to roots[i] (embeddings
 * with XM_EMBEDDINGS), in the caller's order; a node listed twice gets its
 * count twice. One launch for all nodes: the matcher adds each work unit's
 * count to a 128-bit device counter of its start node (Alg. 2 runs the
 * start nodes as independent tasks, so the per-node counts add up to
 * xm_count_roots). Uses the plan's leaf product, and the cut-vertex
 * decomposition where xm_count_range does (one launch per part and per
 * rooted quotient, combined per node on the host). Device counters: 16 B per
 * distinct root per launch, allocated with the graph on first use. Errors as
 * xm_count_roots, XM_ENOMEM.
 */
int xm_count_roots_each(xm_graph g, xm_plan p, const int32_t *roots, int64_t nroots, uint64_t *counts,
                        void *stream);

/* xm_count_roots with the xm_count_stats counters. */
int xm_count_roots_stats(xm_graph g, xm_plan p, const int32_t *roots, int64_t nroots, uint64_t *lo, uint64_t *hi,
                         xm_stats *stats, void *stream);

/* xm_enumerate restricted to start nodes in [root_lo, root_hi). */
int xm_enumerate_range(xm_graph g, xm_plan p, int64_t root_lo, int64_t root_hi, int32_t *dev_out,
                       uint64_t capacity, uint64_t *total, uint64_t *written, void *stream);

/*
 * xm_graph_last_timing -- device time of the last count/enumerate call on
 * this graph handle, from CUDA events recorded on the call's stream around
 * its kernels: *prep_ms covers the first-level, work-unit and scan kernels,
 * *match_ms the persistent matcher kernel, each summed over the call's
 * matching passes (one, or one per part and quotient of a cut-vertex split;
 * the split's product kernel and host steps are not included). Either
 * pointer may be NULL.
 * Errors: XM_EINVAL (no call yet), XM_ECUDA.
 */
int xm_graph_last_timing(xm_graph g, float *prep_ms, float *match_ms);

/* ------------------------------------------------------------- batches */

/*
 * Batched matching: many independent (pattern, graph) matching problems in
 * one persistent kernel launch. Not in the paper, which runs one pattern on
 * one graph; each pair's count is exactly what xm_count returns for it. A
 * pair walks its plan with the plan's leaf product (Sec. 5.3), never the
 * cut-vertex decomposition.
 *
 * xm_batch_create -- describe a batch.
 *   np, plans    compiled plans (borrowed handles; they must outlive the
 *                batch only until this call returns: plans are copied).
 *   ng, graphs   graph handles on the current device (must outlive the
 *                batch: their device memory is read at every run).
 *   npairs       number of (plan, graph) pairs, >= 1.
 *   pair_pg      host array of 2*npairs int32: pair i matches plan
 *                pair_pg[2i] against graph pair_pg[2i+1].
 *   out          receives the batch handle (device descriptor, counters).
 * Errors: XM_EINVAL for bad indices/handles, XM_ENOMEM, XM_ECUDA.
 */
typedef struct xm_batch_s *xm_batch;
int xm_batch_create(int32_t np, const xm_plan *plans, int32_t ng, const xm_graph *graphs, int64_t npairs,
                    const int32_t *pair_pg, xm_batch *out);

/*
 * Launch parameters of the batched kernel: `unit` is the number of start
 * nodes per work unit, `window` the candidate window per level, plus warps
 * per block and blocks per SM (0 = defaults 64, 256, 8, max resident).
 * Synchronous (re-uploads the unit table when `unit` changes).
 */
int xm_batch_set_tuning(xm_batch b, const xm_tuning *t);
int xm_batch_get_tuning(xm_batch b, xm_tuning *t);

/*
 * xm_batch_run -- enqueue one run on `stream`: zero the counters, launch the
 * batched kernel. Does not synchronise and allocates nothing.
 * xm_batch_run_graph -- the same work replayed from a CUDA graph captured
 * on the first call (on a private stream); later calls only launch the
 * graph on `stream`.
 * xm_batch_counts -- copy the 128-bit count of every pair (2 uint64 per
 * pair, lo then hi) into the host array out_counts; synchronises `stream`.
 * Returns XM_ETIMEOUT (counts incomplete) when the run exceeded the batch
 * tuning's budget_ms.
 */
int xm_batch_run(xm_batch b, void *stream);
int xm_batch_run_graph(xm_batch b, void *stream);
int xm_batch_counts(xm_batch b, uint64_t *out_counts, void *stream);

/*
 * xm_batch_tune -- autotuner: times each of the ncand candidate tunings
 * (one warm-up run, then the fastest of `reps` event-timed runs on
 * `stream`), keeps the fastest as the batch's tuning and reports it.
 */
int xm_batch_tune(xm_batch b, const xm_tuning *cand, int32_t ncand, int32_t reps, xm_tuning *best, float *best_ms,
                  void *stream);

/*
 * xm_batch_set_pair_budget -- a device-time budget for every work unit of
 * every pair of the batch (0 = none; the default). A work unit (one block of
 * start nodes of one pair) that has run this long since it started (GPU
 * global timer) stops, its pair's remaining units are skipped and
 * xm_batch_pair_status reports XM_ETIMEOUT for the pair; its count is
 * incomplete. Time a unit waits behind other pairs' units is not charged. The other pairs finish exactly, and xm_batch_counts still
 * returns XM_OK. The tuning's budget_ms, which ends the whole launch, stays
 * separate. Drops a captured CUDA graph (captured again on the next
 * xm_batch_run_graph).
 *
 * xm_batch_pair_status -- after a run: status[i] = XM_OK or XM_ETIMEOUT for
 * pair i (host array of npairs int32). Synchronises `stream`.
 */
int xm_batch_set_pair_budget(xm_batch b, int32_t budget_ms);
int xm_batch_pair_status(xm_batch b, int32_t *status, void *stream);

/* Frees a batch. NULL is a no-op. */
void xm_batch_free(xm_batch b);

/*
 * xm_count_batch -- one-shot batch: create, run, read the counts
 * (out_counts: host, 2 uint64 per pair), free. Synchronises `stream`.
 */
int xm_count_batch(int32_t np, const xm_plan *plans, int32_t ng, const xm_graph *graphs, int64_t npairs,
                   const int32_t *pair_pg, uint64_t *out_counts, void *stream);

/* ------------------------------------------------------------- serving */

/*
 * Serving: graphs stay resident; count queries are admitted into one of a
 * fixed number of slots when a slot is free and the query's scratch fits
 * the memory budget; each slot runs its query's kernels on its own stream,
 * so a query admitted while others are on the GPU overlaps with them
 * (continuous batching driven by the caller's loop). Not in the paper.
 *
 * xm_query_bytes -- the admission estimate of a count query of plan p on
 * graph g: the device scratch of the pipeline (about 4 bytes x (3n +
 * 3.001m) plus control data). Intermediate partial matches are never
 * materialised (bounded per-warp windows), so this is the whole
 * per-query device footprint.
 *
 * xm_server_create -- ng graph handles (borrowed; they must outlive the
 * server), nslots (1..256) concurrent queries, mem_budget_bytes the
 * admission budget over the queries in flight.
 *
 * xm_server_submit -- try to admit a count query of plan p on graph
 * `graph_index`, labelled `tag`. Never blocks: *admitted = 1 when it was
 * enqueued, 0 when no slot or not enough budget is free now (retry after a
 * poll). The plan is copied; its tuning applies (budget_ms bounds the
 * query's device time: such a query completes with XM_ETIMEOUT).
 * Errors: XM_EINVAL (bad index, or a query larger than the whole budget).
 *
 * xm_server_poll -- collect finished queries: up to max_results entries of
 * tags[i], counts[2i..2i+1] (128-bit lo, hi) and status[i] (XM_OK or
 * XM_ETIMEOUT); *n_done receives how many. wait != 0 first blocks until the
 * oldest query in flight has finished.
 *
 * xm_server_info -- busy slots and scratch bytes in flight.
 * xm_server_free -- waits for the queries in flight, then frees the server.
 */
typedef struct xm_server_s *xm_server;
uint64_t xm_query_bytes(xm_graph g, xm_plan p);
int xm_server_create(int32_t ng, const xm_graph *graphs, int32_t nslots, uint64_t mem_budget_bytes, xm_server *out);
int xm_server_submit(xm_server s, xm_plan p, int32_t graph_index, int64_t tag, int32_t *admitted);
int xm_server_poll(xm_server s, int32_t wait, int32_t max_results, int64_t *tags, uint64_t *counts, int32_t *status,
                   int32_t *n_done);
int xm_server_info(xm_server s, int32_t *busy_slots, uint64_t *bytes_in_flight);
void xm_server_free(xm_server s);

/*
 * xm_count_noalloc -- xm_count for callers that cannot allocate device
 * memory. The paper has no counterpart: this is a deployment variant of
 * xm_count, not a step of the method.
 *
 * Who needs it: a process that has given all device memory to its own pool
 * allocator up front, or a latency-critical loop that must not call
 * cudaMalloc/cudaFree (they may synchronise the whole device). xm_count
 * keeps its scratch in buffers that xm_load_graph allocates; this entry
 * point allocates nothing and instead uses one fixed scratch area of
 * XM_NOALLOC_SCRATCH_BYTES that lives in the library as a file-scope
 * device array (every GPU that loads the library holds it until the process
 * exits).
 *
 *   out_off, out_adj, in_off, in_adj
 *             the data graph as device arrays owned by the caller, in the
 *             layout xm_graph_csr exposes: int32 offsets (n+1 each) and
 *             ascending, repeat-free, self-loop-free out- and in-lists (m
 *             each; in_adj must be the transpose of out_adj).
 *   n, m      nodes and arcs of that CSR.
 *   p         compiled plan (its tuning applies).
 *   lo, hi    receive the 128-bit count, exactly as xm_count would.
 *   stream    stream for the kernels; the call synchronises it.
 *
 * Limits and errors: XM_EINVAL when the scratch the graph needs (about
 * 4 bytes x (3n + 3.001m) plus small control data) exceeds
 * XM_NOALLOC_SCRATCH_BYTES -- use xm_count then --, for NULL/invalid
 * sizes, or when out_off[n] or in_off[n] differs from m (the call reads
 * those two entries back before launching anything); XM_ECUDA when a CUDA
 * call fails.
 * Set-up: the first call on each device looks up the scratch array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before capturing any stream into a CUDA graph.
 * Concurrency: all calls on a device share the one scratch area and keep
 * the previous call's contents (the call clears what must start at zero).
 * Calls whose work overlaps on the GPU race with each other; serialise them
 * (for example, one stream).
 */
#define XM_NOALLOC_SCRATCH_BYTES (32u << 20)
int xm_count_noalloc(const int32_t *out_off, const int32_t *out_adj, const int32_t *in_off, const int32_t *in_adj,
                     int32_t n, int64_t m, xm_plan p, uint64_t *lo, uint64_t *hi, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* XM_H */
