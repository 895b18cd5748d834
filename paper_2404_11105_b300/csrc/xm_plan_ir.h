// Flat plan IR shared by the host pattern compiler and the device matcher.
//
// One record per plan level l = 0..k-1; level l matches pattern vertex
// order[l]. Level 0 is the start vertex (Alg. 1 maxDegree): its candidates
// are the nodes passing the degree filter (the "init A^{p.start}" step of
// Alg. 2). For l >= 1 the candidate set is
//
//   C_l = { x in  AND_i L_i  :  x passes the filters of level l }
//
// where each operand list L_i is N_out(m_j) (pattern arc order[j] ->
// order[l]) or N_in(m_j) (pattern arc order[l] -> order[j]) of a node m_j
// matched at an earlier level j (Alg. 2: A^{e.dest} = A^{e.dest} cap
// Pi_{e.dest} A^e). With reuse r >= 1, the operand lists flagged in
// reuse_ops are already intersected in level r's stored candidate set, which
// is used in their place when it is held complete in shared memory
// (Sec. 5.2 intermediate-result reuse). Filters:
//   - order bounds: x > m_j for j in lo_mask, x < m_j for j in hi_mask
//     (symmetry-breaking conditions);
//   - injectivity: x != m_j for j in neq_mask (levels not already excluded
//     by an operand list or an order bound);
//   - degree: outdeg(x) >= dout_min and indeg(x) >= din_min (vertex
//     constraint of Sec. 2; skipped at the last level, where it cannot
//     prune);
//   - difference (induced plans only): x not in N_out(m_j) for each
//     (diff_level, diff_dir = OUT) -- no pattern arc order[j] -> order[l] --
//     and x not in N_in(m_j) for (j, IN) -- no arc order[l] -> order[j].
#pragma once
#include <stdint.h>

#define XM_MAXK 8
#define XM_MAXOPS 14  // an out- and an in-list from each of up to 7 earlier levels

enum { XM_DIR_OUT = 0, XM_DIR_IN = 1 };

struct XmLevel {
    int32_t nops;
    int32_t op_level[XM_MAXOPS];
    int32_t op_dir[XM_MAXOPS];
    int32_t reuse;       // earlier level whose stored set may replace some operands, or -1
    uint32_t reuse_ops;  // bit i: operand i is already applied in level `reuse`'s set
    int32_t dout_min;
    int32_t din_min;
    uint32_t lo_mask;
    uint32_t hi_mask;
    uint32_t neq_mask;
    int32_t ndiff;
    int32_t diff_level[XM_MAXOPS];
    int32_t diff_dir[XM_MAXOPS];
};

// Leaf products (Sec. 5.3: a count multiplies the sizes of the candidate
// sets of the vertices still open once the active nodes are fixed). When
// prod_r > 0 the last r = prod_r levels p = prod_p .. k-1 match pattern
// vertices that share no arc, so each one's candidate set depends on levels
// < p only; counting stops at level p and adds, per partial match
// m_0..m_{p-1}, the number of tuples of pairwise distinct nodes drawn one
// from each set:
//   XM_PROD_CHOOSE: the r sets are one set C (same operands and bounds) and
//     the symmetry conditions order the r vertices totally: C(|C|, r);
//     pv[0] describes C;
//   XM_PROD_IE (r <= 3): sets C_0..C_{r-1}; inclusion-exclusion over the
//     set partitions of the r vertices: r = 2: |C_0||C_1| - |C_0 & C_1|;
//     r = 3: |C_0||C_1||C_2| - |C_0&C_1||C_2| - |C_0&C_2||C_1|
//            - |C_1&C_2||C_0| + 2|C_0&C_1&C_2|;
//     pv[s - 1] describes the intersection over the members in bitmask s.
// A pv[] record is a level over operands of levels < p (order bounds and
// injectivity against those levels only, no degree filter). Enumeration
// ignores the products and walks all k levels.
#define XM_MAXPV 7
enum { XM_PROD_NONE = 0, XM_PROD_CHOOSE = 1, XM_PROD_IE = 2 };

struct XmPlanDev {
    int32_t k;
    int32_t order[XM_MAXK];  // pattern vertex of each level
    int32_t prod_p, prod_r, prod_kind, prod_nv;
    XmLevel lv[XM_MAXK];
    XmLevel pv[XM_MAXPV];
};
