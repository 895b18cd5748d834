"""Slow CPU interpreter of the flat plan IR (test helper, not product code).

It executes a compiled plan level by level exactly as the IR states
(operand lists, reuse of an earlier level's stored candidate set, order
bounds, injectivity and degree filters) so that the compiler's output can
be checked against the oracle on tiny graphs without a GPU. It shares no
code with the device matcher or with the oracle.
"""
from __future__ import annotations

import itertools


def adjacency_lists(n, src, dst):
    out = [set() for _ in range(n)]
    inn = [set() for _ in range(n)]
    for u, v in zip(src, dst):
        u, v = int(u), int(v)
        if u != v:
            out[u].add(v)
            inn[v].add(u)
    return out, inn


def run_plan(n, out, inn, plan, use_reuse=True, use_product=True):
    """Count as the plan states. With a leaf product the walk stops at the
    product level and adds the number of tuples of distinct nodes, one from
    each product vertex's set, counted here by brute force over the sets (not
    by the inclusion-exclusion formula the device uses)."""
    k = plan.k
    levels = [plan.level(l) for l in range(k)]
    prod = plan.product() if use_product else {"r": 0}
    m = [0] * k
    stored = [None] * k
    total = 0

    def candidates(l, L=None, last=None):
        L = levels[l] if L is None else L
        lo = max((m[j] for j in range(l) if L["lo_mask"] >> j & 1), default=-1)
        hi = min((m[j] for j in range(l) if L["hi_mask"] >> j & 1), default=n)
        if l == 0:
            base = set(range(n))
        else:
            lists = []
            if use_reuse and L["reuse"] >= 1:
                lists.append(stored[L["reuse"]])
                ops = [op for i, op in enumerate(L["ops"]) if not (L["reuse_ops"] >> i & 1)]
            else:
                ops = L["ops"]
            for j, d in ops:
                lists.append(out[m[j]] if d == 0 else inn[m[j]])
            base = set.intersection(*[set(x) for x in lists])
        res = set()
        last = (l == k - 1) if last is None else last
        for x in base:
            if not (lo < x < hi):
                continue
            if any(x == m[j] for j in range(l) if L["neq_mask"] >> j & 1):
                continue
            if any(x in (out[m[j]] if d == 0 else inn[m[j]]) for j, d in L.get("diffs", [])):
                continue
            if not last and (len(out[x]) < L["dout_min"] or len(inn[x]) < L["din_min"]):
                continue
            res.add(x)
        return res

    def product_count(p):
        r = prod["r"]
        if prod["kind"] == 1:
            # one common set, vertices totally ordered: increasing tuples
            c = sorted(candidates(p, prod["sets"][0], last=True))
            return sum(1 for t in itertools.combinations(c, r))
        sets = [candidates(p, prod["sets"][(1 << j) - 1], last=True) for j in range(r)]
        return sum(1 for t in itertools.product(*[sorted(x) for x in sets]) if len(set(t)) == r)

    def go(l):
        nonlocal total
        if prod["r"] and l == prod["level"]:
            total += product_count(l)
            return
        c = candidates(l)
        if l == k - 1:
            total += len(c)
            return
        stored[l] = c
        for x in sorted(c):
            m[l] = x
            go(l + 1)

    go(0)
    return total
