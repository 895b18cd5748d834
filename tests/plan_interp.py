"""Slow CPU interpreter of the flat plan IR (test helper, not product code).

It executes a compiled plan level by level exactly as the IR states
(operand lists, reuse of an earlier level's stored candidate set, order
bounds, injectivity and degree filters) so that the compiler's output can
be checked against the oracle on tiny graphs without a GPU. It shares no
code with the device matcher or with the oracle.
"""
from __future__ import annotations


def adjacency_lists(n, src, dst):
    out = [set() for _ in range(n)]
    inn = [set() for _ in range(n)]
    for u, v in zip(src, dst):
        u, v = int(u), int(v)
        if u != v:
            out[u].add(v)
            inn[v].add(u)
    return out, inn


def run_plan(n, out, inn, plan, use_reuse=True):
    k = plan.k
    levels = [plan.level(l) for l in range(k)]
    m = [0] * k
    stored = [None] * k
    total = 0

    def candidates(l):
        L = levels[l]
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
        last = l == k - 1
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

    def go(l):
        nonlocal total
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
