"""Brute-force restatement of the analysis for tiny inputs (pure Python).

Independent of the oracle's loops: every quantity is recomputed by enumerating
all candidates -- the iteration of a sample by re-scanning its rank from the
start, each (rank, iteration, context) cell by a sum over all samples, each
inclusive cell by testing ancestry of every sample's context, statistics with
exact rational arithmetic (fractions.Fraction).
"""
from __future__ import annotations

import math
from fractions import Fraction

NONE = 0xFFFFFFFF


def samples(tr, r):
    b, e = int(tr["rank_off"][r]), int(tr["rank_off"][r + 1])
    return [(int(tr["ts"][i]), int(tr["ctx"][i])) for i in range(b, e)]


def duration(s, j):
    return s[j + 1][0] - s[j][0] if j + 1 < len(s) else 0


def iteration_of(s, j, m):
    """-1 for the prologue, else the number of marker-run starts at or before j, minus one."""
    starts = 0
    for q in range(j + 1):
        if s[q][1] == m and (q == 0 or s[q - 1][1] != m):
            starts += 1
    return starts - 1


def n_iter(s, m):
    return iteration_of(s, len(s) - 1, m) + 1 if s else 0


def tensor(tr):
    """rows[r] = list over it = -1..n_iter-1 of [(ctx, time, cnt)] ctx-ascending."""
    C = len(tr["parent"])
    m = tr["marker"]
    out = []
    for r in range(len(tr["rank_off"]) - 1):
        s = samples(tr, r)
        its = [iteration_of(s, j, m) for j in range(len(s))]
        rows = []
        for it in range(-1, n_iter(s, m)):
            row = []
            for c in range(C):
                sel = [j for j in range(len(s)) if its[j] == it and s[j][1] == c]
                if sel:
                    row.append((c, sum(duration(s, j) for j in sel), len(sel)))
            rows.append(row)
        out.append(rows)
    return out


def ancestors(parent, v):
    a = [v]
    while parent[a[-1]] != NONE:
        a.append(int(parent[a[-1]]))
    return a


def exclusive(tr):
    C = len(tr["parent"])
    out = []
    for r in range(len(tr["rank_off"]) - 1):
        s = samples(tr, r)
        row = []
        for c in range(C):
            sel = [j for j in range(len(s)) if s[j][1] == c]
            if sel:
                row.append((c, sum(duration(s, j) for j in sel), len(sel)))
        out.append(row)
    return out


def inclusive(tr):
    C = len(tr["parent"])
    parent = tr["parent"]
    out = []
    for r in range(len(tr["rank_off"]) - 1):
        s = samples(tr, r)
        row = []
        for a in range(C):
            sel = [j for j in range(len(s)) if a in ancestors(parent, s[j][1])]
            if sel:
                row.append((a, sum(duration(s, j) for j in sel), len(sel)))
        out.append(row)
    return out


def value(rows, r, c):
    for cc, t, n in rows[r]:
        if cc == c:
            return t, n
    return 0, 0


def stats(per_rank, ranks, c, tau=(3, 1)):
    """Exact statistics of context c over ranks (absent ranks count as 0)."""
    xs = [value(per_rank, r, c) for r in ranks]
    n = len(xs)
    vals = [x for x, _ in xs]
    present = sum(1 for _, k in xs if k > 0)
    S1 = sum(vals)
    S2 = sum(v * v for v in vals)
    M = n * S2 - S1 * S1
    mx = max(vals)
    argmax = ranks[vals.index(mx)]
    mean = Fraction(S1, n)
    var = Fraction(M, n * (n - 1)) if n >= 2 else Fraction(0)
    std = math.sqrt(var)  # correctly rounded sqrt of a double of var
    outliers = []
    for r, (x, k) in zip(ranks, xs):
        if k == 0:
            continue
        D = n * x - S1
        if D > 0 and M > 0 and n >= 2:
            if D * D * (n - 1) * tau[1] ** 2 > tau[0] ** 2 * n * M:
                outliers.append(r)
    return dict(n=n, present=present, min=min(vals) if present == n else 0, max=mx,
                argmax=argmax, s1=S1, s2=S2, M=M, mean=mean, var=var, std=std,
                outliers=outliers)
