"""Seeded small and degenerate trace sets for parity and edge-case tests.

Draws inputs only (no analysis arithmetic).  Covers what the structured
generator in ``tagen.cpp`` never produces: empty ranks, traces that start with
the marker, consecutive marker runs, equal timestamps (zero durations),
interleaved contexts that revisit the same context inside an iteration, a
single rank, a one-node tree, very long rows and traces without any marker.
"""
from __future__ import annotations

import numpy as np

NONE = 0xFFFFFFFF


def random_tree(rng: np.random.Generator, C: int, max_depth: int = 6) -> np.ndarray:
    """parent[0] = root; parent[v] uniform over earlier nodes of depth < max_depth."""
    parent = np.zeros(C, np.uint32)
    parent[0] = NONE
    depth = np.zeros(C, np.int64)
    elig = [0]
    for v in range(1, C):
        p = elig[rng.integers(len(elig))] if elig else 0
        parent[v] = p
        depth[v] = depth[p] + 1
        if depth[v] < max_depth:
            elig.append(v)
    return parent


def shuffled_tree(rng: np.random.Generator, C: int, max_depth: int = 6) -> np.ndarray:
    """Same shape as random_tree but with node ids permuted (parents may be > child)."""
    base = random_tree(rng, C, max_depth)
    perm = rng.permutation(C)  # new id of old node
    parent = np.zeros(C, np.uint32)
    for old in range(C):
        p = base[old]
        parent[perm[old]] = NONE if p == NONE else perm[p]
    return parent


def random_traces(rng: np.random.Generator, R: int, C: int, marker: int, max_len: int,
                  p_empty: float = 0.15, p_marker: float = 0.2, p_tie: float = 0.2,
                  max_gap: int = 50, lengths=None):
    """Unstructured traces: ctx uniform, marker with probability p_marker
    (so marker runs of length > 1 appear), gaps uniform in [1, max_gap] or 0
    with probability p_tie."""
    if lengths is None:
        lengths = rng.integers(0, max_len + 1, size=R)
        lengths[rng.random(R) < p_empty] = 0
    lengths = np.asarray(lengths, np.int64)
    rank_off = np.zeros(R + 1, np.uint64)
    rank_off[1:] = np.cumsum(lengths)
    N = int(rank_off[-1])
    ctx = rng.integers(0, C, size=N).astype(np.uint32)
    ctx[rng.random(N) < p_marker] = marker
    gaps = rng.integers(1, max_gap + 1, size=N).astype(np.uint64)
    gaps[rng.random(N) < p_tie] = 0
    ts = np.zeros(N, np.uint64)
    for r in range(R):
        b, e = int(rank_off[r]), int(rank_off[r + 1])
        if e > b:
            t0 = np.uint64(rng.integers(0, 1000))
            g = gaps[b:e].copy()
            g[0] = 0
            ts[b:e] = t0 + np.cumsum(g)
    return rank_off, ts, ctx


def case(name: str, seed: int = 0):
    """Named edge cases: dict(rank_off, ts, ctx, parent, marker)."""
    rng = np.random.default_rng(seed)
    if name == "all_empty":
        C = 5
        R = 7
        return dict(rank_off=np.zeros(R + 1, np.uint64), ts=np.zeros(0, np.uint64),
                    ctx=np.zeros(0, np.uint32), parent=random_tree(rng, C), marker=1)
    if name == "single_record":
        return dict(rank_off=np.array([0, 1], np.uint64), ts=np.array([5], np.uint64),
                    ctx=np.array([0], np.uint32), parent=np.array([NONE], np.uint32), marker=0)
    if name == "root_only_tree":
        rank_off, ts, ctx = random_traces(rng, 3, 1, 0, 40, p_marker=0.3)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=np.array([NONE], np.uint32),
                    marker=0)
    if name == "no_marker":
        C = 30
        rank_off, ts, ctx = random_traces(rng, 4, C, 7, 3000, p_marker=0.0)
        ctx[ctx == 7] = 8
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=random_tree(rng, C), marker=7)
    if name == "all_marker":
        C = 6
        rank_off, ts, ctx = random_traces(rng, 5, C, 2, 100, p_marker=1.0)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=random_tree(rng, C), marker=2)
    if name == "long_row_many_ctx":
        # One iteration row with thousands of distinct contexts.
        C = 9000
        n = 20000
        ctx = rng.integers(2, C, size=n).astype(np.uint32)
        ctx[0] = 1
        ctx[n // 2] = 1
        ts = np.cumsum(rng.integers(0, 4, size=n)).astype(np.uint64)
        return dict(rank_off=np.array([0, n], np.uint64), ts=ts, ctx=ctx,
                    parent=random_tree(rng, C, 20), marker=1)
    if name == "shuffled_tree":
        C = 40
        parent = shuffled_tree(rng, C, 8)
        marker = int(rng.integers(0, C))
        rank_off, ts, ctx = random_traces(rng, 9, C, marker, 400)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=parent, marker=marker)
    if name == "many_empty_then_long":
        C = 50
        R = 3000
        lengths = np.zeros(R, np.int64)
        lengths[-3:] = [5000, 0, 7000]
        rank_off, ts, ctx = random_traces(rng, R, C, 3, 0, lengths=lengths)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=random_tree(rng, C), marker=3)
    if name == "deep_chain":
        C = 300
        parent = np.arange(-1, C - 1, dtype=np.int64).astype(np.uint32)
        parent[0] = NONE
        rank_off, ts, ctx = random_traces(rng, 6, C, 150, 800)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=parent, marker=150)
    if name == "many_iterations":
        # 1200 short iterations per rank: cells of every iteration for many
        # contexts exceed what one pass keeps on chip
        C = 12
        R = 3
        parts_ro, parts_ts, parts_cx = [0], [], []
        for r in range(R):
            body = []
            for _ in range(1200):
                body += [1] + list(rng.integers(2, C, size=int(rng.integers(1, 4))))
            n = len(body)
            parts_cx.append(np.array(body, np.uint32))
            parts_ts.append(np.cumsum(rng.integers(1, 50, size=n)).astype(np.uint64))
            parts_ro.append(parts_ro[-1] + n)
        return dict(rank_off=np.array(parts_ro, np.uint64), ts=np.concatenate(parts_ts),
                    ctx=np.concatenate(parts_cx), parent=random_tree(rng, C), marker=1)
    if name == "large_ctx":
        # enough contexts that per-warp bitmaps live in global memory
        C = 60000
        marker = int(rng.integers(0, C))
        rank_off, ts, ctx = random_traces(rng, 40, C, marker, 4000, p_marker=0.02)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=shuffled_tree(rng, C, 16),
                    marker=marker)
    if name == "random_small":
        C = int(rng.integers(2, 14))
        marker = int(rng.integers(0, C))
        R = int(rng.integers(1, 9))
        rank_off, ts, ctx = random_traces(rng, R, C, marker, 50)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=shuffled_tree(rng, C, 5),
                    marker=marker)
    if name == "random_medium":
        C = int(rng.integers(20, 3000))
        marker = int(rng.integers(0, C))
        R = int(rng.integers(1, 300))
        rank_off, ts, ctx = random_traces(rng, R, C, marker, 20000, p_marker=0.01)
        return dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=shuffled_tree(rng, C, 12),
                    marker=marker)
    raise KeyError(name)


EDGE_CASES = ["all_empty", "single_record", "root_only_tree", "no_marker", "all_marker",
              "long_row_many_ctx", "shuffled_tree", "many_empty_then_long", "deep_chain"]
