"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Small and medium cases compare every output element by element; they span
many 4096-sample tiles with ragged tails, rows that cross tiles, empty and
degenerate ranks, and contexts far apart in the tree."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import (check_products, check_speedup, check_stats, check_topology,
                         load_both, simple_topology)

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF


def _hand(golden_dir):
    with open(os.path.join(golden_dir, "hand_example.json")) as f:
        g = json.load(f)
    lens = [len(r["ts"]) for r in g["ranks"]]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    return dict(rank_off=ro, ts=np.array(sum((r["ts"] for r in g["ranks"]), []), np.uint64),
                ctx=np.array(sum((r["ctx"] for r in g["ranks"]), []), np.uint32),
                parent=np.array(g["parent"], np.uint32), marker=g["marker"]), g


def test_hand_example(golden_dir):
    d, g = _hand(golden_dir)
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    st, _ = check_stats(a, e, ta.EXCLUSIVE, ctxs=[2])
    assert st["std"][0] == pytest.approx(g["stats_excl_ctx2"]["std"], rel=1e-15)
    check_stats(a, e, ta.INCLUSIVE)
    gp, gt = check_speedup(a, e, [1, 2])
    assert gt["speedup_fraction"] == pytest.approx(g["speedup_ctx_1_2"]["speedup_fraction"],
                                                   rel=1e-15)


@pytest.mark.parametrize("name", edge.EDGE_CASES)
def test_edge_cases(name):
    d = edge.case(name, 1)
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    check_stats(a, e, ta.EXCLUSIVE, tau=(1, 1))
    check_stats(a, e, ta.INCLUSIVE, tau=(2, 1))
    ctxs = sorted(set(int(c) for c in d["ctx"][:50]))
    if ctxs:
        check_speedup(a, e, ctxs)


@pytest.mark.parametrize("seed", range(2))
def test_large_context_count(seed):
    # 60,000 contexts: the per-warp bitmaps of the tensor and rank passes are
    # in global memory; two loads in a row check they are left clean
    d = edge.case("large_ctx", seed)
    for _ in range(2):
        tr, a, e = load_both(d)
        check_products(tr, a, e)
    check_stats(a, e, ta.EXCLUSIVE, tau=(2, 1))


def test_inclusive_paths_shallow_and_very_deep():
    # A 30,000-node chain: the ancestor lists of all contexts would exceed the
    # bound, so the inclusive rollup takes the level-by-level sweep; the other
    # cases here take the ancestor lists.
    rng = np.random.default_rng(8)
    C = 30000
    parent = np.arange(-1, C - 1, dtype=np.int64).astype(np.uint32)
    parent[0] = NONE
    ctx = np.concatenate([rng.integers(C - 200, C, size=60), rng.integers(0, C, size=40)])
    ctx[0] = 5
    ctx[60] = 5
    ts = np.concatenate([np.cumsum(rng.integers(1, 9, size=60)),
                         np.cumsum(rng.integers(1, 9, size=40))]).astype(np.uint64)
    d = dict(rank_off=np.array([0, 60, 100], np.uint64), ts=ts, ctx=ctx.astype(np.uint32),
             parent=parent, marker=5)
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    check_stats(a, e, ta.INCLUSIVE, tau=(1, 1))


def test_many_iterations_speedup_paths():
    # I* = 1200: twelve contexts take the multi-kernel path, three the fused one
    d = edge.case("many_iterations", 4)
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    check_speedup(a, e, list(range(12)))
    check_speedup(a, e, [2, 5, 7])


@pytest.mark.parametrize("seed", range(12))
def test_random_small(seed):
    d = edge.case("random_small", seed)
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    check_stats(a, e, ta.EXCLUSIVE, tau=(1, 1))
    check_stats(a, e, ta.INCLUSIVE, tau=(1, 2))
    check_speedup(a, e, list(range(tr.C)))
    topo = simple_topology(tr.R, 2, 2, 1)
    check_topology(a, e, int(d["ctx"][0]) if len(d["ctx"]) else 0, topo, tau=(1, 1))


@pytest.mark.parametrize("seed", range(6))
def test_random_medium(seed):
    d = edge.case("random_medium", seed)
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    rng = np.random.default_rng(seed)
    ranks = np.unique(rng.integers(0, tr.R, size=max(1, tr.R // 2))).astype(np.uint32)
    check_stats(a, e, ta.EXCLUSIVE, tau=(2, 1))
    check_stats(a, e, ta.INCLUSIVE, ranks=ranks, tau=(3, 2))
    ctxs = np.unique(d["ctx"][: 200]).astype(np.uint32)
    check_speedup(a, e, ctxs, ranks=ranks)


def test_capacity_retry_paths():
    """First-try capacities that are far too small are recovered exactly."""
    d = edge.case("random_medium", 3)
    tr, a, e = load_both(d, nnz_hint=7, rows_hint=3)
    check_products(tr, a, e)


def test_borrowed_device_input():
    import torch
    d = edge.case("random_medium", 4)
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    a = oracle.Analysis(tr)
    dev = {k: torch.from_numpy(np.ascontiguousarray(d[k])).cuda()
           for k in ("rank_off", "ts", "ctx", "parent")}
    from gpu_helpers import context
    e = context().load(dev["rank_off"], dev["ts"], dev["ctx"], dev["parent"], d["marker"],
                       borrow=True)
    check_products(tr, a, e)
    check_stats(a, e, ta.EXCLUSIVE)


def test_borrowed_unaligned_device_input_is_copied():
    # Views starting one element into their storage are not 16-byte aligned;
    # the library copies them instead of reading them in place.
    import torch
    d = edge.case("random_medium", 5)
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    a = oracle.Analysis(tr)
    n = len(d["ts"])
    ts = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    cx = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ts[1:] = torch.from_numpy(d["ts"].view(np.int64)).cuda()
    cx[1:] = torch.from_numpy(d["ctx"].view(np.int32)).cuda()
    ts, cx = ts.view(torch.uint64)[1:], cx.view(torch.uint32)[1:]
    assert ts.data_ptr() % 16 and cx.data_ptr() % 16
    from gpu_helpers import context
    e = context().load(torch.from_numpy(d["rank_off"]).cuda(), ts, cx,
                       torch.from_numpy(d["parent"]).cuda(), d["marker"], borrow=True)
    check_products(tr, a, e)


@pytest.mark.parametrize("preset,R", [(0, 8), (1, 64), (2, 96), (3, 1500)])
def test_generated_configs(preset, R):
    """The structured generator at reduced rank counts (full trace lengths)."""
    cfg = synth.preset(preset, seed=11, n_ranks=R)
    g = synth.generate(cfg)
    tr, a, e = load_both(g)
    check_products(tr, a, e)
    check_stats(a, e, ta.EXCLUSIVE)
    check_stats(a, e, ta.INCLUSIVE, tau=(2, 1))
    truth = synth.truth(cfg, g["info"])
    kset = np.unique(truth["segment_ctx"]).astype(np.uint32)
    check_speedup(a, e, kset)
    topo = synth.topology(cfg, g["info"])
    comm = truth["segment_ctx"][truth["comm_segment"].astype(bool)]
    check_topology(a, e, int(comm[0]), topo, tau=(2, 1))


def test_shuffled_segments_every_product():
    """Iterations that run their segments in a fresh random order: no row
    repeats its predecessor's run sequence, so the tensor write pass takes its
    direct path (contexts in the warp's union, each once per row) instead of
    the template path, for 300 ranks of the plain-at-scale generator."""
    cfg = synth.preset(3, seed=12, n_ranks=300, len_mean=8000.0, shuffle_segments=1)
    g = synth.generate(cfg)
    tr, a, e = load_both(g)
    check_products(tr, a, e)
    check_stats(a, e, ta.EXCLUSIVE)
    truth = synth.truth(cfg, g["info"])
    check_speedup(a, e, np.unique(truth["segment_ctx"]).astype(np.uint32))


def test_validation_errors():
    base = edge.case("random_small", 2)
    from gpu_helpers import context

    def load(d):
        try:
            context().load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
            return ta.OK
        except ta.TaError as err:
            return err.status

    def variant(kind):
        d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
        nz = [r for r in range(len(d["rank_off"]) - 1) if d["rank_off"][r + 1] - d["rank_off"][r] >= 2]
        b = int(d["rank_off"][nz[0]])
        if kind == "not_sorted":
            d["ts"][b + 1] = d["ts"][b] - 1 if d["ts"][b] > 0 else 0
            d["ts"][b] = d["ts"][b] + 5
        elif kind == "bad_ctx":
            d["ctx"][b] = len(d["parent"])
        elif kind == "two_roots":
            d["parent"] = d["parent"].copy()
            nonroot = np.nonzero(d["parent"] != NONE)[0]
            d["parent"][nonroot[0]] = NONE
        elif kind == "cycle":
            C = len(d["parent"])
            d["parent"] = np.array([NONE] + [(v % (C - 1)) + 1 for v in range(1, C)], np.uint32)
        elif kind == "rank_off":
            d["rank_off"][1] = d["rank_off"][-1] + 1
        elif kind == "marker":
            d["marker"] = len(d["parent"])
        return d

    for kind, code in [("not_sorted", ta.NOT_SORTED), ("bad_ctx", ta.BAD_CTX),
                       ("two_roots", ta.BAD_CCT), ("cycle", ta.BAD_CCT),
                       ("rank_off", ta.INVALID_ARG), ("marker", ta.INVALID_ARG)]:
        d = variant(kind)
        tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        if kind in ("not_sorted", "bad_ctx", "two_roots", "cycle", "rank_off"):
            assert oracle.validate(tr) == code, kind
        assert load(d) == code, kind
    # the context is still usable afterwards
    tr, a, e = load_both(base)
    check_products(tr, a, e)


def test_rows_repeating_contexts_across_runs():
    # Few contexts and long rows: a row returns to a context after others, so
    # it has more runs than distinct contexts and fills fewer entry slots than
    # the count pass sized (the compaction step), across many tiles.
    rng = np.random.default_rng(31)
    R, C, marker = 48, 20, 3
    rank_off, ts, ctx = edge.random_traces(rng, R, C, marker, 40000, p_empty=0.05, p_marker=0.004)
    d = dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=edge.shuffled_tree(rng, C, 5), marker=marker)
    tr, a, e = load_both(d)
    assert int(rank_off[-1]) > 50 * 4096
    check_products(tr, a, e)
    t = e.tensor()
    runs = int(np.sum(ctx[1:] != ctx[:-1])) + 1
    assert len(t["e_ctx"]) < runs  # rows do repeat contexts here


def test_exclusive_ranks_above_the_scratch_cap():
    # Ranks with more than 256 distinct contexts (written by the second,
    # restricted write pass) mixed with ranks below the cap (the scratch copy).
    rng = np.random.default_rng(32)
    R, C, marker = 40, 3000, 7
    lengths = np.where(np.arange(R) % 3 == 0, 6000, 150)
    rank_off, ts, ctx = edge.random_traces(rng, R, C, marker, 0, p_marker=0.002, lengths=lengths)
    d = dict(rank_off=rank_off, ts=ts, ctx=ctx, parent=edge.shuffled_tree(rng, C, 8), marker=marker)
    tr, a, e = load_both(d)
    x = e.csr(ta.EXCLUSIVE)
    per_rank = np.diff(x["off"].astype(np.int64))
    assert (per_rank > 256).any() and (per_rank <= 256).any()
    check_products(tr, a, e)


def test_large_outlier_sort():
    # Tens of thousands of outliers: the sort runs its shared-memory blocks of
    # 4096 pairs and the global steps between them; the list must equal the
    # oracle's, ordered by (context, rank).
    cfg = synth.preset(2, seed=33, n_ranks=2000, len_mean=3000.0)
    d = synth.generate(cfg)
    tr, a, e = load_both(d)
    gs, go, gn, _ = e.stats(ta.EXCLUSIVE, tau=(1, 2), outlier_cap=1 << 20)
    os_, oo, on, _ = a.stats(ta.EXCLUSIVE, tau=(1, 2), want_z=False)
    assert gn == on and on > 8192
    assert np.array_equal(go["ctx"], oo["ctx"]) and np.array_equal(go["rank"], oo["rank"])

