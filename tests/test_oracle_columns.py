"""Pins of the oracle's column operations (the DataFrame operation classes of
Section IV): the events table against the spans and the pinned exclusive
profile, a group-by on (rank, ctx) that must equal that profile, a stable
sort against brute force and its invariants, filtering and the join by hand."""
import numpy as np

import oracle
from paper_2605_03561_b300.synth import edge

NONE = 0xFFFFFFFF


def _hand():
    ts = np.array([0, 10, 30, 35, 100, 0, 50, 90, 100], np.uint64)
    ctx = np.array([0, 1, 2, 3, 3, 1, 2, 3, 3], np.uint32)
    return oracle.Traces(np.array([0, 5, 9], np.uint64), ts, ctx,
                         np.array([NONE, 0, 1, 0], np.uint32), 3)


def test_events_table_hand_and_spans():
    t = oracle.events_table(_hand(), 0, 2)
    assert t["rank"].tolist() == [0, 0, 0, 0, 0, 1, 1, 1, 1]
    assert t["dur"].tolist() == [10, 20, 5, 65, 0, 50, 40, 10, 0]
    assert oracle.events_table(_hand(), 1, 2)["ts"].tolist() == [0, 50, 90, 100]
    d = edge.case("random_medium", 1)
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    t = oracle.events_table(tr, 0, tr.R)
    per_rank = np.zeros(tr.R, object)
    for r, v in zip(t["rank"].tolist(), t["dur"].tolist()):
        per_rank[r] += v
    assert per_rank.tolist() == oracle.Analysis(tr, rows=False).span().tolist()


def test_group_by_rank_and_ctx_is_the_exclusive_profile():
    for seed in range(3):
        d = edge.case("random_medium", seed)
        tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        t = oracle.events_table(tr, 0, tr.R)
        g = oracle.col_group(d["rank_off"], t["ctx"], t["dur"])
        x = oracle.Analysis(tr, rows=False).csr(oracle.EXCL)
        assert np.array_equal(g["off"], x["off"]) and np.array_equal(g["key"], x["ctx"])
        assert np.array_equal(g["sum"], x["time"]) and np.array_equal(g["cnt"], x["cnt"])


def test_sort_is_stable_and_a_permutation():
    rng = np.random.default_rng(4)
    for n in (0, 1, 7, 300):
        keys = rng.integers(0, 9, size=n).astype(np.uint64)
        ks, perm = oracle.col_sort(keys)
        brute = sorted(range(n), key=lambda i: (int(keys[i]), i))
        assert perm.tolist() == brute
        assert np.array_equal(ks, keys[perm]) and np.all(np.diff(ks.astype(np.int64)) >= 0)
    big = np.array([2**63 + 5, 3, 2**40, 3, 0], np.uint64)
    assert oracle.col_sort(big)[1].tolist() == [4, 1, 3, 2, 0]


def test_filter_and_gather_by_hand():
    col = np.array([5, 0, 9, 5, 12, 7], np.uint64)
    assert oracle.col_filter(col, 5, 9).tolist() == [0, 2, 3, 5]
    assert oracle.col_filter(col, 13, 20).tolist() == []
    dim = np.array([10, 11, 12], np.uint32)
    assert oracle.col_gather(np.array([2, 0, 0, 1], np.uint32), dim).tolist() == [12, 10, 10, 11]
