"""Pins of the oracle's calling-context-tree pruning on the summary profile.

A hand-worked example fixes the summary profile, the threshold rule on both
sides of an exact boundary and the restriction of every rank's profiles; on
generated inputs the kept set must be closed under ancestors (a context's
inclusive time is at least any descendant's) and the root must carry the
total (the sum of the ranks' spans)."""
import numpy as np

import oracle
from paper_2605_03561_b300.synth import edge

NONE = 0xFFFFFFFF


def _hand():
    # Tree: 0 root, 1 child of 0, 2 child of 1, 3 child of 0.  Marker 3.
    # Rank 0 samples (ts, ctx): (0,0) (10,1) (30,2) (35,3) (100,3)
    #   exclusive: ctx0 10, ctx1 20, ctx2 5, ctx3 65 (the last sample lasts 0)
    #   inclusive: ctx0 100, ctx1 25, ctx2 5, ctx3 65
    # Rank 1 samples: (0,1) (50,2) (90,3) (100,3)
    #   exclusive: ctx1 50, ctx2 40, ctx3 10
    #   inclusive: ctx0 100, ctx1 90, ctx2 40, ctx3 10
    # Summary (inclusive summed over ranks): ctx0 200, ctx1 115, ctx2 45, ctx3 75.
    ts = np.array([0, 10, 30, 35, 100, 0, 50, 90, 100], np.uint64)
    ctx = np.array([0, 1, 2, 3, 3, 1, 2, 3, 3], np.uint32)
    rank_off = np.array([0, 5, 9], np.uint64)
    parent = np.array([NONE, 0, 1, 0], np.uint32)
    tr = oracle.Traces(rank_off, ts, ctx, parent, 3)
    return oracle.Analysis(tr)


def test_hand_summary_and_threshold():
    a = _hand()
    kept, summary, x, inc = a.prune(1, 4)  # keep >= 50 of 200
    assert summary.tolist() == [200, 115, 45, 75]
    assert kept.tolist() == [1, 1, 0, 1]
    assert x["off"].tolist() == [0, 3, 5]
    assert x["ctx"].tolist() == [0, 1, 3, 1, 3]
    assert x["time"].tolist() == [10, 20, 65, 50, 10]
    assert x["cnt"].tolist() == [1, 1, 2, 1, 2]
    assert inc["off"].tolist() == [0, 3, 6]
    assert inc["ctx"].tolist() == [0, 1, 3, 0, 1, 3]
    assert inc["time"].tolist() == [100, 25, 65, 100, 90, 10]


def test_hand_boundaries_and_name_drops():
    a = _hand()
    assert a.prune(45, 200)[0].tolist() == [1, 1, 1, 1]  # 45 * 200 >= 200 * 45: kept
    assert a.prune(46, 200)[0].tolist() == [1, 1, 0, 1]
    assert a.prune(0, 1)[0].tolist() == [1, 1, 1, 1]
    assert a.prune(2, 1)[0].tolist() == [0, 0, 0, 0]  # above the total: nothing
    drop = np.array([0, 0, 0, 1], np.uint8)
    kept, _, x, inc = a.prune(0, 1, drop=drop)
    assert kept.tolist() == [1, 1, 1, 0]
    assert 3 not in x["ctx"].tolist() and 3 not in inc["ctx"].tolist()
    assert x["off"].tolist() == [0, 3, 5]


def test_kept_set_closed_under_ancestors_and_root_total():
    for seed in range(4):
        d = edge.case("random_medium", seed)
        tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        a = oracle.Analysis(tr)
        root = int(np.flatnonzero(d["parent"] == NONE)[0])
        for num, den in ((1, 100), (1, 20), (1, 3)):
            kept, summary, _, _ = a.prune(num, den)
            assert int(summary[root]) == int(a.span().astype(object).sum())
            for c in np.flatnonzero(kept):
                p = int(d["parent"][c])
                if p != NONE:
                    assert kept[p] == 1, (seed, num, den, c)
