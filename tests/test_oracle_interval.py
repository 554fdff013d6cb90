"""Pins of the oracle's time-window profiles and call chains.

The whole time range gives back the exclusive and inclusive profiles;
adjacent windows add up exactly, time and sample counts alike; a hand-worked
window clips a sample at both ends; a call chain walks to the root."""
import numpy as np

import oracle
from paper_2605_03561_b300.synth import edge

NONE = 0xFFFFFFFF
BIG = (1 << 64) - 1


def _hand():
    # Tree: 0 root, 1 child of 0, 2 child of 1, 3 child of 0.
    # Rank 0 samples (ts, ctx): (0,0) (10,1) (30,2) (35,3) (100,3)
    # Rank 1 samples: (0,1) (50,2) (90,3) (100,3)
    ts = np.array([0, 10, 30, 35, 100, 0, 50, 90, 100], np.uint64)
    ctx = np.array([0, 1, 2, 3, 3, 1, 2, 3, 3], np.uint32)
    tr = oracle.Traces(np.array([0, 5, 9], np.uint64), ts, ctx,
                       np.array([NONE, 0, 1, 0], np.uint32), 3)
    return oracle.Analysis(tr)


def _as_dicts(csr):
    out = []
    for r in range(len(csr["off"]) - 1):
        b, e = int(csr["off"][r]), int(csr["off"][r + 1])
        out.append({int(c): (int(t), int(n)) for c, t, n in
                    zip(csr["ctx"][b:e], csr["time"][b:e], csr["cnt"][b:e])})
    return out


def test_hand_window():
    a = _hand()
    # [20, 60): rank 0: ctx1 [10,30) clipped to 10 ns, 0 samples inside;
    # ctx2 [30,35) 5 ns, 1 sample; ctx3 [35,100) clipped to 25 ns, 1 sample.
    # rank 1: ctx1 [0,50) clipped to 30 ns, 0 samples; ctx2 [50,90) clipped
    # to 10 ns, 1 sample.
    w = _as_dicts(a.interval(20, 60))
    assert w[0] == {1: (10, 0), 2: (5, 1), 3: (25, 1)}
    assert w[1] == {1: (30, 0), 2: (10, 1)}
    wi = _as_dicts(a.interval(20, 60, incl=True))
    assert wi[0] == {0: (40, 2), 1: (15, 1), 2: (5, 1), 3: (25, 1)}
    assert wi[1] == {0: (40, 1), 1: (40, 1), 2: (10, 1)}
    # the last sample of a rank lasts 0 ns but counts in the window holding it
    assert _as_dicts(a.interval(100, 101))[0] == {3: (0, 1)}


def test_whole_range_and_additivity():
    for seed in range(4):
        d = edge.case("random_medium", seed)
        tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        a = oracle.Analysis(tr)
        for incl, metric in ((False, oracle.EXCL), (True, oracle.INCL)):
            full = a.interval(0, BIG, incl=incl)
            ref = a.csr(metric)
            for k in ("off", "ctx", "time", "cnt"):
                assert np.array_equal(full[k], ref[k]), (seed, incl, k)
        rng = np.random.default_rng(seed)
        hi = int(d["ts"].max()) + 1 if len(d["ts"]) else 1
        t0, tm, t1 = sorted(int(x) for x in rng.integers(0, hi, size=3))
        left, right = _as_dicts(a.interval(t0, tm)), _as_dicts(a.interval(tm, t1))
        whole = _as_dicts(a.interval(t0, t1))
        for r in range(tr.R):
            keys = set(left[r]) | set(right[r])
            summed = {c: (left[r].get(c, (0, 0))[0] + right[r].get(c, (0, 0))[0],
                          left[r].get(c, (0, 0))[1] + right[r].get(c, (0, 0))[1]) for c in keys}
            assert summed == whole[r], (seed, r)


def test_call_chain():
    a = _hand()
    assert a.call_chain(2).tolist() == [2, 1, 0]
    assert a.call_chain(0).tolist() == [0]
