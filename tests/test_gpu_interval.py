"""Parity of ta_interval_profile (per-rank profiles of a time window) and
ta_call_chains (bottom-up calling contexts) with the oracle, bit for bit; the
window's closed-form totals; and the error paths."""
import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import context

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF
BIG = (1 << 64) - 1
KEYS = ("off", "ctx", "time", "cnt")


def _hand():
    ts = np.array([0, 10, 30, 35, 100, 0, 50, 90, 100], np.uint64)
    cx = np.array([0, 1, 2, 3, 3, 1, 2, 3, 3], np.uint32)
    return dict(rank_off=np.array([0, 5, 9], np.uint64), ts=ts, ctx=cx,
                parent=np.array([NONE, 0, 1, 0], np.uint32), marker=3)


def _load(d, **kw):
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    e = context().load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"],
                       keep_traces=True, **kw)
    return tr, e


def _check(tr, e, t0, t1, r0=0, r1=None):
    r1 = tr.R if r1 is None else r1
    a = oracle.Analysis(tr, r0, r1, rows=False, incl=False)
    for metric, incl in ((ta.EXCLUSIVE, False), (ta.INCLUSIVE, True)):
        got = e.interval(t0, t1, r0, r1, metric=metric)
        ref = a.interval(t0, t1, incl=incl)
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), (t0, t1, r0, r1, metric, k)


def _windows(d, rng, n):
    """Windows with edges on sample timestamps, between them, before the first
    and after the last sample, plus the empty and the whole range."""
    ts = d["ts"]
    hi = int(ts.max()) + 2 if len(ts) else 2
    out = [(0, BIG), (5, 5), (7, 3), (hi, hi + 10)]
    for _ in range(n):
        if len(ts) and rng.random() < 0.5:
            a, b = sorted(int(ts[i]) for i in rng.integers(0, len(ts), size=2))
        else:
            a, b = sorted(int(x) for x in rng.integers(0, hi, size=2))
        out.append((a, b + int(rng.integers(0, 2))))
    return out


def test_hand_example():
    d = _hand()
    tr, e = _load(d)
    for t0, t1 in ((20, 60), (100, 101), (0, BIG), (35, 35), (36, 99), (0, 1), (101, 200)):
        _check(tr, e, t0, t1)
        _check(tr, e, t0, t1, 1, 2)
    w = e.interval(20, 60)
    assert w["ctx"].tolist() == [1, 2, 3, 1, 2]
    assert w["time"].tolist() == [10, 5, 25, 30, 10]
    assert w["cnt"].tolist() == [0, 1, 1, 0, 1]


@pytest.mark.parametrize("name", edge.EDGE_CASES)
def test_edge_cases(name):
    d = edge.case(name, 1)
    tr, e = _load(d)
    rng = np.random.default_rng(3)
    for t0, t1 in _windows(d, rng, 4):
        _check(tr, e, t0, t1)


@pytest.mark.parametrize("seed", range(3))
def test_random_windows_and_rank_ranges(seed):
    d = edge.case("random_medium", seed)
    tr, e = _load(d)
    rng = np.random.default_rng(seed + 10)
    for t0, t1 in _windows(d, rng, 5):
        r0 = int(rng.integers(0, tr.R))
        r1 = int(rng.integers(r0, tr.R + 1))
        _check(tr, e, t0, t1, r0, r1)
    _check(tr, e, 0, BIG)


def _iteration_starts(d):
    """Timestamps of every iteration start (first sample of a marker run)."""
    ts, cx, ro = d["ts"], d["ctx"], d["rank_off"].astype(np.int64)
    first = np.zeros(len(cx), bool)
    first[ro[:-1][ro[1:] > ro[:-1]]] = True
    m = cx == d["marker"]
    prev = np.concatenate([[False], m[:-1]])
    return ts[m & (first | ~prev)]


@pytest.mark.parametrize("name", ["many_iterations", "random_medium", "all_marker"])
def test_windows_on_iteration_boundaries(name):
    # window edges exactly at iteration starts: whole iterations inside the
    # window come from the tensor, the edges from the samples
    d = edge.case(name, 2)
    tr, e = _load(d)
    starts = np.unique(_iteration_starts(d))
    rng = np.random.default_rng(7)
    if len(starts) < 2:
        pytest.skip("no iterations")
    for _ in range(6):
        a, b = sorted(int(x) for x in rng.choice(starts, size=2))
        for t0, t1 in ((a, b), (a, b + 1), (a + 1, b), (a, BIG), (0, b)):
            _check(tr, e, t0, t1)


def test_repeated_calls_reuse_and_replace_the_result():
    d = edge.case("random_medium", 5)
    tr, e = _load(d)
    ts = d["ts"]
    t0, t1 = int(ts.max()) // 5, int(ts.max()) // 2
    first = e.interval(t0, t1)
    again = e.interval(t0, t1)
    for k in KEYS:
        assert np.array_equal(first[k], again[k])
    _check(tr, e, t0 + 1, t1)  # other arguments: computed anew
    _check(tr, e, t0, t1)
    e.prune(keep=(1, 100))  # pruning the profiles does not touch the traces
    _check(tr, e, t0, t1)


def test_whole_range_equals_resident_profiles():
    g = synth.generate(synth.preset(2, seed=3, n_ranks=200, len_mean=6000.0))
    tr, e = _load(g)
    for metric in (ta.EXCLUSIVE, ta.INCLUSIVE):
        got = e.interval(0, BIG, metric=metric)
        ref = e.csr(metric)
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), (metric, k)


def test_many_contexts_global_stage_and_bitmaps():
    # C = 60,000: the per-warp bitmaps live in global memory, and windows
    # hold more distinct contexts than the shared-memory stage
    d = edge.case("large_ctx", 2)
    tr, e = _load(d)
    ts = d["ts"]
    lo, hi = int(ts.min()), int(ts.max())
    for t0, t1 in ((lo, hi + 1), (lo + (hi - lo) // 3, lo + 2 * (hi - lo) // 3), (0, BIG)):
        _check(tr, e, t0, t1)


def test_one_rank_over_the_shared_stage():
    # rank 3 of 8 visits 600 distinct contexts, the others 20 each: only
    # that rank's window needs the global stage (sized by the count pass)
    rng = np.random.default_rng(41)
    Cn = 700
    parent = np.full(Cn, 0, np.uint32)
    parent[0] = NONE
    ro, ts, cx = [0], [], []
    for r in range(8):
        k = 600 if r == 3 else 20
        seq = rng.permutation(np.arange(1, Cn))[:k].astype(np.uint32)
        seq = np.concatenate([seq, seq[: k // 2]])
        t = np.cumsum(rng.integers(1, 50, len(seq))).astype(np.uint64)
        ts.append(t)
        cx.append(seq)
        ro.append(ro[-1] + len(seq))
    d = dict(rank_off=np.array(ro, np.uint64), ts=np.concatenate(ts), ctx=np.concatenate(cx),
             parent=parent, marker=1)
    tr, e = _load(d)
    hi = int(d["ts"].max())
    for t0, t1 in ((0, BIG), (hi // 4, 3 * hi // 4), (5, hi // 2)):
        _check(tr, e, t0, t1)


def test_generated_windows_closed_form_totals():
    # every rank's window times add up to the overlap of the window with its
    # span; its counts to the samples whose ts lies in the window; adjacent
    # windows add up entry by entry
    g = synth.generate(synth.preset(2, seed=5, n_ranks=500, len_mean=4000.0))
    tr, e = _load(g)
    ts, ro = g["ts"], g["rank_off"].astype(np.int64)
    lo, hi = int(ts.min()), int(ts.max())
    t0, tm, t1 = lo + (hi - lo) // 5, lo + (hi - lo) // 2, lo + 4 * (hi - lo) // 5
    w = e.interval(t0, t1)
    wo = w["off"].astype(np.int64)
    for r in range(tr.R):
        b, q = int(ro[r]), int(ro[r + 1])
        got_t = int(w["time"][wo[r]:wo[r + 1]].astype(object).sum())
        got_n = int(w["cnt"][wo[r]:wo[r + 1]].astype(object).sum())
        if q == b:
            assert got_t == 0 and got_n == 0
            continue
        first, last = int(ts[b]), int(ts[q - 1])
        assert got_t == max(0, min(t1, last) - max(t0, first)), r
        x = ts[b:q]
        assert got_n == int(np.searchsorted(x, t1, "left") - np.searchsorted(x, t0, "left")), r
    left, right = e.interval(t0, tm), e.interval(tm, t1)
    for r in range(0, tr.R, 7):
        acc = {}
        for part in (left, right):
            for j in range(int(part["off"][r]), int(part["off"][r + 1])):
                v = acc.setdefault(int(part["ctx"][j]), [0, 0])
                v[0] += int(part["time"][j])
                v[1] += int(part["cnt"][j])
        whole = {int(w["ctx"][j]): [int(w["time"][j]), int(w["cnt"][j])]
                 for j in range(int(wo[r]), int(wo[r + 1]))}
        assert acc == whole, r


def test_borrowed_traces_need_no_keep_flag():
    torch = pytest.importorskip("torch")
    d = edge.case("random_medium", 4)
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    dev = {k: torch.from_numpy(np.ascontiguousarray(d[k])).cuda()
           for k in ("rank_off", "ts", "ctx", "parent")}
    e = context().load(dev["rank_off"], dev["ts"], dev["ctx"], dev["parent"], d["marker"],
                       borrow=True)
    _check(tr, e, int(d["ts"].max()) // 4, int(d["ts"].max()) // 2)


def test_interval_errors():
    d = edge.case("random_small", 3)
    ctx = context()
    e = ctx.load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    with pytest.raises(ta.TaError) as ei:
        e.interval(0, 10)  # traces released after loading
    assert ei.value.status == ta.STATE
    e2 = ctx.load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"], keep_traces=True)
    R = len(d["rank_off"]) - 1
    for r0, r1 in ((1, 0), (0, R + 1)):
        with pytest.raises(ta.TaError) as ei:
            e2.interval(0, 10, r0, r1)
        assert ei.value.status == ta.INVALID_ARG
    with pytest.raises(ta.TaError) as ei:
        e2.interval(0, 10, metric=7)
    assert ei.value.status == ta.INVALID_ARG
    empty = e2.interval(0, 10, 0, 0)
    assert empty["off"].tolist() == [0] and len(empty["ctx"]) == 0


@pytest.mark.parametrize("name", ["deep_chain", "shuffled_tree", "large_ctx"])
def test_call_chains(name):
    d = edge.case(name, 0)
    tr, e = _load(d)
    a = oracle.Analysis(tr, rows=False, incl=False)
    rng = np.random.default_rng(1)
    C = len(d["parent"])
    ctxs = np.concatenate([rng.integers(0, C, size=200), [0, C - 1, 0]]).astype(np.uint32)
    got = e.call_chains(ctxs)
    for c, g in zip(ctxs, got):
        assert g.tolist() == a.call_chain(int(c)).tolist(), int(c)
    assert e.call_chains(np.zeros(0, np.uint32)) == []
    with pytest.raises(ta.TaError) as ei:
        e.call_chains(np.array([0, C], np.uint32))
    assert ei.value.status == ta.INVALID_ARG
