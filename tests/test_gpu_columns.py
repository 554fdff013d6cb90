"""Parity of the column operations (ta_events_table, ta_col_*) with the
oracle and with their plain definitions, bit for bit, on generated events
and adversarial columns (ties, all-equal keys, 64-bit keys, empty inputs),
and their error paths."""
import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _cols():
    return ta.Columns(context())


def _np(t):
    return t.cpu().numpy()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _load(d):
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    e = context().load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"],
                       keep_traces=True)
    return tr, e


@pytest.mark.parametrize("name", ["random_medium", "many_empty_then_long", "all_empty",
                                  "single_record"])
def test_events_table_and_group_by(name):
    d = edge.case(name, 2)
    tr, e = _load(d)
    cols = _cols()
    for r0, r1 in ((0, tr.R), (tr.R // 3, tr.R), (0, 0)):
        t = cols.events(e, r0, r1)
        o = oracle.events_table(tr, r0, r1)
        for k in ("rank", "ts", "ctx", "dur"):
            assert np.array_equal(_np(t[k]), o[k]), (name, r0, r1, k)
    t = cols.events(e)
    g = cols.group(_dev(d["rank_off"]), t["ctx"], len(d["parent"]), t["dur"])
    o = oracle.col_group(d["rank_off"], _np(t["ctx"]), _np(t["dur"]))
    for k in ("off", "key", "sum", "cnt"):
        assert np.array_equal(_np(g[k]), o[k]), k


def test_group_many_keys_per_segment():
    # 60,000 keys (global bitmaps) and segments with thousands of keys (the
    # global stage)
    rng = np.random.default_rng(5)
    seg = np.concatenate([[0], np.cumsum(rng.integers(0, 6000, size=40))]).astype(np.uint64)
    n = int(seg[-1])
    key = rng.integers(0, 60000, size=n).astype(np.uint32)
    val = rng.integers(0, 2**40, size=n).astype(np.uint64)
    g = _cols().group(_dev(seg), _dev(key), 60000, _dev(val))
    o = oracle.col_group(seg, key, val)
    for k in ("off", "key", "sum", "cnt"):
        assert np.array_equal(_np(g[k]), o[k]), k


@pytest.mark.parametrize("case", ["ties", "all_zero", "all_equal", "wide", "sorted", "reverse",
                                  "tile_edges"])
def test_sort(case):
    rng = np.random.default_rng(sum(map(ord, case)))
    n = {"tile_edges": 4096 * 3 + 17}.get(case, 50_000)
    if case == "ties":
        keys = rng.integers(0, 40, size=n)
    elif case == "all_zero":
        keys = np.zeros(n, np.int64)
    elif case == "all_equal":
        keys = np.full(n, 12345)
    elif case == "wide":
        keys = rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64, endpoint=True)
    elif case == "sorted":
        keys = np.arange(n) * 3
    elif case == "reverse":
        keys = (n - np.arange(n)) * 1000
    else:
        keys = rng.integers(0, 2**20, size=n)
    keys = keys.astype(np.uint64)
    ks, perm = _cols().sort(_dev(keys))
    ok, op = oracle.col_sort(keys)
    assert np.array_equal(_np(perm), op) and np.array_equal(_np(ks), ok)


def test_sort_generated_durations_and_small_sizes():
    g = synth.generate(synth.preset(2, seed=2, n_ranks=64, len_mean=20000.0))
    tr, e = _load(g)
    dur = _cols().events(e)["dur"]
    ks, perm = _cols().sort(dur)
    ok, op = oracle.col_sort(_np(dur))
    assert np.array_equal(_np(perm), op) and np.array_equal(_np(ks), ok)
    for n in (0, 1, 2, 31, 33, 4095, 4097):
        keys = np.random.default_rng(n).integers(0, 1000, size=n).astype(np.uint64)
        ks, perm = _cols().sort(_dev(keys))
        assert np.array_equal(_np(perm), oracle.col_sort(keys)[1])


def test_filter_gather_and_elementwise():
    rng = np.random.default_rng(9)
    n = 100_003
    a = rng.integers(0, 1000, size=n).astype(np.uint64)
    b = rng.integers(0, 2**62, size=n).astype(np.uint64)
    cols = _cols()
    da, db = _dev(a), _dev(b)
    for lo, hi in ((100, 200), (0, 0), (999, 5000), (2000, 3000), (0, 2**64 - 1)):
        assert np.array_equal(_np(cols.filter(da, lo, hi)), oracle.col_filter(a, lo, hi))
    dim = rng.integers(0, 2**32, size=777).astype(np.uint32)
    key = rng.integers(0, 777, size=n).astype(np.uint32)
    assert np.array_equal(_np(cols.gather(_dev(key), _dev(dim))), oracle.col_gather(key, dim))
    assert np.array_equal(_np(cols.compare(da, 500)), (a > 500).astype(np.uint8))
    assert np.array_equal(_np(cols.add(da, db)), a + b)
    assert np.array_equal(_np(cols.cumsum(db)), np.cumsum(b, dtype=np.uint64))
    assert cols.sum(db) == int(b.astype(object).sum()) % 2**64
    sc = _dev(b)
    cols.scale(sc, 3)
    assert np.array_equal(_np(sc), b * np.uint64(3))


def test_column_errors():
    cols = _cols()
    with pytest.raises(ta.TaError) as ei:
        cols.gather(_dev(np.array([0, 5], np.uint32)), _dev(np.array([1, 2], np.uint32)))
    assert ei.value.status == ta.INVALID_ARG
    with pytest.raises(ta.TaError) as ei:  # segment offsets must end at n
        cols.group(_dev(np.array([0, 2], np.uint64)), _dev(np.zeros(3, np.uint32)), 4,
                   _dev(np.zeros(3, np.uint64)))
    assert ei.value.status == ta.INVALID_ARG
    with pytest.raises(ta.TaError) as ei:  # a key >= n_keys
        cols.group(_dev(np.array([0, 3], np.uint64)), _dev(np.array([0, 4, 1], np.uint32)), 4,
                   _dev(np.zeros(3, np.uint64)))
    assert ei.value.status == ta.INVALID_ARG
    d = edge.case("random_small", 1)
    e = context().load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    with pytest.raises(ta.TaError) as ei:
        cols.events(e)
    assert ei.value.status == ta.STATE
