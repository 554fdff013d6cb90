"""Parity of ta_prune_profiles (pruning on the summary profile) with the
oracle: kept set, summary profile and every rank's pruned exclusive and
inclusive CSR, bit for bit; and its error paths."""
import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import context, load_both

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF


def _check(a, e, keep, drop=None):
    ok, osum, ox, oi = a.prune(keep[0], keep[1], drop=drop)
    got = e.prune(keep=keep, drop=drop)
    assert np.array_equal(got["kept"], ok)
    assert np.array_equal(got["summary"], osum)
    assert got["n_kept"] == int(ok.sum())
    for name, metric, o in (("exclusive", ta.EXCLUSIVE, ox), ("inclusive", ta.INCLUSIVE, oi)):
        g = e.csr(metric)
        for k in ("off", "ctx", "time", "cnt"):
            assert np.array_equal(g[k], o[k]), (name, k)
    assert got["excl_nnz"] == len(ox["ctx"]) and got["incl_nnz"] == len(oi["ctx"])


def test_hand_example():
    ts = np.array([0, 10, 30, 35, 100, 0, 50, 90, 100], np.uint64)
    cx = np.array([0, 1, 2, 3, 3, 1, 2, 3, 3], np.uint32)
    d = dict(rank_off=np.array([0, 5, 9], np.uint64), ts=ts, ctx=cx,
             parent=np.array([NONE, 0, 1, 0], np.uint32), marker=3)
    tr, a, e = load_both(d)
    _check(a, e, (1, 4))


@pytest.mark.parametrize("seed", range(3))
def test_random_thresholds_and_drops(seed):
    d = edge.case("random_medium", seed)
    rng = np.random.default_rng(seed)
    for keep in ((1, 100), (1, 20), (0, 1)):
        tr, a, e = load_both(d)
        drop = None
        if keep == (1, 20):
            drop = (rng.random(len(d["parent"])) < 0.05).astype(np.uint8)
        _check(a, e, keep, drop)
        e.free()


def test_generated_profile_twice():
    # The paper's 1 % rule on a generated profile, then pruning the pruned
    # profiles again (the kept set can only stay or shrink).
    g = synth.generate(synth.preset(2, seed=7, n_ranks=300, len_mean=5000.0))
    tr, a, e = load_both(g)
    _check(a, e, (1, 100))
    first = e.csr(ta.INCLUSIVE)
    again = e.prune(keep=(1, 100))
    assert again["incl_nnz"] == len(first["ctx"])


def test_prune_errors():
    d = edge.case("random_small", 3)
    ctx = context()
    e = ctx.load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    with pytest.raises(ta.TaError) as ei:
        e.prune(keep=(1, 0))
    assert ei.value.status == ta.INVALID_ARG
    s = ta.Server(ctx, result_bytes=1 << 20)
    s.add(e, None)
    with pytest.raises(ta.TaError) as ei:
        e.prune(keep=(1, 100))
    assert ei.value.status == ta.STATE
    s.close()
    e.prune(keep=(1, 100))  # allowed again once the server is closed
    e2 = ctx.load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"], inclusive=False)
    with pytest.raises(ta.TaError) as ei:
        e2.prune(keep=(1, 100))
    assert ei.value.status == ta.STATE
