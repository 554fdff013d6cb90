"""The potential speedup's within-rank terms taken from the exclusive
entries' iteration moments (ranks whose iteration rows all hold the same
contexts and number exactly I*) against the oracle, on experiments that mix
such ranks with ranks that read their rows: extra iterations (n_iter > I*),
one iteration with a different context set, and the moments dropped by a
prune."""
import numpy as np
import pytest

from paper_2605_03561_b300 import synth
from gpu_helpers import check_products, check_speedup, load_both

pytestmark = pytest.mark.gpu


def _mixed(seed, n_ranks=64):
    """A generated experiment (10 iterations per rank) with every fifth rank
    given one more iteration (a copy of its last) and every seventh rank one
    iteration whose second context's samples move to the prologue context."""
    g = synth.generate(synth.preset(1, seed=seed, n_ranks=n_ranks))
    ro, ts, cx, m = g["rank_off"], g["ts"], g["ctx"], int(g["marker"])
    pro = int(g["info"].prologue_ctx)
    out_ts, out_cx, lens = [], [], []
    extended, changed = [], []
    for r in range(len(ro) - 1):
        t = ts[int(ro[r]):int(ro[r + 1])].copy()
        c = cx[int(ro[r]):int(ro[r + 1])].copy()
        starts = np.flatnonzero(c == m)
        if r % 5 == 1 and len(starts):
            s = int(starts[-1])
            gap = t[-1] - t[-2] if len(t) > 1 else 1
            t = np.concatenate([t, t[s:] - t[s] + t[-1] + gap])
            c = np.concatenate([c, c[s:]])
            extended.append(r)
        elif r % 7 == 3 and len(starts) > 4:
            a, b = int(starts[3]), int(starts[4])
            seg = [x for x in np.unique(c[a:b]) if x != m and x != pro]
            if seg:
                c[a:b][c[a:b] == seg[0]] = pro
                changed.append(r)
        out_ts.append(t)
        out_cx.append(c)
        lens.append(len(t))
    d = dict(rank_off=np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64),
             ts=np.concatenate(out_ts).astype(np.uint64),
             ctx=np.concatenate(out_cx).astype(np.uint32), parent=g["parent"], marker=m)
    return d, extended, changed


@pytest.mark.parametrize("seed", range(3))
def test_mixed_ranks_all_contexts(seed):
    d, extended, changed = _mixed(seed)
    assert extended and changed
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    ctxs = list(range(len(d["parent"])))  # two chunks of within-rank terms
    check_speedup(a, e, ctxs)  # I* = 10: the extended ranks read their rows
    # I* = 11 over the extended ranks: their moments hold all of their rows
    check_speedup(a, e, ctxs, ranks=np.array(extended, np.uint32))
    rest = np.array([r for r in range(tr.R) if r not in changed], np.uint32)
    check_speedup(a, e, ctxs[::3], ranks=rest)


def test_many_ranks_and_prune():
    d, _, _ = _mixed(11, n_ranks=900)
    tr, a, e = load_both(d)
    segs = sorted(set(int(x) for x in d["ctx"][: 4000]))
    check_speedup(a, e, segs)
    e.prune(keep=(1, 100))  # the moments follow the unpruned entries: dropped
    check_speedup(a, e, segs)


def test_speedup_argument_errors_then_valid():
    # Context sets are checked on the device and reported at the call's end
    # (the maps skip ids >= C meanwhile); rank subsets before any kernel.
    d, extended, _ = _mixed(5)
    tr, a, e = load_both(d)
    C = len(d["parent"])
    import paper_2605_03561_b300 as ta
    for bad in ([3, 2], [2, 2], [1, C], [C + 1000]):
        with pytest.raises(ta.TaError) as ei:
            e.speedup(bad)
        assert ei.value.status == ta.INVALID_ARG, bad
    with pytest.raises(ta.TaError) as ei:
        e.speedup([1, 2], ranks=np.array([5, 3], np.uint32))
    assert ei.value.status == ta.INVALID_ARG
    check_speedup(a, e, list(range(C)))
    check_speedup(a, e, [1, 2], ranks=np.array(extended, np.uint32))


def test_alternating_templates():
    # Odd ranks move one segment context's samples to the prologue context in
    # every iteration: they keep one context list across their iterations (so
    # both the moments and the cells' by-position reading apply), but a list
    # different from the even ranks', so a warp's template is rebuilt as it
    # goes from rank to rank.
    g = synth.generate(synth.preset(1, seed=13, n_ranks=200))
    ro, ts, cx, m = g["rank_off"], g["ts"], g["ctx"].copy(), int(g["marker"])
    pro = int(g["info"].prologue_ctx)
    for r in range(1, len(ro) - 1, 2):
        a, b = int(ro[r]), int(ro[r + 1])
        starts = np.flatnonzero(cx[a:b] == m)
        if not len(starts):
            continue
        it = cx[a + int(starts[0]):b]
        seg = [x for x in np.unique(it) if x != m and x != pro]
        if seg:
            it[it == seg[0]] = pro
    d = dict(rank_off=ro, ts=ts, ctx=cx, parent=g["parent"], marker=m)
    tr, a, e = load_both(d)
    check_products(tr, a, e)
    check_speedup(a, e, list(range(len(d["parent"]))))
    check_speedup(a, e, sorted(set(int(x) for x in cx[:3000])), ranks=np.arange(0, 200, 3, dtype=np.uint32))
