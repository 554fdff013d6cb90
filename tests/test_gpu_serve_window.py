"""Parity of the serving form's fifth query kind, TA_Q_WINDOW (the time of a
context in a time window on every rank of a range), with the oracle's
time-window profiles, and byte equality of its results alone and mixed with
the other kinds in continuous batches."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import context

pytestmark = pytest.mark.gpu

BIG = (1 << 64) - 1


@pytest.fixture(scope="module")
def served():
    ctx = context()
    items = []
    sets = [synth.generate(synth.preset(2, seed=8, n_ranks=80, len_mean=4000.0)),
            edge.case("random_medium", 4), edge.case("many_iterations", 1),
            edge.case("many_empty_then_long", 2)]
    for d in sets:
        tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        e = ctx.load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"], keep_traces=True)
        items.append(dict(d=d, tr=tr, e=e))
    return items


def _window_queries(items, n, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for _ in range(n):
        x = int(rng.integers(0, len(items)))
        d, R = items[x]["d"], items[x]["tr"].R
        ts = d["ts"]
        present = np.unique(d["ctx"]) if len(d["ctx"]) else np.array([0])
        c = int(rng.choice(present))
        hi = int(ts.max()) + 2 if len(ts) else 2
        u = rng.random()
        if u < 0.1:
            t0, t1 = 0, BIG
        elif u < 0.5 and len(ts):
            t0, t1 = sorted(int(ts[i]) for i in rng.integers(0, len(ts), size=2))
        else:
            t0, t1 = sorted(int(v) for v in rng.integers(0, hi, size=2))
        r0 = int(rng.integers(0, R))
        r1 = int(rng.integers(r0, R + 1))
        qs.append(ta.make_query(ta.Q_WINDOW, x, c, r0=r0, r1=r1, t0=t0, t1=t1))
    return qs


def _oracle_window(items, q):
    tr = items[q.experiment]["tr"]
    a = oracle.Analysis(tr, q.r0, q.r1, rows=False, incl=False)
    w = a.interval(q.t0, q.t1)
    n = q.r1 - q.r0
    t, c = np.zeros(n, np.uint64), np.zeros(n, np.uint64)
    for r in range(n):
        for j in range(int(w["off"][r]), int(w["off"][r + 1])):
            if int(w["ctx"][j]) == q.ctx:
                t[r], c[r] = w["time"][j], w["cnt"][j]
    return t, c


def _server(items, **kw):
    s = ta.Server(context(), result_bytes=64 << 20, **kw)
    for k, it in enumerate(items):
        assert s.add(it["e"], None) == k
    return s


def test_window_queries_match_oracle(served):
    s = _server(served)
    for q in _window_queries(served, 50, 1):
        got = s.query(q)
        t, c = _oracle_window(served, q)
        assert np.array_equal(got["time"], t), (q.experiment, q.ctx, q.t0, q.t1, q.r0, q.r1)
        assert np.array_equal(got["cnt"], c)
    s.close()


def test_window_alone_equals_mix(served):
    rng = np.random.default_rng(5)
    qs = _window_queries(served, 120, 2)
    for _ in range(60):  # other kinds in the same batches
        x = int(rng.integers(0, len(served)))
        R = served[x]["tr"].R
        c = int(rng.choice(np.unique(served[x]["d"]["ctx"])))
        qs.append(ta.make_query(ta.Q_SLICE, x, c, r0=0, r1=R, i0=0, i1=8) if rng.random() < 0.5
                  else ta.make_query(ta.Q_TOPK, x, c, k=10))
    rng.shuffle(qs)
    plain = _server(served, max_batch=1, n_streams=1)
    alone = []
    for q in qs:
        t = plain.submit(q)
        res = ta.QueryResult()
        assert ta.lib().ta_serve_poll(plain.h, t, -1, res) == ta.OK
        alone.append(ctypes.string_at(res.data, res.bytes))
        plain.release(t)
    plain.close()
    mix = _server(served, max_batch=64, n_streams=3)
    tickets = [mix.submit(q) for q in qs]
    for q, t, ref in zip(qs, tickets, alone):
        res = ta.QueryResult()
        assert ta.lib().ta_serve_poll(mix.h, t, -1, res) == ta.OK
        assert ctypes.string_at(res.data, res.bytes) == ref, (q.kind, q.experiment)
        mix.release(t)
    mix.close()


def test_window_query_needs_kept_traces(served):
    d = edge.case("random_small", 3)
    e = context().load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    s = ta.Server(context(), result_bytes=1 << 20)
    s.add(e, None)
    with pytest.raises(ta.TaError) as ei:
        s.submit(ta.make_query(ta.Q_WINDOW, 0, 0, r0=0, r1=1, t0=0, t1=10))
    assert ei.value.status == ta.INVALID_ARG
    s.close()
    s = _server(served)
    with pytest.raises(ta.TaError) as ei:
        s.submit(ta.make_query(ta.Q_WINDOW, 0, 0, r0=5, r1=2, t0=0, t1=10))
    assert ei.value.status == ta.INVALID_ARG
    s.close()
