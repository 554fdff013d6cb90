"""Parity of the serving form (ta_serve_*) with the oracle, and the
alone-versus-mix equality of every query result.

Four query kinds over resident experiments: statistics of one context over a
rank subset, a (rank, iteration) slice of one context, the top-k ranks of a
context with z, and the rack rollup of a context.  Results must equal the
oracle's (integers bit for bit, FP64 within 1e-12 relative) and be byte for
byte the same whether a query runs alone or packed with others into
continuous batches on several streams."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import FP_FIELDS, INT_FIELDS, close, context, simple_topology

pytestmark = pytest.mark.gpu


def _experiments():
    out = []
    for cfg in (synth.preset(1, seed=5, n_ranks=40),
                synth.preset(2, seed=6, n_ranks=300, len_mean=8000.0)):
        g = synth.generate(cfg)
        topo = synth.topology(cfg, g["info"])
        out.append((g, topo))
    d = edge.case("random_medium", 3)
    out.append((d, simple_topology(len(d["rank_off"]) - 1, 3, 4, 2)))
    return out


@pytest.fixture(scope="module")
def served():
    ctx = context()
    items = []
    for d, topo in _experiments():
        tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        a = oracle.Analysis(tr)
        e = ctx.load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        items.append(dict(d=d, topo=topo, tr=tr, a=a, e=e))
    return items


def _random_queries(items, n, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for _ in range(n):
        x = int(rng.integers(0, len(items)))
        it = items[x]
        R, Cn = it["tr"].R, it["tr"].C
        present = np.unique(it["d"]["ctx"]) if len(it["d"]["ctx"]) else np.array([0])
        c = int(rng.choice(present)) if rng.random() < 0.9 else int(rng.integers(0, Cn))
        kind = int(rng.choice([1, 1, 1, 1, 2, 2, 2, 3, 3, 4]))
        metric = int(rng.integers(0, 2))
        if kind == ta.Q_STATS:
            m = int(np.exp(rng.uniform(0, np.log(R)))) if R > 1 else 1
            ranks = np.sort(rng.choice(R, size=max(1, min(R, m)), replace=False)).astype(np.uint32)
            q = ta.make_query(kind, x, c, metric, ranks=ranks,
                              tau=(int(rng.integers(1, 4)), int(rng.integers(1, 3))))
        elif kind == ta.Q_SLICE:
            r0 = int(rng.integers(0, R))
            r1 = int(rng.integers(r0, R + 1))
            i0 = int(rng.integers(0, 60))
            i1 = int(rng.integers(i0, i0 + 70))
            q = ta.make_query(kind, x, c, r0=r0, r1=r1, i0=i0, i1=i1)
        elif kind == ta.Q_TOPK:
            q = ta.make_query(kind, x, c, metric, k=int(rng.choice([1, 10, 100, 1024])))
        else:
            q = ta.make_query(kind, x, c, metric, tau=(int(rng.integers(1, 4)), 1),
                              min_ranks=int(rng.integers(1, 3)))
        qs.append(q)
    return qs


def _oracle_answer(items, q):
    it = items[q.experiment]
    a = it["a"]
    if q.kind == ta.Q_STATS:
        ranks = q._ranks
        st, _, n_out, _ = a.stats(q.metric, ranks=ranks, ctxs=[q.ctx], tau=(q.tau_num, q.tau_den))
        d = {k: v[0] for k, v in st.items()}
        d["n_outliers"] = n_out
        return d
    if q.kind == ta.Q_SLICE:
        return a.slice(q.ctx, q.r0, q.r1, q.i0, q.i1).reshape(-1)
    if q.kind == ta.Q_TOPK:
        rk, x, z = a.topk(q.ctx, q.k, q.metric)
        return dict(rank=rk, x=x, z=z)
    t = it["topo"]
    o = a.topology(q.ctx, t["node_of_rank"], t["rack_of_node"], t["chassis_of_node"],
                   t["n_racks"], t["n_chassis"], metric=q.metric, tau=(q.tau_num, q.tau_den),
                   min_ranks=q.min_ranks)
    return {k: o[k] for k in ("rack_sum", "rack_flagged", "rack_nodes", "flagged_racks")}


def _check(q, got, want):
    if q.kind == ta.Q_STATS:
        for k in INT_FIELDS:
            assert int(got[k]) == int(want[k]), k
        for k in FP_FIELDS:
            close([got[k]], [want[k]], k)
        assert got["n_outliers"] == want["n_outliers"]
    elif q.kind == ta.Q_SLICE:
        assert np.array_equal(got, want)
    elif q.kind == ta.Q_TOPK:
        assert np.array_equal(got["rank"], want["rank"])
        assert np.array_equal(got["x"], want["x"])
        close(got["z"], want["z"], "z")
    else:
        for k in want:
            assert np.array_equal(got[k], want[k]), k


def _server(items, **kw):
    kw.setdefault("result_bytes", 64 << 20)
    s = ta.Server(context(), **kw)
    for k, it in enumerate(items):
        assert s.add(it["e"], it["topo"]) == k
    return s


def test_each_kind_matches_oracle(served):
    s = _server(served)
    for q in _random_queries(served, 120, 1):
        _check(q, s.query(q), _oracle_answer(served, q))
    s.close()


def test_alone_equals_mix(served):
    qs = _random_queries(served, 400, 2)
    plain = _server(served, max_batch=1, n_streams=1)
    alone = []
    for q in qs:  # one query per launch, one at a time
        t = plain.submit(q)
        res = ta.QueryResult()
        assert ta.lib().ta_serve_poll(plain.h, t, -1, res) == ta.OK
        alone.append(ctypes.string_at(res.data, res.bytes))
        plain.release(t)
    plain.close()
    mix = _server(served, max_batch=64, n_streams=3)
    tickets = [mix.submit(q) for q in qs]  # all in flight together
    for q, t, ref in zip(qs, tickets, alone):
        res = ta.QueryResult()
        assert ta.lib().ta_serve_poll(mix.h, t, -1, res) == ta.OK
        got = ctypes.string_at(res.data, res.bytes)
        assert got == ref, (q.kind, q.experiment, q.ctx)
        assert res.t_submit_ns <= res.t_admit_ns <= res.t_launch_ns <= res.t_done_ns
        mix.release(t)
    mix.close()
    for q, ref in list(zip(qs, alone))[::7]:
        _check(q, ta.parse_payload(q.kind, ref, len(ref)), _oracle_answer(served, q))


def test_admission_by_memory_with_tiny_arenas(served):
    # Results of the whole stream do not fit the result arena at once: queries
    # wait until earlier results are released, and all complete correctly.
    qs = [ta.make_query(ta.Q_SLICE, 1, int(served[1]["d"]["ctx"][k * 101]), r0=0, r1=300, i0=0,
                        i1=51) for k in range(40)]
    s = _server(served, result_bytes=300 * 51 * 8 * 3, scratch_bytes=1 << 20, max_batch=8,
                n_streams=2)
    lat, wall = s.replay(qs, np.arange(len(qs), dtype=np.uint64) * 1000)
    assert len(lat) == len(qs) and wall > 0
    for q in qs[:5]:
        _check(q, s.query(q), _oracle_answer(served, q))
    big = ta.make_query(ta.Q_SLICE, 1, 1, r0=0, r1=300, i0=0, i1=1000)
    with pytest.raises(ta.TaError) as ei:
        s.submit(big)
    assert ei.value.status == ta.CAPACITY
    s.close()


def test_replay_latencies_and_results(served):
    qs = _random_queries(served, 300, 3)
    s = _server(served)
    rng = np.random.default_rng(3)
    arrival = np.cumsum(rng.exponential(20000.0, size=len(qs))).astype(np.uint64)
    lat, wall = s.replay(qs, arrival)
    assert (lat > 0).all() and wall >= int(arrival[-1])
    s.close()


def test_invalid_queries_and_budget(served):
    s = ta.Server(context(), result_bytes=1 << 20,
                  device_budget=served[0]["e"].info()["device_bytes"] + (1 << 20))
    s.add(served[0]["e"], None)
    with pytest.raises(ta.TaError) as ei:
        s.add(served[1]["e"], served[1]["topo"])
    assert ei.value.status == ta.OOM
    bad = [ta.make_query(ta.Q_STATS, 0, 10 ** 6, ranks=[0, 1]),
           ta.make_query(ta.Q_STATS, 0, 1, ranks=[3, 2]),
           ta.make_query(ta.Q_TOPK, 0, 1, k=0),
           ta.make_query(ta.Q_TOPK, 0, 1, k=5000),
           ta.make_query(ta.Q_RACKS, 0, 1),  # no topology registered
           ta.make_query(ta.Q_SLICE, 0, 1, r0=5, r1=3),
           ta.make_query(ta.Q_STATS, 7, 1, ranks=[0])]
    for q in bad:
        with pytest.raises(ta.TaError) as ei:
            s.submit(q)
        assert ei.value.status == ta.INVALID_ARG
    s.close()
