"""Parity at the full plain-at-scale size (100,000 ranks, C = 20,000, about
2e9 records), in the launch configuration the benchmark times.

The oracle analyses sampled rank ranges one by one (their tensor, exclusive
and inclusive CSR and spans must match bit for bit); the rest is checked
through properties that hold at any size: every rank's exclusive times sum to
its span and its inclusive root equals it, the tensor sums back to the
exclusive CSR, and the statistics' integer moments equal sums over the
exclusive CSR.  The FP64 statistics (mean, std, cv, balance, every outlier's
z), the outlier lists, the rack rollup and the potential speedup are compared
with the oracle over a contiguous subset of 3,000 ranks, which the oracle
analyses on its own."""
import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from gpu_helpers import (INT_FIELDS, check_speedup, check_stats, check_topology, context,
                         per_rank_rows)

pytestmark = pytest.mark.gpu


def _enough_host_memory(gb):
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024 > gb * 2**30
    except OSError:
        pass
    return False


@pytest.mark.skipif(not _enough_host_memory(96), reason="needs ~96 GB of host memory")
def test_full_size_config3_sampled_and_invariants():
    cfg = synth.preset(3, seed=1)
    g = synth.generate(cfg)
    R = cfg.n_ranks
    assert R == 100000 and int(g["rank_off"][-1]) > 1.5e9
    e = context().load(g["rank_off"], g["ts"], g["ctx"], g["parent"], g["marker"],
                       keep_traces=True)
    tr = oracle.Traces(g["rank_off"], g["ts"], g["ctx"], g["parent"], g["marker"])
    t = e.tensor()
    x = e.csr(ta.EXCLUSIVE)
    inc = e.csr(ta.INCLUSIVE)
    span = e.span()
    rng = np.random.default_rng(5)
    for r0 in [0, R - 4] + sorted(rng.integers(1, R - 4, size=6).tolist()):
        a = oracle.Analysis(tr, r0, r0 + 4)
        ot = a.tensor()
        assert np.array_equal(t["n_iter"][r0:r0 + 4], ot["n_iter"])
        for r in range(r0, r0 + 4):
            assert per_rank_rows(t, r) == per_rank_rows(ot, r - r0), r
        for g_csr, metric in ((x, ta.EXCLUSIVE), (inc, ta.INCLUSIVE)):
            o = a.csr(metric)
            for r in range(r0, r0 + 4):
                b, q = int(g_csr["off"][r]), int(g_csr["off"][r + 1])
                ob, oq = int(o["off"][r - r0]), int(o["off"][r - r0 + 1])
                for k in ("ctx", "time", "cnt"):
                    assert np.array_equal(g_csr[k][b:q], o[k][ob:oq]), (metric, r, k)
        assert np.array_equal(span[r0:r0 + 4], a.span())
    # invariants over every rank
    xo = x["off"].astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(x["time"].astype(np.uint64), dtype=np.uint64)])
    per_rank = cs[xo[1:]] - cs[xo[:-1]]
    assert np.array_equal(per_rank, span)  # a rank's exclusive times add up to its span
    io = inc["off"].astype(np.int64)
    nonempty = np.diff(io) > 0
    first = io[:-1][nonempty]
    assert (inc["ctx"][first] == 0).all()  # the root leads every non-empty list
    assert np.array_equal(inc["time"][first], span[nonempty])
    tot_t = int(t["e_time"].astype(np.uint64).sum(dtype=np.uint64))
    assert tot_t == int(x["time"].astype(np.uint64).sum(dtype=np.uint64))
    assert int(t["e_cnt"].sum(dtype=np.uint64)) == int(g["rank_off"][-1])
    # statistics of sampled contexts against sums over the exclusive CSR
    ctxs = np.unique(x["ctx"][rng.integers(0, len(x["ctx"]), size=12)]).astype(np.uint32)
    gs, _, _, _ = e.stats(ta.EXCLUSIVE, ctxs=ctxs, tau=(3, 1), outlier_cap=1 << 20)
    for i, c in enumerate(ctxs):
        sel = x["ctx"] == c
        vals = x["time"][sel].astype(object)
        assert int(gs["n"][i]) == R
        assert int(gs["present"][i]) == int(sel.sum())
        assert int(gs["s1"][i]) == int(sum(vals))
        s2 = int(sum(v * v for v in vals))
        assert int(gs["s2_lo"][i]) + (int(gs["s2_hi"][i]) << 64) == s2
        assert int(gs["max"][i]) == int(max(vals))
        assert set(INT_FIELDS) <= set(gs)
    # FP64 statistics, outliers, rack rollup and speedup over a contiguous
    # subset of ranks the oracle analyses by itself (global rank ids)
    s0 = int(rng.integers(0, R - 3000))
    S = np.arange(s0, s0 + 3000, dtype=np.uint32)
    a = oracle.Analysis(tr, s0, s0 + 3000)
    check_stats(a, e, ta.EXCLUSIVE, ranks=S, tau=(3, 1), want_z=False)
    check_stats(a, e, ta.EXCLUSIVE, ranks=S, tau=(2, 1), want_z=False)
    check_stats(a, e, ta.INCLUSIVE, ranks=S, tau=(3, 1), want_z=False)
    truth = synth.truth(cfg, g["info"])
    kset = np.unique(truth["segment_ctx"]).astype(np.uint32)
    check_speedup(a, e, kset, ranks=S)
    topo = synth.topology(cfg, g["info"])
    comm = truth["segment_ctx"][truth["comm_segment"].astype(bool)]
    check_topology(a, e, int(comm[0]), topo, tau=(2, 1), ranks=S)
    del a
    # time-window profiles: sampled rank ranges against the oracle, every
    # rank's totals against the closed form (overlap of the window with the
    # rank's span; samples with ts in the window)
    ts, ro = g["ts"], g["rank_off"].astype(np.int64)
    lo, hi = int(ts[ro[:-1][ro[1:] > ro[:-1]]].min()), int(ts.max()) + 1
    t0, t1 = lo + (hi - lo) * 45 // 100, lo + (hi - lo) * 55 // 100
    win = e.interval(t0, t1)
    for r0 in [0, R - 4] + sorted(rng.integers(1, R - 4, size=4).tolist()):
        a = oracle.Analysis(tr, r0, r0 + 4, rows=False, incl=False)
        o = a.interval(t0, t1)
        for r in range(r0, r0 + 4):
            b, q = int(win["off"][r]), int(win["off"][r + 1])
            ob, oq = int(o["off"][r - r0]), int(o["off"][r - r0 + 1])
            for k in ("ctx", "time", "cnt"):
                assert np.array_equal(win[k][b:q], o[k][ob:oq]), ("interval", r, k)
    wo = win["off"].astype(np.int64)
    ct = np.concatenate([[0], np.cumsum(win["time"].astype(np.uint64), dtype=np.uint64)])
    cn = np.concatenate([[0], np.cumsum(win["cnt"].astype(np.uint64), dtype=np.uint64)])
    got_t, got_n = ct[wo[1:]] - ct[wo[:-1]], cn[wo[1:]] - cn[wo[:-1]]
    for r in range(R):
        b, q = int(ro[r]), int(ro[r + 1])
        if q == b:
            assert got_t[r] == 0 and got_n[r] == 0
            continue
        x = ts[b:q]
        assert int(got_t[r]) == max(0, min(t1, int(x[-1])) - max(t0, int(x[0]))), r
        assert int(got_n[r]) == int(np.searchsorted(x, t1) - np.searchsorted(x, t0)), r
