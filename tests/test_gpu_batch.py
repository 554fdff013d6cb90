"""Parity of the batched form (ta_batch_plan / ta_batch_run) with the oracle.

Every set of a batch must give, through its set-relative views, exactly the
products the oracle gives for that set alone: the iteration tensor, the
exclusive and inclusive CSR, spans, and the cross-rank statistics of the
exclusive metric over all ranks with their outliers.  Sets differ in rank
count, context count, marker and length, include empty and degenerate sets,
and share 4096-sample tiles with nobody."""
import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import FP_FIELDS, INT_FIELDS, close, context

pytestmark = pytest.mark.gpu


def _sets_mixed(seed):
    sets = [edge.case(n, seed) for n in edge.EDGE_CASES]
    sets += [edge.case("random_small", seed * 10 + k) for k in range(6)]
    sets += [edge.case("random_medium", seed * 10 + k) for k in range(3)]
    sets.append(synth.generate(synth.preset(1, seed=seed + 3, n_ranks=24)))
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(sets))
    return [sets[i] for i in order]


def _tuple(d):
    return (d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])


def _check_set(got, d, tau):
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    a = oracle.Analysis(tr, 0, None, rows=True, incl=True)
    assert got["R"] == tr.R and got["C"] == tr.C
    gt, ot = got["tensor"], a.tensor()
    for k in ("n_iter", "row_off_of_rank", "entry_off", "e_ctx", "e_time", "e_cnt"):
        assert np.array_equal(gt[k], ot[k]), k
    assert np.array_equal(gt["span"], a.span())
    for name, metric in (("exclusive", ta.EXCLUSIVE), ("inclusive", ta.INCLUSIVE)):
        g, o = got[name], a.csr(metric)
        for k in ("off", "ctx", "time", "cnt"):
            assert np.array_equal(g[k], o[k]), (name, k)
    os_, oo, on, _ = a.stats(ta.EXCLUSIVE, tau=tau, want_z=False)
    gs, go = got["stats"], got["outliers"]
    for k in INT_FIELDS:
        assert np.array_equal(gs[k], os_[k]), k
    for k in FP_FIELDS:
        close(gs[k], os_[k], k)
    assert len(go["ctx"]) == on
    assert np.array_equal(go["ctx"], oo["ctx"]) and np.array_equal(go["rank"], oo["rank"])
    close(go["z"], oo["z"], "outlier z")


@pytest.mark.parametrize("seed", range(3))
def test_batch_mixed_sets(seed):
    sets = _sets_mixed(seed)
    tau = (1, 1)
    b = ta.Batch(context(), [_tuple(d) for d in sets], tau=tau)
    info = b.info()
    assert info["n_sets"] == len(sets)
    assert info["graph_kernels"] > 0
    assert info["tune_trials"] >= 12 and info["count_warps"] in (4, 8, 16)
    assert info["tile_width"] in (2048, 4096)  # both widths were tried
    assert info["write_warps"] in (4, 8, 16) and info["write_grid"] >= 1
    for s, d in enumerate(sets):
        _check_set(b.products(s), d, tau)
    b.free()


def test_batch_rerun_is_identical_and_counts_launches():
    sets = _sets_mixed(7)
    b = ta.Batch(context(), [_tuple(d) for d in sets], tau=(2, 1))
    first = [b.products(s) for s in range(len(sets))]
    n0 = context().launches()
    b.run()
    b.run()
    kern = b.info()["graph_kernels"]
    assert context().launches() - n0 >= 2 * kern
    for s in range(len(sets)):
        again = b.products(s)
        for part in ("tensor", "exclusive", "inclusive", "stats", "outliers"):
            for k, v in first[s][part].items():
                assert np.array_equal(v, again[part][k]), (s, part, k)
    _check_set(b.products(len(sets) - 1), sets[-1], (2, 1))


def test_batch_many_generated_sets():
    # Uneven generated sets (ranks, contexts, lengths) as the batched workload draws them.
    rng = np.random.default_rng(11)
    sets = []
    for k in range(40):
        R = int(rng.integers(4, 60))
        Cn = int(np.exp(rng.uniform(np.log(100), np.log(3000))))
        cfg = synth.preset(1, seed=100 + k, n_ranks=R, n_ctx=Cn,
                           len_mean=float(rng.integers(2000, 12000)))
        sets.append(synth.generate(cfg))
    b = ta.Batch(context(), [_tuple(d) for d in sets])
    for s in (0, 7, 19, 39):
        _check_set(b.products(s), sets[s], (3, 1))


def test_batch_capacity_then_views_empty():
    sets = _sets_mixed(1)
    b = ta.Batch(context(), [_tuple(d) for d in sets], tau=(1, 2), outlier_cap=2)
    with pytest.raises(ta.TaError) as ei:
        b.run()
    assert ei.value.status == ta.CAPACITY
    assert b.info()["n_outliers"] > 2
    assert b.view(0).n_outliers == 0
    # the other products stay valid
    got = b.products(3)
    tr = oracle.Traces(*_tuple(sets[3]))
    a = oracle.Analysis(tr, 0, None, rows=True, incl=True)
    assert np.array_equal(got["tensor"]["e_time"], a.tensor()["e_time"])


def test_batch_rejects_invalid_sets():
    good = edge.case("random_small", 1)
    bad_ctx = dict(good)
    bad_ctx["ctx"] = good["ctx"].copy()
    if len(bad_ctx["ctx"]):
        bad_ctx["ctx"][0] = len(good["parent"])
        with pytest.raises(ta.TaError) as ei:
            ta.Batch(context(), [_tuple(good), _tuple(bad_ctx)])
        assert ei.value.status == ta.BAD_CTX
    two_roots = dict(good)
    p = np.full(3, 0xFFFFFFFF, np.uint32)
    two_roots.update(parent=p, ctx=np.zeros_like(good["ctx"]), marker=0)
    with pytest.raises(ta.TaError) as ei:
        ta.Batch(context(), [_tuple(good), _tuple(two_roots)])
    assert ei.value.status == ta.BAD_CCT and "set 1" in str(ei.value)
    unsorted = dict(good)
    ts = good["ts"].copy()
    ro = good["rank_off"]
    r = int(np.argmax(np.diff(ro.astype(np.int64)) >= 2))
    b0 = int(ro[r])
    ts[b0], ts[b0 + 1] = ts[b0] + 5, ts[b0]
    unsorted["ts"] = ts
    with pytest.raises(ta.TaError) as ei:
        ta.Batch(context(), [_tuple(unsorted), _tuple(good)])
    assert ei.value.status == ta.NOT_SORTED


def test_batch_speedup_and_rollup_per_set():
    # Every set asks for the potential speedup over a context list and a rack
    # rollup of one context (as ta_potential_speedup / ta_topology_rollup over
    # all its ranks); sets differ in shape, iterations and topology.
    from gpu_helpers import SP_FP, SP_INT, simple_topology
    rng = np.random.default_rng(21)
    sets = _sets_mixed(4)
    sets += [synth.generate(synth.preset(1, seed=40 + k, n_ranks=int(rng.integers(8, 40))))
             for k in range(4)]
    args = []
    for k, d in enumerate(sets):
        R = len(d["rank_off"]) - 1
        Cn = len(d["parent"])
        present = np.unique(d["ctx"]) if len(d["ctx"]) else np.array([0], np.uint32)
        if k % 5 == 4:
            args.append(None)  # no requests for this set
            continue
        kset = np.unique(rng.choice(present, size=min(len(present), 70))).astype(np.uint32)
        topo = simple_topology(R, int(rng.integers(1, 4)), int(rng.integers(1, 4)), 2)
        args.append(dict(speedup_ctxs=kset, app_time_ns=0 if k % 2 else 10**9, topology=topo,
                         topo_ctx=int(rng.choice(present)), topo_tau=(int(rng.integers(1, 3)), 1),
                         min_ranks=int(rng.integers(1, 3))))
    b = ta.Batch(context(), [_tuple(d) for d in sets], tau=(2, 1), set_args=args)
    for s, d in enumerate(sets):
        got = b.products(s)
        if args[s] is None:
            assert "speedup" not in got and "topology" not in got
            continue
        tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
        a = oracle.Analysis(tr)
        gp, gt = got["speedup"]
        op, ot = a.speedup(args[s]["speedup_ctxs"], app_time_ns=args[s]["app_time_ns"])
        for k in SP_INT:
            assert np.array_equal(gp[k], op[k]), (s, k)
        for k in SP_FP:
            close(gp[k], op[k], k)
        for k in ("i_star", "excluded_iterations", "sum_G", "t_app"):
            assert gt[k] == ot[k], (s, k)
        for k in ("total_reduction", "speedup_fraction"):
            close([gt[k]], [ot[k]], k)
        t = args[s]["topology"]
        o = a.topology(args[s]["topo_ctx"], t["node_of_rank"], t["rack_of_node"],
                       t["chassis_of_node"], t["n_racks"], t["n_chassis"], metric=ta.EXCLUSIVE,
                       tau=args[s]["topo_tau"], min_ranks=args[s]["min_ranks"])
        for k in o:
            assert np.array_equal(got["topology"][k], o[k]), (s, k)
    # a second replay gives the same results
    before = b.products(1)
    b.run()
    again = b.products(1)
    if "speedup" in before:
        assert np.array_equal(before["speedup"][0]["G_lo"], again["speedup"][0]["G_lo"])
