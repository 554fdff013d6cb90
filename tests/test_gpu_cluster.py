"""Parity of ta_cluster_ranks (DBSCAN and K-Means over the ranks' values of a
context, with the node view) with the oracle: labels, cluster sums, bounds,
means and centroids, K-Means update counts and node counts, exactly; and its
error paths."""
import numpy as np
import pytest

import oracle
import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from paper_2605_03561_b300.synth import edge
from gpu_helpers import context, load_both

pytestmark = pytest.mark.gpu

NONE = 0xFFFFFFFF


def _experiment_of_values(x):
    """Rank r holds ctx 1 for x[r] ns (then the root): its exclusive value of
    ctx 1 is x[r]."""
    R = len(x)
    ts = np.zeros(2 * R, np.uint64)
    ts[1::2] = np.asarray(x, np.uint64)
    cx = np.tile(np.array([1, 0], np.uint32), R)
    d = dict(rank_off=np.arange(0, 2 * R + 1, 2, dtype=np.uint64), ts=ts, ctx=cx,
             parent=np.array([NONE, 0], np.uint32), marker=0)
    return load_both(d, rows=False)


def _check_info(got, x_sorted_groups, centroids=None):
    cl = got["clusters"]
    for j, g in enumerate(x_sorted_groups):
        assert int(cl["n"][j]) == len(g)
        if len(g):
            assert int(cl["sum"][j]) == sum(g)
            assert int(cl["min"][j]) == min(g) and int(cl["max"][j]) == max(g)
            assert cl["mean"][j] == float(sum(g)) / float(len(g))
        if centroids is not None:
            s, c = centroids[j]
            assert cl["centroid"][j] == float(s) / float(c)
        elif len(g):
            assert cl["centroid"][j] == cl["mean"][j]


def _dbscan_check(e, x, eps, mp, ranks=None, nodes=None, n_nodes=0, ctx=1, metric=ta.EXCLUSIVE):
    labels, _ = oracle.dbscan(x, eps, mp)
    got = e.cluster(ctx, "dbscan", eps=eps, min_pts=mp, metric=metric, ranks=ranks,
                    node_of_rank=nodes, n_nodes=n_nodes)
    assert got["labels"].tolist() == labels
    nc = max(labels) + 1 if labels else 0
    assert got["n_clusters"] == nc and got["n_noise"] == labels.count(-1)
    _check_info(got, [[v for v, l in zip(x, labels) if l == j] for j in range(nc)])
    if nodes is not None and nc <= 64:
        sub = list(range(len(x))) if ranks is None else list(ranks)
        per, pair, noise = oracle.cluster_nodes(labels, [int(nodes[r]) for r in sub], n_nodes, nc)
        assert got["cluster_nodes"].tolist() == per
        assert got["pair_nodes"].tolist() == [[pair[i][j] if i < j else 0 for j in range(nc)]
                                              for i in range(nc)]
        assert got["noise_nodes"] == noise
    return got


def _kmeans_check(e, x, k, max_iter=300, ranks=None, nodes=None, n_nodes=0, ctx=1,
                  metric=ta.EXCLUSIVE):
    labels, cents, it, pairs = oracle.kmeans(x, k, max_iter)
    got = e.cluster(ctx, "kmeans", k=k, max_iter=max_iter, metric=metric, ranks=ranks,
                    node_of_rank=nodes, n_nodes=n_nodes)
    assert got["labels"].tolist() == labels
    assert got["n_clusters"] == k and got["n_noise"] == 0 and got["iterations"] == it
    _check_info(got, [[v for v, l in zip(x, labels) if l == j] for j in range(k)], pairs)
    if nodes is not None:
        sub = list(range(len(x))) if ranks is None else list(ranks)
        per, pair, noise = oracle.cluster_nodes(labels, [int(nodes[r]) for r in sub], n_nodes, k)
        assert got["cluster_nodes"].tolist() == per
        assert got["pair_nodes"].tolist() == [[pair[i][j] if i < j else 0 for j in range(k)]
                                              for i in range(k)]
    return got


def test_hand_examples():
    tr, a, e = _experiment_of_values([1, 2, 3, 10, 11, 12, 30, 6])
    _dbscan_check(e, [1, 2, 3, 10, 11, 12, 30, 6], 1, 2)
    tr, a, e = _experiment_of_values([0, 1, 2, 4, 6, 7, 8])
    got = _dbscan_check(e, [0, 1, 2, 4, 6, 7, 8], 2, 4)
    assert got["labels"].tolist() == [0, 0, 0, 0, 1, 1, 1]  # the equidistant border goes low
    tr, a, e = _experiment_of_values([1, 2, 3, 10, 11, 12])
    got = _kmeans_check(e, [1, 2, 3, 10, 11, 12], 2)
    assert got["clusters"]["centroid"].tolist() == [2.0, 11.0] and got["iterations"] == 1
    tr, a, e = _experiment_of_values([5, 5, 5, 5, 9])
    got = _kmeans_check(e, [5, 5, 5, 5, 9], 3)  # an empty cluster keeps its centroid
    assert got["clusters"]["n"].tolist() == [4, 0, 1]


def _clumps(rng, n, centers, spread):
    c = rng.choice(centers, size=n)
    return np.maximum(c + rng.integers(-spread, spread + 1, size=n), 0).astype(np.int64)


@pytest.mark.parametrize("seed", range(4))
def test_random_values_subsets_and_nodes(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(300, 3000))
    x = _clumps(rng, n, [1000, 1600, 5000, 5200, 9000], int(rng.integers(20, 200)))
    scatter = rng.random(n) < 0.05  # sparse values between the clumps
    x[scatter] = rng.integers(0, 12000, size=int(scatter.sum()))
    x = x.tolist()
    tr, a, e = _experiment_of_values(x)
    nodes = (np.arange(n) // int(rng.integers(1, 20))).astype(np.uint32)
    n_nodes = int(nodes.max()) + 1
    for eps, mp in ((5, 3), (40, 10), (0, 1), (300, 2), (10_000, 1)):
        _dbscan_check(e, x, eps, mp, nodes=nodes, n_nodes=n_nodes)
    sub = np.sort(rng.choice(n, size=n // 3, replace=False)).astype(np.uint32)
    _dbscan_check(e, [x[r] for r in sub], 30, 5, ranks=sub, nodes=nodes, n_nodes=n_nodes)
    for k in (1, 2, 3, 5, 8, 64):
        _kmeans_check(e, x, k, nodes=nodes if k <= 8 else None, n_nodes=n_nodes)
    _kmeans_check(e, x, 4, max_iter=2)  # stopped before convergence
    _kmeans_check(e, [x[r] for r in sub], 3, ranks=sub, nodes=nodes, n_nodes=n_nodes)


def test_duplicates_ties_and_tiny_sets():
    for x in ([7], [7, 7, 7], [0, 0, 5, 5, 10, 10], [3, 9], list(range(0, 200, 2)) + [99] * 50):
        tr, a, e = _experiment_of_values(x)
        for eps, mp in ((0, 1), (0, 2), (2, 2), (5, 3)):
            _dbscan_check(e, x, eps, mp)
        for k in (1, 2, 3, 7):
            _kmeans_check(e, x, k)


def test_generated_profiles_both_metrics():
    d = edge.case("random_medium", 6)
    tr, a, e = load_both(d)
    csr = a.csr(oracle.EXCL)
    ctx = int(np.bincount(csr["ctx"].astype(np.int64)).argmax())
    for metric, om in ((ta.EXCLUSIVE, oracle.EXCL), (ta.INCLUSIVE, oracle.INCL)):
        x = a.values(ctx, om)
        med = int(np.median(x)) or 1
        _dbscan_check(e, x, med // 20, 4, ctx=ctx, metric=metric)
        _kmeans_check(e, x, 3, ctx=ctx, metric=metric)


def test_planted_slowed_racks():
    cfg = synth.preset(3, seed=4, n_ranks=1200, len_mean=20000.0, n_segments=8, len_kind=0)
    g = synth.generate(cfg)
    truth = synth.truth(cfg, g["info"])
    topo = synth.topology(cfg, g["info"])
    tr, a, e = load_both(g, rows=False)
    ctx = int(truth["segment_ctx"][int(np.flatnonzero(truth["comm_segment"])[0])])
    x = a.values(ctx, oracle.EXCL)
    node = topo["node_of_rank"]
    nn = int(topo["n_nodes"])
    slow_nodes = set(np.flatnonzero(truth["slowed_rack"][topo["rack_of_node"]]).tolist())
    for got in (_dbscan_check(e, x, int(np.median(x)) // 100, 5, nodes=node, n_nodes=nn, ctx=ctx),
                _kmeans_check(e, x, 2, nodes=node, n_nodes=nn, ctx=ctx)):
        assert got["n_clusters"] == 2 and got["pair_nodes"][0, 1] == 0
        assert got["cluster_nodes"].tolist() == [85, 15]
        assert {int(node[r]) for r in np.flatnonzero(got["labels"] == 1)} == slow_nodes


def test_twenty_thousand_ranks():
    rng = np.random.default_rng(11)
    x = _clumps(rng, 20000, [10_000, 14_000, 30_000], 800).tolist()
    tr, a, e = _experiment_of_values(x)
    _dbscan_check(e, x, 3, 4)
    _kmeans_check(e, x, 5)


def test_cluster_errors():
    tr, a, e = _experiment_of_values([1, 2, 3, 50, 51, 52, 100, 101, 102])
    for kw in (dict(method="kmeans", k=0), dict(method="kmeans", k=65),
               dict(method="dbscan", min_pts=0)):
        with pytest.raises(ta.TaError) as ei:
            e.cluster(1, **kw)
        assert ei.value.status == ta.INVALID_ARG
    with pytest.raises(ta.TaError) as ei:
        e.cluster(2, "dbscan", eps=1, min_pts=1)  # ctx >= n_ctx
    assert ei.value.status == ta.INVALID_ARG
    with pytest.raises(ta.TaError) as ei:
        e.cluster(1, "dbscan", eps=1, min_pts=1, node_of_rank=np.array([0] * 8 + [5], np.uint32),
                  n_nodes=3)
    assert ei.value.status == ta.INVALID_ARG
    with pytest.raises(ta.TaError) as ei:
        e.cluster(1, "dbscan", eps=1, min_pts=1, ranks=np.array([3, 2], np.uint32))
    assert ei.value.status == ta.INVALID_ARG
    # too small a cluster capacity: the labels are written, n_clusters is set
    a_ = ta.ClusterArgs()
    a_.method, a_.metric, a_.ctx, a_.mem_kind, a_.eps, a_.min_pts = ta.CLUSTER_DBSCAN, 0, 1, 0, 2, 2
    labels = np.zeros(9, np.int32)
    cl = (ta.ClusterInfo * 1)()
    o = ta.ClusterOut()
    o.labels, o.clusters, o.cluster_cap = labels.ctypes.data, ta.C.addressof(cl), 1
    s = ta.lib().ta_cluster_ranks(e.h, ta.C.byref(a_), ta.C.byref(o))
    assert s == ta.CAPACITY and o.n_clusters == 3
    assert labels.tolist() == [0, 0, 0, 1, 1, 1, 2, 2, 2]
    d = edge.case("random_small", 2)
    e2 = context().load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"],
                        inclusive=False)
    with pytest.raises(ta.TaError) as ei:
        e2.cluster(0, "kmeans", k=2, metric=ta.INCLUSIVE)
    assert ei.value.status == ta.STATE
