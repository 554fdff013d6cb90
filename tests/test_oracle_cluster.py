"""Pins of the oracle's clustering of per-rank values (DBSCAN and K-Means,
the paper's outlier grouping) and of its node view.

Hand-worked examples fix cores, borders (including an equidistant one),
noise and a Lloyd fixed point; scikit-learn's DBSCAN and K-Means (a library
implementation of the same textbook algorithms) must agree wherever the
algorithms leave nothing open; min_pts = 1 reduces DBSCAN to splitting the
sorted values at gaps above eps; and on the generator's config-3 structure
DBSCAN must recover the slowed racks' nodes."""
import numpy as np
import pytest

import oracle
from paper_2605_03561_b300 import synth


def test_dbscan_hand_examples():
    labels, core = oracle.dbscan([1, 2, 3, 10, 11, 12, 30, 6], 1, 2)
    assert labels == [0, 0, 0, 1, 1, 1, -1, -1]
    assert core == [True] * 6 + [False, False]
    # cores 2 and 6 (4 neighbours each within 2); 4 is 2 away from both:
    # the equidistant border joins the cluster of smaller values
    labels, core = oracle.dbscan([0, 1, 2, 4, 6, 7, 8], 2, 4)
    assert core == [False, False, True, False, True, False, False]
    assert labels == [0, 0, 0, 0, 1, 1, 1]
    labels, _ = oracle.dbscan([8, 7, 6, 4, 2, 1, 0], 2, 4)  # order of input irrelevant
    assert labels == [1, 1, 1, 0, 0, 0, 0]
    assert oracle.dbscan([], 3, 2) == ([], [])


def test_dbscan_min_pts_one_splits_at_gaps():
    rng = np.random.default_rng(1)
    for _ in range(20):
        x = rng.integers(0, 400, size=int(rng.integers(1, 80))).tolist()
        eps = int(rng.integers(0, 12))
        labels, core = oracle.dbscan(x, eps, 1)
        assert all(core)
        xs = sorted(set(x))
        cid, expect = 0, {xs[0]: 0}
        for a, b in zip(xs, xs[1:]):
            if b - a > eps:
                cid += 1
            expect[b] = cid
        assert labels == [expect[v] for v in x]


def _clumps(rng, n, centers, spread):
    c = rng.choice(centers, size=n)
    return (c + rng.integers(-spread, spread + 1, size=n)).astype(np.int64)


def test_dbscan_matches_scikit_learn():
    DBSCAN = pytest.importorskip("sklearn.cluster").DBSCAN
    rng = np.random.default_rng(2)
    for trial in range(12):
        x = np.concatenate([_clumps(rng, int(rng.integers(50, 600)), [1000, 1400, 3000], 60),
                            rng.integers(0, 5000, size=int(rng.integers(0, 40)))])
        eps = int(rng.integers(3, 30))
        mp = int(rng.integers(2, 12))
        labels, core = oracle.dbscan(x.tolist(), eps, mp)
        sk = DBSCAN(eps=eps, min_samples=mp).fit(x.reshape(-1, 1).astype(np.float64))
        sk_core = np.zeros(len(x), bool)
        sk_core[sk.core_sample_indices_] = True
        assert np.array_equal(np.array(core), sk_core), trial
        lab = np.array(labels)
        assert np.array_equal(lab == -1, sk.labels_ == -1), trial  # the same noise
        # the same partition of the core points
        pairs = {(a, b) for a, b in zip(lab[sk_core], sk.labels_[sk_core])}
        assert len({a for a, _ in pairs}) == len(pairs) == len({b for _, b in pairs}), trial
        # a border point reachable from one cluster only has no choice to make
        xs = x.tolist()
        for i in np.flatnonzero(~sk_core & (lab >= 0)):
            near = {labels[j] for j in np.flatnonzero(sk_core) if abs(xs[j] - xs[i]) <= eps}
            assert labels[i] in near
            if len(near) == 1:
                assert (labels[i], sk.labels_[i]) in pairs


def test_kmeans_hand_example_and_empty_cluster():
    labels, cents, it, _ = oracle.kmeans([1, 2, 3, 10, 11, 12], 2, 50)
    assert labels == [0, 0, 0, 1, 1, 1] and cents == [2, 11] and it == 1
    # duplicate starts: the second centroid equals the first and stays empty
    labels, cents, it, _ = oracle.kmeans([5, 5, 5, 5, 9], 3, 50)
    assert cents[0] == cents[1] == 5 and cents[2] == 9
    assert labels == [0, 0, 0, 0, 2]
    # one cluster: the mean
    labels, cents, it, _ = oracle.kmeans([4, 8, 9], 1, 10)
    assert labels == [0, 0, 0] and cents == [7]


def test_kmeans_fixed_point_and_scikit_learn():
    KMeans = pytest.importorskip("sklearn.cluster").KMeans
    rng = np.random.default_rng(3)
    for trial in range(10):
        x = np.unique(_clumps(rng, 400, [100, 900, 1500, 4000, 4100], 200))
        rng.shuffle(x)
        k = int(rng.integers(2, 6))
        labels, cents, it, _ = oracle.kmeans(x.tolist(), k, 300)
        assert it < 300
        lab = np.array(labels)
        for j in range(k):  # centroids are the means; points sit at their nearest
            m = x[lab == j]
            if len(m):
                assert cents[j] * len(m) == int(m.sum())
        d = np.array([[abs(v - c) for c in cents] for v in x.tolist()], dtype=object)
        for i in range(len(x)):
            assert d[i][labels[i]] == min(d[i])
        xs = np.sort(x)
        init = np.array([[float(xs[(2 * j + 1) * len(x) // (2 * k)])] for j in range(k)])
        sk = KMeans(n_clusters=k, init=init, n_init=1, algorithm="lloyd", tol=0.0,
                    max_iter=300).fit(x.reshape(-1, 1).astype(np.float64))
        pairs = {(a, b) for a, b in zip(labels, sk.labels_)}
        assert len(pairs) == len({a for a, _ in pairs}) == len({b for _, b in pairs}), trial


def test_cluster_nodes_hand():
    labels = [0, 0, 1, 1, -1, 1, 0, 2]
    nodes = [0, 0, 0, 1, 1, 2, 3, 3]
    per, pair, noise = oracle.cluster_nodes(labels, nodes, 5, 3)
    assert per == [2, 3, 1]
    assert pair[0][1] == 1 and pair[0][2] == 1 and pair[1][2] == 0
    assert noise == 1


def test_clustering_recovers_the_slowed_racks_where_z_scores_mask_them():
    # config-3 structure (22 racks, 3 of them 1.3x slower in communication)
    # at 1,200 ranks = 100 nodes, fixed trace lengths and 8 segments so that a
    # communication context holds ~2,500 samples per rank: with 15 % of the
    # ranks slowed, z stays near 2.4 and the tau = 3 rule flags none of them,
    # while DBSCAN and K-Means (k = 2) both split off exactly the slowed
    # racks' nodes, with no node in both groups
    cfg = synth.preset(3, seed=4, n_ranks=1200, len_mean=20000.0, n_segments=8, len_kind=0)
    g = synth.generate(cfg)
    truth = synth.truth(cfg, g["info"])
    topo = synth.topology(cfg, g["info"])
    node, rack = topo["node_of_rank"], topo["rack_of_node"]
    tr = oracle.Traces(g["rank_off"], g["ts"], g["ctx"], g["parent"], g["marker"])
    a = oracle.Analysis(tr, rows=False)
    seg = int(np.flatnonzero(truth["comm_segment"])[0])
    ctx = int(truth["segment_ctx"][seg])
    _, outl, n_out, _ = a.stats(oracle.EXCL, ctxs=[ctx], tau=(3, 1))
    assert n_out == 0  # masked
    x = a.values(ctx, oracle.EXCL)
    slow_nodes = set(np.flatnonzero(truth["slowed_rack"][rack]).tolist())
    assert len(slow_nodes) == 15
    for labels in (oracle.dbscan(x, int(np.median(x)) // 100, 5)[0],
                   oracle.kmeans(x, 2, 100)[0]):
        assert max(labels) + 1 == 2 and -1 not in labels
        per, pair, noise = oracle.cluster_nodes(labels, node.tolist(), len(rack), 2)
        assert pair[0][1] == 0 and per == [85, 15] and noise == 0
        assert {int(node[r]) for r, l in enumerate(labels) if l == 1} == slow_nodes
