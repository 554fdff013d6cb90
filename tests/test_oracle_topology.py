"""Pins of the oracle's topology rollup (Section VI-B: outlier ranks joined to
their compute nodes, nodes to chassis and racks).

Hand-built topologies fix every output array by hand: which nodes are
flagged (a node, not a rank, is what a chassis or rack counts), the node
sums over all of a node's ranks (outliers or not), the min_ranks boundary,
and a rank subset (ranks outside it add nothing).  On the generator's
config-3 structure the rollup at tau = 2 must flag exactly the planted slow
racks."""
import numpy as np
import pytest

import oracle
from paper_2605_03561_b300 import synth

NONE = 0xFFFFFFFF

# 24 ranks, 4 per node -> 6 nodes; chassis = node // 2 (3 chassis), rack =
# node // 3 (2 racks).  Chassis 1 (nodes 2, 3) straddles the two racks.
NODE = np.arange(24, dtype=np.uint32) // 4
CHASSIS = np.arange(6, dtype=np.uint32) // 2
RACK = np.arange(6, dtype=np.uint32) // 3


def _traces(x):
    """Rank r: a sample of context 2 at t = 0, then one of context 3 at
    t = x[r], so rank r's exclusive time of context 2 is x[r]."""
    R = len(x)
    ts = np.zeros(2 * R, np.uint64)
    ts[1::2] = x
    cx = np.tile(np.array([2, 3], np.uint32), R)
    ro = np.arange(0, 2 * R + 1, 2, dtype=np.uint64)
    parent = np.array([NONE, 0, 0, 0], np.uint32)
    return oracle.Traces(ro, ts, cx, parent, 1)


def _values():
    # ranks 16..19 (all of node 4) and rank 5 (one rank of node 1) are slow
    x = np.full(24, 100, np.uint64)
    x[16:20] = 1000
    x[5] = 1000
    return x


def _topo(a, x, tau=(3, 2), min_ranks=1, ranks=None):
    return a.topology(2, NODE, RACK, CHASSIS, 2, 3, tau=tau, min_ranks=min_ranks, ranks=ranks)


def test_outliers_of_the_hand_topology():
    # over all 24 ranks: mean 287.5, std 373.4 (ddof 1); the five slow ranks
    # have z = 1.91 > 1.5, the others z = -0.50
    x = _values()
    a = oracle.Analysis(_traces(x))
    _, outl, n, _ = a.stats(oracle.EXCL, ctxs=[2], tau=(3, 2))
    assert n == 5 and outl["rank"].tolist() == [5, 16, 17, 18, 19]


def test_hand_topology_every_output():
    x = _values()
    o = _topo(oracle.Analysis(_traces(x)), x)
    assert o["node_outliers"].tolist() == [0, 1, 0, 0, 4, 0]
    assert o["node_ranks"].tolist() == [4] * 6
    # sums over ALL of a node's ranks, not just its outliers
    assert o["node_sum"].tolist() == [400, 1300, 400, 400, 4000, 400]
    assert o["node_flag"].tolist() == [0, 1, 0, 0, 1, 0]
    # chassis and racks count flagged NODES (node 4's four outliers are one)
    assert o["chassis_flagged"].tolist() == [1, 0, 1]
    assert o["chassis_nodes"].tolist() == [2, 2, 2]
    assert o["chassis_sum"].tolist() == [1700, 800, 4400]
    assert o["rack_flagged"].tolist() == [1, 1]
    assert o["rack_nodes"].tolist() == [3, 3]
    assert o["rack_sum"].tolist() == [2100, 4800]
    assert o["flagged_racks"].tolist() == [0, 1]


def test_one_whole_node_flags_exactly_that_node_and_its_rack():
    x = np.full(24, 100, np.uint64)
    x[16:20] = 1000  # every rank of node 4, nothing else
    o = _topo(oracle.Analysis(_traces(x)), x, tau=(2, 1))  # their z = 2.19
    assert o["node_outliers"].tolist() == [0, 0, 0, 0, 4, 0]
    assert o["node_flag"].tolist() == [0, 0, 0, 0, 1, 0]
    assert o["chassis_flagged"].tolist() == [0, 0, 1]
    assert o["rack_flagged"].tolist() == [0, 1]
    assert o["flagged_racks"].tolist() == [1]
    assert o["rack_sum"].tolist() == [1200, 4800]


@pytest.mark.parametrize("min_ranks,flags,racks", [
    (1, [0, 1, 0, 0, 1, 0], [0, 1]),
    (2, [0, 0, 0, 0, 1, 0], [1]),
    (3, [0, 0, 0, 0, 1, 0], [1]),
    (4, [0, 0, 0, 0, 1, 0], [1]),   # k outliers flag the node at min_ranks = k
    (5, [0, 0, 0, 0, 0, 0], []),    # and not at k + 1
])
def test_min_ranks_boundary(min_ranks, flags, racks):
    x = _values()
    o = _topo(oracle.Analysis(_traces(x)), x, min_ranks=min_ranks)
    assert o["node_outliers"].tolist() == [0, 1, 0, 0, 4, 0]  # independent of min_ranks
    assert o["node_flag"].tolist() == flags
    assert o["flagged_racks"].tolist() == racks
    assert o["rack_flagged"].tolist() == [int(flags[0] + flags[1] + flags[2]),
                                          int(flags[3] + flags[4] + flags[5])]


def test_rank_subset_adds_nothing_outside_it():
    # S = ranks 0..15 without 2 and 5, plus 17: node 1 keeps 3 ranks and
    # loses its slow one, node 4 keeps one slow rank, node 5 has none.
    # Over S (15 ranks, one of them at 1000): mean 160, z(17) = 3.61, others -0.26
    x = _values()
    S = np.array([r for r in range(16) if r not in (2, 5)] + [17], np.uint32)
    a = oracle.Analysis(_traces(x))
    _, outl, n, _ = a.stats(oracle.EXCL, ctxs=[2], ranks=S, tau=(3, 1))
    assert n == 1 and outl["rank"].tolist() == [17]
    o = _topo(a, x, tau=(3, 1), ranks=S)
    assert o["node_ranks"].tolist() == [3, 3, 4, 4, 1, 0]
    assert o["node_sum"].tolist() == [300, 300, 400, 400, 1000, 0]
    assert o["node_outliers"].tolist() == [0, 0, 0, 0, 1, 0]
    assert o["node_flag"].tolist() == [0, 0, 0, 0, 1, 0]
    assert o["chassis_nodes"].tolist() == [2, 2, 2]  # topology counts, not subset counts
    assert o["chassis_sum"].tolist() == [600, 800, 1000]
    assert o["rack_sum"].tolist() == [1000, 1400]
    assert o["flagged_racks"].tolist() == [1]


def test_planted_slow_racks_recovered_at_tau_two():
    # config-3 structure (12 ranks per node, 22 racks, 3 racks 1.3x slower in
    # communication contexts) at 1,200 ranks with fixed trace lengths: the
    # slowed ranks' z sits near 2.5, so tau = 2 flags them (tau = 3 would
    # not: the masking of a 15 % slow minority), and the rollup must name
    # exactly the planted racks and their nodes
    cfg = synth.preset(3, seed=4, n_ranks=1200, len_mean=20000.0, n_segments=8, len_kind=0)
    g = synth.generate(cfg)
    truth = synth.truth(cfg, g["info"])
    topo = synth.topology(cfg, g["info"])
    tr = oracle.Traces(g["rank_off"], g["ts"], g["ctx"], g["parent"], g["marker"])
    a = oracle.Analysis(tr, rows=False)
    seg = int(np.flatnonzero(truth["comm_segment"])[0])
    ctx = int(truth["segment_ctx"][seg])
    o = a.topology(ctx, topo["node_of_rank"], topo["rack_of_node"], topo["chassis_of_node"],
                   topo["n_racks"], topo["n_chassis"], tau=(2, 1))
    slow_racks = np.flatnonzero(truth["slowed_rack"]).tolist()
    assert len(slow_racks) == 3
    assert o["flagged_racks"].tolist() == slow_racks
    slow_nodes = truth["slowed_rack"][topo["rack_of_node"]].astype(bool)
    assert np.array_equal(o["node_flag"].astype(bool), slow_nodes)
    # no rank outside the slowed racks is an outlier; the slowed ranks' z
    # scatters around 2.5 with their own sampling noise, so most (not all)
    # of them clear tau = 2 -- at least one per node, which flags every node
    slowed_per_node = np.bincount(topo["node_of_rank"], weights=truth["slowed_rank"],
                                  minlength=len(topo["rack_of_node"]))
    assert np.all(o["node_outliers"] <= slowed_per_node)
    assert o["node_outliers"].sum() >= 0.9 * truth["slowed_rank"].sum()
    assert np.array_equal(o["node_ranks"], np.bincount(topo["node_of_rank"],
                                                       minlength=len(topo["rack_of_node"])))
    for q in range(topo["n_racks"]):
        nodes = topo["rack_of_node"] == q
        assert o["rack_nodes"][q] == nodes.sum()
        assert o["rack_sum"][q] == o["node_sum"][nodes].sum()
        assert o["rack_flagged"][q] == (nodes & slow_nodes).sum()
