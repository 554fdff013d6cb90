"""The sharded form: a job's ranks split into contiguous shards, each loaded
as its own experiment, and merged through one exchange of partials (here
summed, min-ed and max-ed over the shards on one GPU, as an all-reduce
would) against the unsharded experiment.  Statistics of both metrics (every
integer and FP64 field, argmax), the outlier lists, the rack rollup and the
potential speedup must match bit for bit; only cv_within, a sum of FP64 terms
merged across shards, is compared within 1e-12 relative."""
import numpy as np
import pytest

import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth
from gpu_helpers import RTOL, context

pytestmark = pytest.mark.gpu


def _shards(g, bounds, R):
    out = []
    for r0, r1 in zip(bounds[:-1], bounds[1:]):
        ro = g["rank_off"][r0:r1 + 1]
        a, b = int(ro[0]), int(ro[-1])
        e = context().load((ro - ro[0]).astype(np.uint64), g["ts"][a:b], g["ctx"][a:b],
                           g["parent"], g["marker"])
        out.append((r0, r1, ta.Shard(e, r0, R)))
    return out


def _reduce(parts, op):
    import torch
    x = torch.stack(parts)
    return {"sum": x.sum(0), "min": x.min(0).values, "max": x.max(0).values}[op]


@pytest.mark.parametrize("bounds", [[0, 600], [0, 170, 171, 600], [0, 150, 300, 450, 600]])
def test_shards_equal_the_whole_job(bounds):
    import torch
    cfg = synth.preset(3, seed=9, n_ranks=600, len_mean=6000.0)
    g = synth.generate(cfg)
    R = cfg.n_ranks
    whole = context().load(g["rank_off"], g["ts"], g["ctx"], g["parent"], g["marker"])
    shards = _shards(g, bounds, R)
    truth = synth.truth(cfg, g["info"])
    topo = synth.topology(cfg, g["info"])
    comm = int(truth["segment_ctx"][truth["comm_segment"].astype(bool)][0])
    for metric, tau in ((ta.EXCLUSIVE, (2, 1)), (ta.INCLUSIVE, (3, 1))):
        parts = [s.stats_partials(metric) for _, _, s in shards]
        merged = {k: _reduce([p[k] for p in parts], op)
                  for k, op in (("sums", "sum"), ("mins", "min"), ("maxs", "max"))}
        fin = [s.stats_finalize(merged, metric, tau) for _, _, s in shards]
        argmax = _reduce([f[1] for f in fin], "min")
        got = shards[0][2].set_argmax(fin[0][0], argmax)
        ref, ref_out, ref_n, _ = whole.stats(metric, tau=tau)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (metric, k)  # FP64 too: same integers in
        ctx_ = np.concatenate([f[2]["ctx"] for f in fin])
        rank = np.concatenate([f[2]["rank"] for f in fin])
        z = np.concatenate([f[2]["z"] for f in fin])
        order = np.lexsort((rank, ctx_))
        assert len(order) == ref_n
        assert np.array_equal(ctx_[order], ref_out["ctx"])
        assert np.array_equal(rank[order], ref_out["rank"])
        assert np.array_equal(z[order], ref_out["z"])
        # rack rollup of a communication context
        node = topo["node_of_rank"]
        nn = int(topo["n_nodes"])
        nparts = [s.topology_partials(merged, comm, node[r0:r1], nn, metric, tau)
                  for r0, r1, s in shards]
        rolled = ta.topology_finalize(context(), _reduce(nparts, "sum"), topo["rack_of_node"],
                                      topo["chassis_of_node"], topo["n_racks"],
                                      topo["n_chassis"])
        ref_t = whole.topology(comm, node, topo["rack_of_node"], topo["chassis_of_node"],
                               topo["n_racks"], topo["n_chassis"], metric=metric, tau=tau)
        for k in ref_t:
            assert np.array_equal(rolled[k], ref_t[k]), (metric, k)
    # potential speedup over the iteration program
    kset = np.unique(truth["segment_ctx"]).astype(np.uint32)
    b = [s.speedup_bounds() for _, _, s in shards]
    i_star = min(x[0] for x in b)
    excluded = sum(x[1] for x in b) - R * i_star
    t_app = max(x[2] for x in b)
    sp = [s.speedup_partials(kset, i_star) for _, _, s in shards]
    msp = {"cells": _reduce([p["cells"] for p in sp], "sum"),
           "cell_max": _reduce([p["cell_max"] for p in sp], "max"),
           "within": torch.stack([p["within"] for p in sp]).sum(0)}
    gp, gt = ta.speedup_finalize(context(), msp, R, i_star, excluded, t_app, len(kset))
    rp, rt = whole.speedup(kset)
    for k in ("A", "B", "G_lo", "G_hi", "avg_mean", "avg_max", "savings_per_iter",
              "total_reduction", "share", "cv_across"):
        assert np.array_equal(gp[k], rp[k]), k
    np.testing.assert_allclose(gp["cv_within"], rp["cv_within"], rtol=RTOL, atol=0)
    for k in ("i_star", "excluded_iterations", "sum_G", "t_app", "total_reduction",
              "speedup_fraction"):
        assert gt[k] == rt[k], k
    for _, _, s in shards:
        s.e.free()
    whole.free()
