"""Shared checks of the CUDA path against the CPU oracle (used by -m gpu tests).

Integer outputs must match bit for bit; FP64 statistics within 1e-12
relative (the tolerance the method states for moments and z-scores)."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2605_03561_b300 as ta

RTOL = 1e-12

_ctx = None


def context():
    global _ctx
    if _ctx is None:
        _ctx = ta.Context(0)
    return _ctx


def per_rank_rows(t, r, base_row=0):
    rows = []
    for row in range(int(t["row_off_of_rank"][r]), int(t["row_off_of_rank"][r + 1])):
        b, e = int(t["entry_off"][row]), int(t["entry_off"][row + 1])
        rows.append((t["e_ctx"][b:e].tolist(), t["e_time"][b:e].tolist(), t["e_cnt"][b:e].tolist()))
    return rows


def close(a, b, what):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape, what
    np.testing.assert_allclose(a, b, rtol=RTOL, atol=0, err_msg=what)


def load_both(d, r0=0, r1=None, rows=True, incl=True, **kw):
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    a = oracle.Analysis(tr, r0, r1, rows=rows, incl=incl)
    e = context().load(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"], **kw)
    return tr, a, e


def check_products(tr, a, e, r0=0, r1=None):
    """Tensor, exclusive, inclusive and spans of ranks [r0, r1) bit-exact."""
    r1 = tr.R if r1 is None else r1
    gt, ot = e.tensor(), a.tensor()
    assert np.array_equal(gt["n_iter"][r0:r1], ot["n_iter"])
    go = gt["row_off_of_rank"]
    assert np.array_equal(np.diff(go.astype(np.int64))[r0:r1],
                          np.diff(ot["row_off_of_rank"].astype(np.int64)))
    if r0 == 0 and r1 == tr.R:
        for k in ("row_off_of_rank", "entry_off", "e_ctx", "e_time", "e_cnt"):
            assert np.array_equal(gt[k], ot[k]), k
    else:
        for r in range(r0, r1):
            assert per_rank_rows(gt, r) == per_rank_rows(ot, r - r0), r
    for metric in (ta.EXCLUSIVE, ta.INCLUSIVE):
        g, o = e.csr(metric), a.csr(metric)
        if r0 == 0 and r1 == tr.R:
            for k in ("off", "ctx", "time", "cnt"):
                assert np.array_equal(g[k], o[k]), (metric, k)
        else:
            for r in range(r0, r1):
                b, q = int(g["off"][r]), int(g["off"][r + 1])
                ob, oq = int(o["off"][r - r0]), int(o["off"][r - r0 + 1])
                for k in ("ctx", "time", "cnt"):
                    assert np.array_equal(g[k][b:q], o[k][ob:oq]), (metric, r, k)
    assert np.array_equal(e.span()[r0:r1], a.span())


INT_FIELDS = ("n", "present", "argmax", "min", "max", "s1", "s2_lo", "s2_hi")
FP_FIELDS = ("mean", "std", "cv", "balance")


def check_stats(a, e, metric, ranks=None, ctxs=None, tau=(3, 1), want_z=True):
    gs, go, gn, gz = e.stats(metric, ranks=ranks, ctxs=ctxs, tau=tau, want_z=want_z)
    os_, oo, on, oz = a.stats(metric, ranks=ranks, ctxs=ctxs, tau=tau, want_z=want_z)
    for k in INT_FIELDS:
        assert np.array_equal(gs[k], os_[k]), k
    for k in FP_FIELDS:
        close(gs[k], os_[k], k)
    assert gn == on
    assert np.array_equal(go["ctx"], oo["ctx"]) and np.array_equal(go["rank"], oo["rank"])
    close(go["z"], oo["z"], "outlier z")
    if want_z and a.r0 == 0 and a.r1 == a.tr.R:
        close(gz, oz, "z per entry")
    return gs, go


SP_INT = ("A", "B", "G_lo", "G_hi")
SP_FP = ("avg_mean", "avg_max", "savings_per_iter", "total_reduction", "share", "cv_across",
         "cv_within")


def check_speedup(a, e, ctxs, ranks=None, app_time_ns=0):
    gp, gt = e.speedup(ctxs, ranks=ranks, app_time_ns=app_time_ns)
    op, ot = a.speedup(ctxs, ranks=ranks, app_time_ns=app_time_ns)
    for k in SP_INT:
        assert np.array_equal(gp[k], op[k]), k
    for k in SP_FP:
        close(gp[k], op[k], k)
    for k in ("i_star", "excluded_iterations", "sum_G", "t_app"):
        assert gt[k] == ot[k], k
    for k in ("total_reduction", "speedup_fraction"):
        close(gt[k], ot[k], k)
    return gp, gt


def check_topology(a, e, ctx, topo, metric=ta.EXCLUSIVE, tau=(3, 1), min_ranks=1, ranks=None):
    g = e.topology(ctx, topo["node_of_rank"], topo["rack_of_node"], topo["chassis_of_node"],
                   topo["n_racks"], topo["n_chassis"], metric=metric, tau=tau,
                   min_ranks=min_ranks, ranks=ranks)
    o = a.topology(ctx, topo["node_of_rank"], topo["rack_of_node"], topo["chassis_of_node"],
                   topo["n_racks"], topo["n_chassis"], metric=metric, tau=tau,
                   min_ranks=min_ranks, ranks=ranks)
    for k in o:
        assert np.array_equal(g[k], o[k]), k
    return g


def simple_topology(R, ranks_per_node=3, nodes_per_rack=4, nodes_per_chassis=2):
    nn = (R + ranks_per_node - 1) // ranks_per_node
    node = (np.arange(R) // ranks_per_node).astype(np.uint32)
    rack = (np.arange(nn) // nodes_per_rack).astype(np.uint32)
    chassis = (np.arange(nn) // nodes_per_chassis).astype(np.uint32)
    return dict(node_of_rank=node, rack_of_node=rack, chassis_of_node=chassis,
                n_racks=int(rack.max()) + 1, n_chassis=int(chassis.max()) + 1, n_nodes=nn)
