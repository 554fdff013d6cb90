"""The seeded generator: deterministic, chunkable, and shaped as documented."""
import numpy as np

from paper_2605_03561_b300 import synth


def test_deterministic_and_chunked():
    cfg = synth.preset(2, seed=4, n_ranks=40, len_mean=3000.0)
    a = synth.generate(cfg)
    b = synth.generate(cfg, n_threads=1)
    assert np.array_equal(a["ts"], b["ts"]) and np.array_equal(a["ctx"], b["ctx"])
    ro = a["rank_off"]
    ts = np.empty(int(ro[40] - ro[13]), np.uint64)
    cx = np.empty_like(ts, dtype=np.uint32)
    synth.fill(cfg, ro, 13, 40, ts.ctypes.data, cx.ctypes.data, 3)
    assert np.array_equal(ts, a["ts"][int(ro[13]):]) and np.array_equal(cx, a["ctx"][int(ro[13]):])
    c = synth.generate(synth.preset(2, seed=5, n_ranks=40, len_mean=3000.0))
    assert not np.array_equal(c["ts"][:100], a["ts"][:100])


def test_structure():
    cfg = synth.preset(1, seed=2, n_ranks=6)
    g = synth.generate(cfg)
    ro, ts, ctx, parent = g["rank_off"], g["ts"], g["ctx"], g["parent"]
    assert int(ro[-1]) == 6 * 20000 and np.all(np.diff(ro) == 20000)
    assert np.all(ctx < cfg.n_ctx)
    depth = np.zeros(cfg.n_ctx, int)
    for v in range(1, cfg.n_ctx):
        assert parent[v] < v
        depth[v] = depth[parent[v]] + 1
    assert depth.max() <= cfg.max_depth and parent[0] == 0xFFFFFFFF
    for r in range(6):
        t = ts[int(ro[r]):int(ro[r + 1])]
        c = ctx[int(ro[r]):int(ro[r + 1])]
        assert np.all(np.diff(t.astype(np.int64)) >= 1)
        starts = (c == 1) & np.concatenate([[True], c[:-1] != 1])
        assert starts.sum() == cfg.n_iter
        assert np.all(c[:cfg.prologue_len] == g["info"].prologue_ctx)
        assert len(np.unique(c)) == g["info"].n_segments + 2  # segments, marker, prologue


def test_lognormal_lengths_and_topology():
    cfg = synth.preset(3, seed=1, n_ranks=5000)
    ro, parent, info = synth.plan(cfg)
    L = np.diff(ro).astype(np.float64)
    assert abs(L.mean() / 20000 - 1) < 0.05
    assert L.min() >= cfg.n_iter * 65 + 16 and L.max() <= 20 * 20000
    topo = synth.topology(cfg, info)
    assert topo["n_nodes"] == (5000 + 11) // 12
    assert topo["rack_of_node"].max() == 21 and np.all(np.diff(topo["rack_of_node"].astype(int)) >= 0)
    tr = synth.truth(cfg, info)
    assert tr["slowed_rack"].sum() == 3 and tr["comm_segment"].sum() == 6
