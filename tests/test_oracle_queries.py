"""Pins of the oracle's serving queries (slice of the tri-dimensional model and
the top-k ranks of a context) against hand-worked values and a brute-force
restatement that shares none of the oracle's loops."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import bruteforce as bf
from paper_2605_03561_b300.synth import edge


def _hand(golden_dir):
    with open(os.path.join(golden_dir, "hand_example.json")) as f:
        g = json.load(f)
    lens = [len(r["ts"]) for r in g["ranks"]]
    ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    tr = oracle.Traces(ro, np.array(sum((r["ts"] for r in g["ranks"]), []), np.uint64),
                       np.array(sum((r["ctx"] for r in g["ranks"]), []), np.uint32),
                       np.array(g["parent"], np.uint32), g["marker"])
    return tr, g


def test_slice_hand_example(golden_dir):
    tr, g = _hand(golden_dir)
    a = oracle.Analysis(tr)
    s = a.slice(2, 0, 2, 0, 3)
    # context 2: rank 0 iterations (25, 20), rank 1 iterations (30, 60); a
    # third iteration does not exist
    assert s.tolist() == [[25, 20, 0], [30, 60, 0]]
    assert a.slice(3, 0, 2, 1, 2).tolist() == [[0], [0]]  # present with 0 ns
    assert a.slice(0, 1, 2, 0, 2).tolist() == [[0, 0]]  # the root never sampled
    assert a.slice(1, 0, 2, 0, 0).shape == (2, 0)


def test_topk_hand_example(golden_dir):
    tr, g = _hand(golden_dir)
    a = oracle.Analysis(tr)
    rk, x, z = a.topk(2, 5)
    assert rk.tolist() == [1, 0] and x.tolist() == [90, 45]
    ref = g["stats_excl_ctx2"]["z"]
    assert z[0] == pytest.approx(ref[1], rel=1e-15) and z[1] == pytest.approx(ref[0], rel=1e-15)
    rk, x, z = a.topk(3, 1)  # both ranks 10 and 0 ns: rank 0 first
    assert rk.tolist() == [0] and x.tolist() == [10]


def _excl_values(dd, c):
    per = bf.exclusive(dd)
    return [bf.value(per, r, c)[0] for r in range(len(dd["rank_off"]) - 1)]


@pytest.mark.parametrize("seed", range(30))
def test_slice_bruteforce(seed):
    d = edge.case("random_small", seed)
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    a = oracle.Analysis(tr)
    dd = dict(rank_off=d["rank_off"], ts=d["ts"], ctx=d["ctx"], parent=d["parent"],
              marker=d["marker"])
    rows = bf.tensor(dd)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        c = int(rng.integers(0, tr.C))
        r0 = int(rng.integers(0, tr.R))
        r1 = int(rng.integers(r0, tr.R + 1))
        i0 = int(rng.integers(0, 4))
        i1 = int(rng.integers(i0, 8))
        got = a.slice(c, r0, r1, i0, i1)
        for r in range(r0, r1):
            for i in range(i0, i1):
                want = 0
                if i + 1 < len(rows[r]):  # rows[r][0] is the prologue
                    for cc, t, _ in rows[r][i + 1]:
                        if cc == c:
                            want = t
                assert int(got[r - r0, i - i0]) == want, (r, i, c)


def _z_exact(xs, j):
    n = len(xs)
    S1 = sum(xs)
    M = n * sum(v * v for v in xs) - S1 * S1
    if n < 2 or M == 0:
        return 0.0
    return (n * xs[j] - S1) / (n * math.sqrt(Fraction(M, n * (n - 1))))


@pytest.mark.parametrize("seed", range(30))
def test_topk_bruteforce(seed):
    d = edge.case("random_small", seed)
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    a = oracle.Analysis(tr)
    dd = dict(rank_off=d["rank_off"], ts=d["ts"], ctx=d["ctx"], parent=d["parent"],
              marker=d["marker"])
    for c in range(tr.C):
        xs = _excl_values(dd, c)
        order = sorted(range(len(xs)), key=lambda r: (-xs[r], r))
        for k in (1, 3, 100):
            rk, x, z = a.topk(c, k)
            assert rk.tolist() == order[:k]
            assert x.tolist() == [xs[r] for r in order[:k]]
            for j, r in enumerate(order[:k]):
                assert z[j] == pytest.approx(_z_exact(xs, r), rel=1e-13, abs=1e-300)


def test_topk_ties_go_to_lower_rank():
    # Four ranks, context 1 lasts 10, 30, 30, 10 ns: order 1, 2, 0, 3.
    ts, cx, ro = [], [], [0]
    for dur in (10, 30, 30, 10):
        ts += [0, dur]
        cx += [1, 0]
        ro.append(len(ts))
    tr = oracle.Traces(np.array(ro, np.uint64), np.array(ts, np.uint64),
                       np.array(cx, np.uint32), np.array([0xFFFFFFFF, 0], np.uint32), 1)
    a = oracle.Analysis(tr)
    rk, x, z = a.topk(1, 4)
    assert rk.tolist() == [1, 2, 0, 3] and x.tolist() == [30, 30, 10, 10]
    # mean 20, std (ddof 1) = sqrt(400/3): z = +-10 / sqrt(400/3) = +-sqrt(3)/2
    assert z[0] == pytest.approx(math.sqrt(3) / 2, rel=1e-15)
    assert z[3] == pytest.approx(-math.sqrt(3) / 2, rel=1e-15)


@pytest.mark.parametrize("seed", range(10))
def test_cv_terms_against_exact_means(seed):
    # cv_within = mean over ranks of each rank's CV over iterations, cv_across =
    # mean over iterations of the CV over ranks (ddof 1); recomputed from a
    # brute-force tensor with exact variances and an exactly rounded mean.
    d = edge.case("random_small", seed)
    tr = oracle.Traces(d["rank_off"], d["ts"], d["ctx"], d["parent"], d["marker"])
    a = oracle.Analysis(tr)
    dd = dict(rank_off=d["rank_off"], ts=d["ts"], ctx=d["ctx"], parent=d["parent"],
              marker=d["marker"])
    rows = bf.tensor(dd)
    ctxs = list(range(tr.C))
    per, tot = a.speedup(ctxs)
    I = tot["i_star"]
    if I == 0:
        return

    def cv(xs):
        n = len(xs)
        s = sum(xs)
        if s == 0:
            return 0.0
        var = Fraction(n * sum(x * x for x in xs) - s * s, n * (n - 1)) if n > 1 else 0
        return math.sqrt(var) / (s / n)

    def t(r, i, c):
        for cc, tt, _ in rows[r][i + 1]:
            if cc == c:
                return tt
        return 0

    for k, c in enumerate(ctxs):
        within = math.fsum(cv([t(r, i, c) for i in range(I)]) for r in range(tr.R)) / tr.R
        across = math.fsum(cv([t(r, i, c) for r in range(tr.R)]) for i in range(I)) / I
        assert per["cv_within"][k] == pytest.approx(within, rel=1e-13, abs=1e-300)
        assert per["cv_across"][k] == pytest.approx(across, rel=1e-13, abs=1e-300)
