"""The allocation-free statistics entry point (ta_context_stats_noalloc).

Some callers cannot allocate device memory when they call the library -- for
example a host runtime that owns all device memory and hands libraries only
its own buffers, or a service held to a fixed device-memory budget.  This
entry point takes device inputs and outputs and keeps its temporaries in a
fixed array inside the library.  These tests call it through the C ABI twice
in a row (the array keeps the previous call's contents) and check it against
the allocating ta_context_stats, integers bit for bit and FP64 within 1e-12
relative.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2605_03561_b300 as ta
from paper_2605_03561_b300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(e, ranks=None, tau=(2, 1), cap=4096, n_ctx=None):
    import torch
    v = ta.CsrView()
    ta._check(ta.lib().ta_csr_get_view(e.h, ta.EXCLUSIVE, C.byref(v)))
    n_ctx = e.C if n_ctx is None else n_ctx
    stats = torch.zeros(n_ctx * C.sizeof(ta.CtxStats), dtype=torch.uint8, device="cuda")
    outl = torch.zeros(max(cap, 1) * C.sizeof(ta.Outlier), dtype=torch.uint8, device="cuda")
    rk = None if ranks is None else torch.as_tensor(np.asarray(ranks, np.uint32)).cuda()
    n = C.c_uint64(0)
    s = ta.lib().ta_context_stats_noalloc(
        e.ctx.stream.cuda_stream, v.off, v.ctx, v.time, e.R, n_ctx,
        None if rk is None else rk.data_ptr(), 0 if ranks is None else len(ranks),
        tau[0], tau[1], stats.data_ptr(), outl.data_ptr(), cap, C.byref(n))
    if s != ta.OK:
        return s, None, None
    st = (ta.CtxStats * n_ctx).from_buffer_copy(stats.cpu().numpy().tobytes())
    ol = (ta.Outlier * max(cap, 1)).from_buffer_copy(outl.cpu().numpy().tobytes())
    k = int(n.value)
    stats_d = {f: np.array([getattr(x, f) for x in st]) for f, _ in ta.CtxStats._fields_
               if f != "reserved"}
    out = dict(ctx=np.array([o.ctx for o in ol[:k]], np.uint32),
               rank=np.array([o.rank for o in ol[:k]], np.uint32),
               z=np.array([o.z for o in ol[:k]], np.float64))
    return s, stats_d, out


def _check_equal(ref_stats, ref_out, got_stats, got_out):
    for k in ("n", "present", "argmax", "min", "max", "s1", "s2_lo", "s2_hi"):
        assert np.array_equal(got_stats[k], ref_stats[k]), k
    for k in ("mean", "std", "cv", "balance"):
        np.testing.assert_allclose(got_stats[k], ref_stats[k], rtol=1e-12, atol=0)
    assert np.array_equal(got_out["ctx"], ref_out["ctx"])
    assert np.array_equal(got_out["rank"], ref_out["rank"])
    np.testing.assert_allclose(got_out["z"], ref_out["z"], rtol=1e-12, atol=0)


@pytest.fixture(scope="module")
def experiment():
    cfg = synth.preset(1, seed=21, n_ranks=48)
    g = synth.generate(cfg)
    ctx = ta.Context(0)
    e = ctx.load(g["rank_off"], g["ts"], g["ctx"], g["parent"], g["marker"])
    return ctx, e


def test_noalloc_matches_allocating_call_twice(experiment):
    ctx, e = experiment
    ref_stats, ref_out, ref_n, _ = e.stats(ta.EXCLUSIVE, tau=(2, 1))
    assert ref_n > 0
    for _ in range(2):  # the second call starts from the first call's leftovers
        s, got_stats, got_out = _noalloc(e, tau=(2, 1))
        assert s == ta.OK, ta.lib().ta_last_error_message()
        _check_equal(ref_stats, ref_out, got_stats, got_out)


def test_noalloc_rank_subset_twice(experiment):
    ctx, e = experiment
    ranks = np.arange(3, 48, 2, dtype=np.uint32)
    ref_stats, ref_out, _, _ = e.stats(ta.EXCLUSIVE, ranks=ranks, tau=(1, 1))
    for _ in range(2):
        s, got_stats, got_out = _noalloc(e, ranks=ranks, tau=(1, 1))
        assert s == ta.OK, ta.lib().ta_last_error_message()
        _check_equal(ref_stats, ref_out, got_stats, got_out)


@pytest.fixture(scope="module")
def many_outliers():
    # 256 ranks and a low threshold: thousands of outliers, more than the
    # one-block sort holds, so the padded multi-block sort runs
    cfg = synth.preset(1, seed=22, n_ranks=256)
    g = synth.generate(cfg)
    ctx = ta.Context(0)
    e = ctx.load(g["rank_off"], g["ts"], g["ctx"], g["parent"], g["marker"])
    return ctx, e


def test_noalloc_many_outliers_twice(many_outliers):
    ctx, e = many_outliers
    ref_stats, ref_out, ref_n, _ = e.stats(ta.EXCLUSIVE, tau=(1, 10))
    assert ref_n > 4096
    for _ in range(2):
        s, got_stats, got_out = _noalloc(e, tau=(1, 10), cap=1 << 16)
        assert s == ta.OK, ta.lib().ta_last_error_message()
        _check_equal(ref_stats, ref_out, got_stats, got_out)


def test_noalloc_capacity_error_reports_full_count_twice(many_outliers):
    import torch
    ctx, e = many_outliers
    _, _, ref_n, _ = e.stats(ta.EXCLUSIVE, tau=(1, 10))
    v = ta.CsrView()
    ta._check(ta.lib().ta_csr_get_view(e.h, ta.EXCLUSIVE, C.byref(v)))
    stats = torch.zeros(e.C * C.sizeof(ta.CtxStats), dtype=torch.uint8, device="cuda")
    outl = torch.zeros(100 * C.sizeof(ta.Outlier), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        n = C.c_uint64(0)
        s = ta.lib().ta_context_stats_noalloc(
            e.ctx.stream.cuda_stream, v.off, v.ctx, v.time, e.R, e.C, None, 0, 1, 10,
            stats.data_ptr(), outl.data_ptr(), 100, C.byref(n))
        assert s == ta.CAPACITY
        assert int(n.value) == ref_n


def test_noalloc_rejects_context_ids_beyond_n_ctx(experiment):
    ctx, e = experiment
    ref_stats, ref_out, _, _ = e.stats(ta.EXCLUSIVE, tau=(2, 1))
    s, got_stats, got_out = _noalloc(e, tau=(2, 1))  # leaves a full slot map behind
    assert s == ta.OK
    x = e.csr(ta.EXCLUSIVE)
    small = int(x["ctx"].max())  # the largest id used is then out of range
    s, _, _ = _noalloc(e, tau=(2, 1), n_ctx=small)
    assert s == ta.BAD_CTX, ta.lib().ta_last_error_message()
    s, got_stats, got_out = _noalloc(e, tau=(2, 1))
    assert s == ta.OK
    _check_equal(ref_stats, ref_out, got_stats, got_out)


def test_noalloc_rejects_sizes_beyond_its_array(experiment):
    ctx, e = experiment
    s, _, _ = _noalloc(e, cap=(1 << 16) + 1)
    assert s == ta.INVALID_ARG
    assert b"fixed maximum" in ta.lib().ta_last_error_message()
    s, _, _ = _noalloc(e, n_ctx=(1 << 16) + 1)
    assert s == ta.INVALID_ARG
