"""The sharded form's exchange (include/ta.h, "sharded form") on CPU with two
gloo ranks: each rank packs its shard's statistics partials in the stated
layout -- per context present, S1, S2 as four 32-bit limbs in 64-bit words
(SUM), min with absent ranks counting 0 (MIN), max (MAX), and the argmax
candidate (MIN) -- and all_reduce over int64 views merges them.  The merge
must give the whole job's values exactly, with values near 2^46 so that the
sums of squares carry between limbs."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

R, C = 96, 7  # 96 ranks, 7 contexts; shard 0 = ranks [0, 40), shard 1 = [40, 96)
BOUNDS = (0, 40, 96)
NONE = 0xFFFFFFFF


def _values():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 1 << 46, size=(R, C), dtype=np.uint64)
    absent = rng.random((R, C)) < 0.2
    x[absent] = 0
    x[:, 3] = 0  # a context no rank holds
    x[5, 2] = x[77, 2] = np.uint64((1 << 46) + 5)  # a tie for the max across shards
    return x, ~absent


def _pack(x, present, r0, r1):
    """Partials of ranks [r0, r1) in the exchange layout (int64 words)."""
    sums, mins, maxs, cand = [], [], [], []
    for c in range(C):
        col = [int(v) for v in x[r0:r1, c]]
        pres = int(present[r0:r1, c].sum()) if c != 3 else 0
        s2 = sum(v * v for v in col)
        sums += [pres, sum(col)] + [(s2 >> (32 * l)) & 0xFFFFFFFF for l in range(4)]
        mins.append(min(col) if pres == r1 - r0 else 0)
        maxs.append(max(col))
        cand.append(r0 + col.index(max(col)))
    return [torch.tensor(np.array(a, dtype=np.uint64).view(np.int64)) for a in
            (sums, mins, maxs, cand)]


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        x, present = _values()
        sums, mins, maxs, cand = _pack(x, present, BOUNDS[rank], BOUNDS[rank + 1])
        dist.all_reduce(sums, op=dist.ReduceOp.SUM)
        dist.all_reduce(mins, op=dist.ReduceOp.MIN)
        dist.all_reduce(maxs, op=dist.ReduceOp.MAX)
        # the candidate counts only where the shard holds the job's max
        mine = torch.where(torch.tensor([int(x[BOUNDS[rank]:BOUNDS[rank + 1], c].max())
                                         for c in range(C)]) == maxs, cand,
                           torch.full_like(cand, NONE))
        dist.all_reduce(mine, op=dist.ReduceOp.MIN)
        out[rank] = [t.numpy().view(np.uint64).tolist() for t in (sums, mins, maxs, mine)]
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_shards_merge_to_the_whole_job():
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(_free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1]
    sums, mins, maxs, argmax = out[0]
    x, present = _values()
    for c in range(C):
        col = [int(v) for v in x[:, c]]
        q = sums[6 * c + 2: 6 * c + 6]
        s2 = sum(int(q[l]) << (32 * l) for l in range(4))  # merged limbs carry here
        assert s2 == sum(v * v for v in col), c
        assert sums[6 * c] == (int(present[:, c].sum()) if c != 3 else 0)
        assert sums[6 * c + 1] == sum(col)
        assert maxs[c] == max(col)
        assert mins[c] == (min(col) if (c != 3 and present[:, c].all()) else 0)
        assert argmax[c] == col.index(max(col))  # lowest rank on ties (ranks 5 and 77)
    assert max(int(v) for v in sums[2::6]) > 0xFFFFFFFF  # a low limb did carry
