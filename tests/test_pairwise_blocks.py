"""The identity the two-phase pairwise sum of the CV terms rests on.

cv_within sums its per-rank terms level by level: element i of the next
level is v[2i] + v[2i+1], and an odd last element moves up unchanged.  The
CUDA path first reduces blocks of 2^11 terms, each with the same rule, and
then reduces the block values.  Element i of level l is that rule applied to
the terms [i 2^l, min((i + 1) 2^l, n)) alone, so both orders perform the same
additions.  These tests check that claim bit for bit in plain Python floats,
for sizes around the block edges and for smaller blocks that give many
levels of each phase."""
import random

import pytest


def levels(v):
    v = list(v)
    if not v:
        return 0.0
    while len(v) > 1:
        nxt = [v[2 * i] + v[2 * i + 1] for i in range(len(v) // 2)]
        if len(v) % 2:
            nxt.append(v[-1])
        v = nxt
    return v[0]


def two_phase(v, block):
    blocks = [levels(v[b:b + block]) for b in range(0, len(v), block)]
    return levels(blocks)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 9, 2047, 2048, 2049, 4096, 5000, 6145])
@pytest.mark.parametrize("block", [2, 8, 2048])
def test_two_phase_equals_level_by_level(n, block):
    rng = random.Random(n * 31 + block)
    # magnitudes over many binades, so that the order of additions shows
    v = [rng.uniform(0.0, 1.0) * 10.0 ** rng.randint(-8, 8) for _ in range(n)]
    assert two_phase(v, block) == levels(v)


def test_block_boundary_changes_the_result_when_not_a_power_of_two():
    # Blocks of 3 terms do not follow the levels: the identity needs
    # power-of-two blocks, and these values show the difference in the last
    # place (so the tests above would catch a block size that is not one).
    e = 2.0 ** -53
    v = [e, 1.0, 0.5, 3e-16, 1e-16, e, 1.0]
    assert two_phase(v, 4) == levels(v) == two_phase(v, 2)
    assert two_phase(v, 3) != levels(v)
