"""The autotuner's host logic (coordinate descent, size buckets), on the CPU
with synthetic timings; its GPU use is in tests/test_gpu_batch.py."""
import pytest

from paper_2410_08946_gb300 import autotune


def test_descend_finds_the_minimum_of_a_separable_cost():
    calls = []

    def cost(p):
        calls.append(dict(p))
        return (p["jumps_per_round"] - 8) ** 2 + 10 * (p["levels_ctas_per_sm"] - 2) ** 2 + 1.0

    best, ms, table = autotune.descend(cost, space=autotune.SPACE_FIXED_SHAPE)
    assert best == {"tile_shape": 0, "jumps_per_round": 8, "levels_ctas_per_sm": 2}
    assert ms == 1.0
    # one timing per candidate of each parameter, the second with the first fixed at its best
    n = sum(len(v) for v in autotune.SPACE_FIXED_SHAPE.values())
    assert len(table) == len(calls) == n
    assert all(c["jumps_per_round"] == 8 for c in calls[len(autotune.SPACE["jumps_per_round"]):])


def test_descend_over_tile_shapes():
    """The tile shape is the first coordinate; the later ones are timed on the
    shape chosen for it."""
    calls = []

    def cost(p):
        calls.append(dict(p))
        return {0: 5.0, 1: 4.0, 2: 3.0, 3: 6.0}[p["tile_shape"]] + abs(p["jumps_per_round"] - 12) * 0.1

    best, ms, table = autotune.descend(cost)
    assert best["tile_shape"] == 2 and best["jumps_per_round"] == 12
    assert abs(ms - 3.0) < 1e-12
    assert all(c["tile_shape"] == 2 for c in calls[len(autotune.SPACE["tile_shape"]):])
    assert set(autotune.SHAPES) == set(autotune.SPACE["tile_shape"])


def test_descend_ties_keep_the_first_candidate():
    best, _, _ = autotune.descend(lambda p: 5.0, space={"jumps_per_round": [4, 6, 8]}, start={})
    assert best["jumps_per_round"] == 4


def test_size_bucket():
    assert autotune.size_bucket(1) == "4^0"
    assert autotune.size_bucket(3) == "4^0" and autotune.size_bucket(4) == "4^1"
    assert autotune.size_bucket(256 * 256) == "4^8"
    assert autotune.size_bucket(928 ** 3) == autotune.size_bucket(900 ** 3)
