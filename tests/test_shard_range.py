"""motif_shard_range on the host (no device work): the split of the candidate space [0, total)
into per-rank contiguous ranges (the per-worker first/last l-mer index of Sec. IV.A).

Equal weights give boundary r = floor(total * r / world) exactly, up to totals of 2^64 - 1;
given weights give contiguous ranges that cover [0, total) with each rank's share within one
code per 2^40 of the exact proportion; bad arguments are MOTIF_ERR_ARG.
"""
import math

import pytest

import paper_1403_1313_gb300 as m

TOTALS = [0, 1, 7, 4 ** 9, 4 ** 15, 4 ** 31, 2 ** 63 + 12345, 2 ** 64 - 1]


@pytest.mark.parametrize("total", TOTALS)
@pytest.mark.parametrize("world", [1, 2, 3, 7, 8, 152])
def test_equal_weights_exact_boundaries(total, world):
    prev = 0
    for r in range(world):
        lo, hi = m.motif_shard_range(total, r, world)
        assert lo == total * r // world
        assert hi == total * (r + 1) // world
        assert lo == prev
        prev = hi
    assert prev == total


@pytest.mark.parametrize("total", TOTALS)
@pytest.mark.parametrize("weights", [[1, 2, 3], [0, 1, 0], [0.1] * 5, [5, 0, 0, 1e-9],
                                     [1e6, 1, 1e-3, 7]])
def test_weighted_ranges_cover_in_order(total, weights):
    world = len(weights)
    s = sum(weights)
    prev = 0
    acc = 0.0
    for r in range(world):
        lo, hi = m.motif_shard_range(total, r, world, weights)
        assert lo == prev and lo <= hi <= total
        acc += weights[r]
        if r + 1 < world:  # the boundary follows the cumulative share
            assert abs(hi - total * (acc / s)) <= max(2.0, total * 2.0 ** -40)
        if weights[r] == 0:
            assert hi == lo
        prev = hi
    assert prev == total


@pytest.mark.parametrize("args", [
    (100, 0, 0, None),            # no ranks
    (100, 2, 2, None),            # rank out of range
    (100, -1, 2, None),
    (100, 0, 2, [1.0, -1.0]),     # negative weight
    (100, 0, 2, [1.0, math.nan]),
    (100, 0, 2, [0.0, 0.0]),      # nothing to split by
])
def test_bad_arguments(args):
    total, rank, world, weights = args
    with pytest.raises(m.MotifError) as e:
        if world == 0:
            m.motif_shard_range(total, rank, 0, None)
        else:
            m.motif_shard_range(total, rank, world, weights)
    assert e.value.status == m.ERR_ARG


def test_rank_range_uses_whole_tiles():
    from paper_1403_1313_gb300.shard import TILE, rank_range
    for total, world in ((4 ** 15, 3), (4 ** 15, 8), (4 ** 9, 4), (4 ** 17, 7)):
        bounds = [rank_range(total, r, world) for r in range(world)]
        assert bounds[0][0] == 0 and bounds[-1][1] == total
        assert all(a[1] == b[0] for a, b in zip(bounds, bounds[1:]))
        assert all(lo % TILE == 0 and hi % TILE == 0 for lo, hi in bounds)
        sizes = [hi - lo for lo, hi in bounds]
        assert max(sizes) - min(sizes) <= TILE
    # fewer tiles than ranks: the candidates split evenly
    bounds = [rank_range(4 ** 8, r, 3) for r in range(3)]
    assert bounds[-1][1] == 4 ** 8 and all(a[1] == b[0] for a, b in zip(bounds, bounds[1:]))
