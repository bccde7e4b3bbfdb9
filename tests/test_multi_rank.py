"""The multi-GPU host logic on CPU with world_size-2 gloo groups: query-row
sharding (row ranges and the all-gather that assembles kappa) and the
benchmark's whole-job timing of replicas (max over ranks)."""
import pytest

from paper_2606_06329_gb300 import shard

import dist_helpers as H


@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("n", [0, 1, 7, 100, 1_000_001])
def test_row_ranges_tile_the_rows(world, n):
    ranges = [shard.row_range(r, world, n) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
    sizes = [e - b for b, e in ranges]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.row_range(world, world, n)


def test_gather_rows_assembles_uneven_blocks():
    res = H.run_group(H.gather_case, world=2)
    expect = [[float(i), -float(i)] for i in range(11)]
    assert res[0] == expect and res[1] == expect


def test_replica_timing_takes_the_slowest_rank():
    res = H.run_group(H.timing_case, world=2)
    for slowest, value in res:
        assert slowest == 150.0
        assert value == pytest.approx(1000 * 2 * 3 / 0.150)


def test_sharded_curvature_gathers_every_row():
    res = H.run_group(H.sharded_case, world=2)
    expect = [0.5 * i + 1.0 for i in range(9)]
    assert res[0] == expect and res[1] == expect
