"""Sharding of a batch over ranks: partition properties, and the multi-process path with two
gloo ranks on the CPU (each rank takes its share, the time reduction is a max over ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_2208_06588_gb300 import shard
from paper_2208_06588_gb300 import workloads as W


def offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


@pytest.mark.parametrize("B,world", [(1, 1), (7, 2), (64, 3), (4096, 8), (3, 8), (100, 7)])
def test_partition_covers_every_instance_once(B, world):
    rng = np.random.default_rng(B * 31 + world)
    off = offsets(rng.integers(256, 16385, size=B))
    ranges = [shard.partition(off, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == B
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0 and a0 <= a1
    # balance: each rank's cells are within one largest instance of the even share
    big = int(np.diff(off).max())
    for a, b in ranges:
        cells = int(off[b] - off[a])
        assert abs(cells - off[-1] / world) <= big + 1


def test_partition_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.partition(offsets([5, 5]), 2, 2)


def test_subset_matches_instances():
    bt = W.many_basins(B=9, n_min=16, n_max=40, seed=5)
    sb = shard.subset(bt, 3, 7)
    assert sb.B == 4 and sb.off[0] == 0
    for k in range(4):
        a, b = sb.instance(k), bt.instance(3 + k)
        for f in ("x", "h", "hu", "b", "E", "profile"):
            np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
        assert a.cfl == b.cfl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bt = W.many_basins(B=37, n_min=16, n_max=64, seed=11)
        i0, i1 = shard.partition(bt.off, world, rank)
        mine = shard.subset(bt, i0, i1)
        shard.barrier()
        t_max = shard.max_over_ranks(1.0 + rank)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([i0, i1, int(mine.off[-1]), t_max, float(mine.E.sum())]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_batch(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    bt = W.many_basins(B=37, n_min=16, n_max=64, seed=11)
    assert res[0][0] == 0 and res[0][1] == res[1][0] and res[1][1] == bt.B
    assert res[0][2] + res[1][2] == bt.off[-1]
    assert all(r[3] == float(world) for r in res)  # max over ranks of 1 + rank
    assert np.isclose(res[0][4] + res[1][4], bt.E.sum(), rtol=1e-13)
