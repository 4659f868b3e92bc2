"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank draws its own candidate poses over the same cloud (independent units, no
data-path collective), and the reported time is the slowest rank's."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        scene, views, st = bench.workload(rank, n_gauss=2000, n_views=4, size=32, grid=32)
        t = bench.max_over_ranks(1.0 + rank, world, "cpu")
        out[rank] = (views.world_to_cam.copy(), scene.means[:5].copy(), t)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_poses_and_take_max_time():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (p0, m0, t0), (p1, m1, t1) = res[0], res[1]
    assert not np.allclose(p0, p1)          # different candidate poses per rank
    assert np.array_equal(m0, m1)           # the same (replicated) cloud
    assert t0 == t1 == 2.0                  # max over ranks
    assert bench.shard_seed(0) != bench.shard_seed(1)
