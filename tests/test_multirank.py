"""The replica path of the benchmark on two CPU ranks (gloo, 127.0.0.1): every rank
draws its own seeded system of the same workload, and the job's time is the slowest
rank's (max over ranks after a barrier)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg, sysd = bench.make_inputs("C1", seed_offset=rank)
        dist.barrier()
        t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        out[rank] = (t, float(np.abs(sysd["H0"]).sum()), sysd["H0"].shape)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_and_max_time():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0            # every rank reports the slowest time
    assert res[0][2] == res[1][2]                    # same workload shapes
    assert res[0][1] != res[1][1]                    # independently seeded systems


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, "cpu") == 3.25
