"""Replica bookkeeping of `bench.py --gpus N` on world-size-2 gloo processes
(CPU): the reported time is the slowest rank's, the count is the sum."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2306_09855_gb300 import replicas
    replicas.init("gloo")
    assert replicas.world() == (rank, world, rank)
    replicas.barrier()
    ms, n = replicas.reduce_timing(100.0 + 25.0 * rank, 1000 * (rank + 1))
    with open(out_path + ".%d" % rank, "w") as f:
        f.write("%r %r\n" % (ms, n))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_total_count(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for rank in range(2):
        ms, n = open(out + ".%d" % rank).read().split()
        assert float(ms) == 125.0 and float(n) == 3000.0


def test_single_process_is_identity():
    from paper_2306_09855_gb300 import replicas
    assert replicas.reduce_timing(12.5, 7) == (12.5, 7.0)
