"""The multi-GPU launch of bench.py runs one independent lattice per rank
(replicas; the step has no collective). Its only cross-rank operations are a
barrier around the timed region and the maximum of the per-rank times; both
are checked here with two gloo ranks on the host."""

import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    out[rank] = bench.max_over_ranks(world, 10.0 + rank)
    bench.barrier(world)
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        assert dict(out) == {0: 11.0, 1: 11.0}
