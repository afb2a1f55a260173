"""Host logic of the z-slab domain decomposition (no GPU).

The halo-exchange plan of paper_1609_01479_gb300.slab: every halo plane of
every slab is written exactly once per exchange, from an own plane of the
neighbouring slab that holds the same global plane. Then the plan is run as
a two-rank exchange over gloo on host arrays, one slab per rank: each rank
packs the planes its transfers send, sends and receives them, and unpacks
into its halos; afterwards every halo holds the global planes it stands for.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1609_01479_gb300 import slab


@pytest.mark.parametrize("nz,nslabs,steps", [(48, 2, 1), (48, 3, 1), (48, 1, 1), (60, 3, 2), (36, 4, 1)])
def test_plan_fills_every_halo_from_the_right_plane(nz, nslabs, steps):
    m = nz // nslabs
    h = slab.halo_depth(m, steps)
    assert h >= 3 * steps and (m % 2 or (m + 2 * h) % 4 == 0)
    written = {k: np.zeros(m + 2 * h, dtype=int) for k in range(nslabs)}
    for t in slab.exchange_plan(nslabs, m, h):
        for j in range(t.nplanes):
            src_p, dst_p = t.src_z0 + j, t.dst_z0 + j
            assert h <= src_p < h + m, "a transfer reads only own planes"
            assert dst_p < h or dst_p >= h + m, "a transfer writes only halo planes"
            assert slab.local_to_global(t.src, m, h, nz, src_p) == slab.local_to_global(t.dst, m, h, nz, dst_p)
            written[t.dst][dst_p] += 1
    for k in range(nslabs):
        halo = np.r_[0:h, h + m:m + 2 * h]
        assert np.all(written[k][halo] == 1) and np.all(written[k][h:h + m] == 0)


def test_plan_refuses_slabs_thinner_than_their_halos():
    with pytest.raises(ValueError):
        slab.exchange_plan(8, 2, 4)
    with pytest.raises(ValueError):
        slab.halo_depth(0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


NZ, NY, NX, WORLD = 16, 3, 4, 2


def _global_code(gz):
    """A value per (component, global plane, y, x) that identifies them."""
    c = np.arange(38)[:, None, None]
    y = np.arange(NY)[None, :, None]
    x = np.arange(NX)[None, None, :]
    return (c * 1000 + gz) * 100 + y * 10 + x + 0.5


def _rank(rank, port, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    m = NZ // WORLD
    h = slab.halo_depth(m)
    state = np.full((38, m + 2 * h, NY, NX), -1.0)
    for p in range(h, h + m):
        state[:, p] = _global_code(slab.local_to_global(rank, m, h, NZ, p))
    plan = slab.exchange_plan(WORLD, m, h)
    # send every packed block this rank owns, then receive into the halos
    reqs = []
    for i, t in enumerate(plan):
        if t.src == rank:
            packed = torch.from_numpy(np.ascontiguousarray(state[:, t.src_z0:t.src_z0 + t.nplanes]))
            reqs.append(dist.isend(packed, dst=t.dst, tag=i))
    for i, t in enumerate(plan):
        if t.dst == rank:
            buf = torch.empty((38, t.nplanes, NY, NX), dtype=torch.float64)
            dist.recv(buf, src=t.src, tag=i)
            state[:, t.dst_z0:t.dst_z0 + t.nplanes] = buf.numpy()
    for r in reqs:
        r.wait()
    ok = all(np.array_equal(state[:, p], _global_code(slab.local_to_global(rank, m, h, NZ, p)))
             for p in range(m + 2 * h))
    out[rank] = ok
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_plan_over_gloo_two_ranks():
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(_free_port(), out), nprocs=WORLD, start_method="spawn")
        assert dict(out) == {0: True, 1: True}
