"""The multi-GPU partition of the all-agents radius query (z slabs with halo
planes, one exchange after binning), run as two gloo ranks on the CPU: slab
ownership and halo planes (cyclic wrap, clipped non-cyclic axis), and the
union of the ranks' lists against the oracle over the whole scene.  Each
rank's query is the oracle over its local points, standing in for the
library's call on a GPU rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_cs_0608108_b300 import slabs, synth


def test_slab_plans_cover_the_planes_and_wrap():
    for gz, ranks in ((16, 2), (17, 3), (64, 8)):
        plans = [slabs.plan(gz, ranks, r, 1.4, 1.0, True) for r in range(ranks)]
        cover = np.zeros(gz, int)
        for p in plans:
            cover[p.z0:p.z1] += 1
            assert p.reach == 3
        assert np.all(cover == 1)
    p0 = slabs.plan(16, 2, 0, 1.4, 1.0, True)
    assert p0.halo_planes() == [13, 14, 15, 8, 9, 10]
    q0 = slabs.plan(16, 2, 0, 1.4, 1.0, False)
    assert q0.halo_planes() == [8, 9, 10]
    q1 = slabs.plan(16, 2, 1, 1.4, 1.0, False)
    assert q1.halo_planes() == [5, 6, 7]
    with pytest.raises(ValueError):
        slabs.plan(8, 2, 0, 3.0, 1.0, True)      # halo would wrap onto the slab
    # ownership partitions the points; a point outside a non-cyclic region
    # belongs to the slab of the nearest plane
    z = np.array([-3.5, -0.2, 0.3, 7.9, 8.0, 15.99, 16.2, 30.0], np.float32)
    planes = slabs.planes_of(z, 0.0, 1.0)
    own = np.stack([slabs.owned_mask(planes, slabs.plan(16, 2, r, 1.4, 1.0, False)) for r in range(2)])
    assert np.all(own.sum(0) == 1)
    assert own[0].tolist() == [True, True, True, True, False, False, False, False]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, mask, out_q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pos = synth.uniform_points(6000, 900 + mask)
        if not (mask >> 2) & 1:
            pos[:12, 2] = np.float32(-0.05)     # outside below the region
            pos[12:20, 2] = np.float32(1.04)    # and above it
        scene = synth.Scene(pos, (0, 0, 0), 1 / 16, (4, 4, 4), mask, 1.5 / 16)
        plans = [slabs.plan(16, world, r, scene.r, scene.cell_size, bool((mask >> 2) & 1))
                 for r in range(world)]
        # each rank starts with an interleaved shard of the input
        mine = np.arange(rank, scene.n, world)
        ids, lpos = slabs.exchange(mine, scene.pos[mine], plans, 0.0, scene.cell_size)

        def query(local, q):
            return oracle.radius(local, local[q], scene.box, mask, scene.r, q, threads=1)

        owned, off, nbr = slabs.rank_query(ids, lpos, plans[rank], 0.0, scene.cell_size, query)
        parts = [None] * world
        dist.all_gather_object(parts, (owned, off, nbr))
        if rank == 0:
            off_o, ids_o = oracle.radius(scene.pos, scene.pos, scene.box, mask, scene.r, np.arange(scene.n),
                                         threads=1)
            seen = np.zeros(scene.n, int)
            ok = True
            for own, o, nb in parts:
                seen[own] += 1
                for t, q in enumerate(own):
                    ok &= np.array_equal(nb[o[t]:o[t + 1]], ids_o[off_o[q]:off_o[q + 1]])
            out_q.put(bool(ok and np.all(seen == 1)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mask", [7, 3])
def test_two_gloo_ranks_union_equals_oracle(mask):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mask, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=10) is True
