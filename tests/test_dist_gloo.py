"""The multi-rank path on CPU (gloo, world size 2): root shards partition
the render, the summed shard images equal the single-process image, and the
timing reduction takes the maximum."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2406_16302_gb300.dist import shard_roots

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shards_partition_the_roots():
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            ranges = [shard_roots(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0 and a0 <= a1
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_roots(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2406_16302_gb300 import scenes
    from paper_2406_16302_gb300.dist import max_over_ranks, shard_roots, sum_images
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scene, edit = scenes.cfg1_box_sphere(width=8, height=8, max_depth=4)
    o = oracle.Oracle(scene, edit)
    spp = 4
    r0, r1 = shard_roots(o.n_roots(spp), rank, world)
    img = torch.from_numpy(o.render_residual(spp, 9, r0, r1))
    sum_images(img)
    t = max_over_ranks(10.0 + rank)
    dist.barrier()
    if rank == 0:
        q.put((img.numpy(), t))
    dist.destroy_process_group()


def test_two_rank_render_equals_single_process():
    import oracle
    from paper_2406_16302_gb300 import scenes
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    img, t = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    scene, edit = scenes.cfg1_box_sphere(width=8, height=8, max_depth=4)
    full = oracle.Oracle(scene, edit).render_residual(4, 9)
    assert np.allclose(img, full, rtol=1e-12, atol=1e-15)
    assert t == 11.0
