"""The multi-GPU path's host logic on CPU ranks (gloo, world size 2): the step
shards cover the job exactly once, and the sum-reduce of per-rank partial
images (each rank imaging its own steps with the oracle) equals the
single-process image, since the images are a plain sum over steps
(Algorithm 1); the timing reduction takes the slowest rank."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2310_09200_b300.distributed import shard_steps


@pytest.mark.parametrize("n_t,world", [(10, 2), (7, 3), (3, 4), (100, 8)])
def test_shards_cover_every_step_once(n_t, world):
    shards = [shard_steps(n_t, r, world) for r in range(world)]
    steps = [t for s in shards for t in s]
    assert steps == list(range(n_t))
    sizes = [len(s) for s in shards]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2310_09200_b300 import inputs
    from paper_2310_09200_b300.distributed import max_over_ranks, sum_images

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = inputs.make_config(0, n_t=5, n_side=12)
        b = np.array([[50.0, np.inf], [-np.inf, 50.0]])
        img = np.zeros((inp.n_pix, 2), order="F")
        for t in shard_steps(inp.n_t, rank, world):
            img, *_ = oracle.ss_step(inp.pix, inp.wl, b, inp.n_eig, inp.st_xyz[t], inp.vis[t], img=img)
        tot = sum_images(torch.from_numpy(np.ascontiguousarray(img)))
        slowest = max_over_ranks(1.0 + rank)
        if rank == 0:
            q.put((tot.numpy(), slowest))
    finally:
        dist.destroy_process_group()


def test_sharded_steps_sum_to_the_single_process_image():
    import oracle
    from paper_2310_09200_b300 import inputs

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, slowest = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    inp = inputs.make_config(0, n_t=5, n_side=12)
    b = np.array([[50.0, np.inf], [-np.inf, 50.0]])
    want = None
    for p_, V in zip(inp.st_xyz, inp.vis):
        want, *_ = oracle.ss_step(inp.pix, inp.wl, b, inp.n_eig, p_, V, img=want)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert slowest == 2.0
