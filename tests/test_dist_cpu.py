"""The multi-rank path of the decoder (frame sharding, max-over-ranks timing, counter
sums) with world_size = 2 on the gloo backend, on CPU."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2412_20828_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = D.env_ranks()
        base = D.frame_base(r)
        # each rank's frames: same recipe, disjoint indices
        aut = O.draw_autos(63, 3, 5, base, 4)
        t = D.max_over_ranks(1.0 + r)
        ctr = torch.tensor([10 * (r + 1), r], dtype=torch.int64)
        D.sum_over_ranks(ctr)
        q.put((r, w, lr, base, aut.tolist(), t, ctr.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, b0, a0, t0, c0), (r1, w1, l1, b1, a1, t1, c1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert b1 - b0 == D.FRAMES_PER_RANK_SPAN
    # rank 1's frames equal a single-process draw at the same indices
    assert a1 == O.draw_autos(63, 3, 5, b1, 4).tolist()
    assert a0 != a1
    assert t0 == t1 == 2.0  # the slowest rank's time
    assert c0 == c1 == [30, 1]  # summed counters
    assert D.job_throughput(1000, 2, 2.0) == 1000.0


def test_single_process_defaults():
    assert D.env_ranks()[1] >= 1
    assert D.max_over_ranks(3.5) == 3.5
