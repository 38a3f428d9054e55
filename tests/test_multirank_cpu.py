"""The N > 1 path on the CPU: two gloo ranks each protect their shard of a batch (with the CPU
oracle standing in for the GPU kernels), and the union of their outputs equals the
single-process result.  Also checks the slowest-rank timing reduction."""
import os
import socket

import numpy as np
import pytest

from paper_1512_02951_gb300 import shard, synth


def test_shard_is_a_balanced_partition():
    costs = [5, 1, 9, 3, 3, 7, 2, 8]
    parts = shard.shard(costs, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert shard.shard(costs, 3) == parts                      # deterministic
    assert shard.shard([], 2) == [[], []]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _specs():
    sizes = [(64, 48), (24, 16), (8, 8), (40, 64), (16, 32)]
    return [(w, h, synth.make_image(w, h, 90 + i), synth.make_key(60 + i), synth.make_iv(70 + i))
            for i, (w, h) in enumerate(sizes)]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from oracle import fds as ofds

    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = _specs()
    mine = shard.shard([w * h for w, h, *_ in specs], world)[rank]
    out = {i: ofds.protect(specs[i][2], specs[i][3], specs[i][4], 5) for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, {i: (p.tobytes(), c) for i, (p, c) in out.items()})
    slowest = shard.max_over_ranks(float(rank + 1))
    if rank == 0:
        q.put((gathered, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_the_batch_exactly_once():
    mp = pytest.importorskip("torch.multiprocessing")
    from oracle import fds as ofds

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, slowest = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert slowest == 2.0
    merged = {}
    for part in gathered:
        assert not set(part) & set(merged)                      # no image done twice
        merged.update(part)
    specs = _specs()
    assert sorted(merged) == list(range(len(specs)))
    for i, (w, h, img, key, iv) in enumerate(specs):
        pub, priv = ofds.protect(img, key, iv, 5)
        assert merged[i][0] == pub.tobytes() and merged[i][1] == priv
