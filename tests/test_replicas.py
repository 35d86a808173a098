"""The multi-GPU path is replicas only: whole pairs shard across ranks, no
collective touches the data, the timing reduces with MAX and the units with
SUM.  Two gloo ranks on the CPU run that logic end to end, with the oracle
standing in for each rank's matcher."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2203_02300_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pairs():
    from paper_2203_02300_gb300 import scenes
    return [scenes.plane_scene(48 + 8 * (i % 3), 32, 8, 2, seed=scenes.seed_for(3, 800 + i), drange=(1, 6))
            for i in range(6)]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.rank_env() == (rank, rank, world)
        pairs = _pairs()
        mine = {i: O.match(pairs[i].left, pairs[i].right, pairs[i].D).disp for i in replicas.shard(len(pairs), rank, world)}
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)   # results to the host, as the bench's rank 0 reports them
        units = sum(pairs[i].W * pairs[i].H * pairs[i].D for i in mine)
        total, slowest, rate = replicas.job_rate(units, 1.0 + rank, dist)
        if rank == 0:
            q.put((gathered, total, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_shard_partitions_the_items():
    for n in (0, 1, 5, 32):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in replicas.shard(n, r, world))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_reductions_are_identities():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_rate(10.0, 2.0) == (10.0, 2.0, 5.0)


def test_two_gloo_ranks_match_one_process():
    from oracle import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, total, slowest, rate = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pairs = _pairs()
    merged = {}
    for part in gathered:
        assert not set(part) & set(merged)   # disjoint shards
        merged.update(part)
    assert sorted(merged) == list(range(len(pairs)))
    for i, s in enumerate(pairs):
        assert np.array_equal(merged[i], O.match(s.left, s.right, s.D).disp)
    assert total == sum(s.W * s.H * s.D for s in pairs)
    assert slowest == 2.0 and rate == total / 2.0
