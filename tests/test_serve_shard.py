"""Serving across GPUs shards by scene with no collective: on two gloo ranks (CPU)
each rank's requests are exactly those for its scenes, the two shards are
disjoint, and together they are the whole stream in arrival order.
"""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2602_00395_gb300 import serve as SV
    from paper_2602_00395_gb300 import synth as S
    stream = S.request_stream(300, 500.0, 16, 8, seed=99)
    mine = SV.shard_requests(stream, rank, world)
    scenes = SV.scene_shard(16, rank, world)
    got = [None] * world
    dist.all_gather_object(got, (mine, scenes))
    if rank == 0:
        out.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_the_stream_by_scene():
    from paper_2602_00395_gb300 import synth as S
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29611
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (req0, sc0), (req1, sc1) = got
    assert set(sc0).isdisjoint(sc1) and sorted(sc0 + sc1) == list(range(16))
    assert all(r[2] in sc0 for r in req0) and all(r[2] in sc1 for r in req1)
    full = S.request_stream(300, 500.0, 16, 8, seed=99)
    assert sorted(req0 + req1) == sorted(full) and len(req0) + len(req1) == len(full)
    assert req0 == [r for r in full if r[2] in sc0]
