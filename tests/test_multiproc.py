"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Each rank solves an independent instance (no collective on the data path);
the only collective is the max over ranks of the timed duration.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    inst = bench.instance_for_rank(rank)
    img, mask, _ = synth.workload(1, instance=inst)
    slowest = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
    out[rank] = (inst, float(img.sum()), int(mask.sum()), slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_solve_distinct_instances_and_agree_on_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] != res[1][0]
    assert res[0][1] != res[1][1]           # different images
    assert res[0][3] == res[1][3] == 11.0   # max over ranks


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
