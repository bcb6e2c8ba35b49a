"""Multi-rank logic of bench.py on CPU (gloo, world size 2): every rank gets
its own acquisition seed, the step time is the maximum over ranks, and the
whole-job rate counts all ranks' histories."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = bench._dist()
        my_ms = 100.0 + 50.0 * rank
        ms = bench._maxreduce(my_ms, ws)
        bench._barrier(ws)
        q.put((r, bench.shard_seed(1, r), ms, bench.whole_job_rate(ws, 1000, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_timing_and_split_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [o[1] for o in out]
    assert len(set(seeds)) == world                       # independent acquisitions
    assert all(o[2] == pytest.approx(150.0) for o in out)  # slowest rank's time
    assert all(o[3] == pytest.approx(2 * 1000 / 0.150) for o in out)
