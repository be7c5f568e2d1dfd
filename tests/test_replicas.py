"""The N > 1 path on CPU: world_size-2 gloo ranks (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2509_23180_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = replicas.seeds_for_rank(rank, world, 10)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    job = replicas.job_time(local_ms, world)
    rate = replicas.aggregate_rate(len(seeds), world, job)
    q.put((rank, seeds, job, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_seeds_and_take_the_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds0, seeds1 = out[0][1], out[1][1]
    assert set(seeds0).isdisjoint(seeds1) and sorted(seeds0 + seeds1) == list(range(20))
    assert out[0][2] == out[1][2] == 150.0                       # max over ranks
    assert abs(out[0][3] - 20 / 0.150) < 1e-9                    # whole-job rate


def test_single_process_is_the_identity():
    assert replicas.job_time(12.5, 1) == 12.5
    assert replicas.seeds_for_rank(0, 1, 3) == [0, 1, 2]
    with pytest.raises(ValueError):
        replicas.seeds_for_rank(2, 2, 3)
