"""Multi-rank host logic on CPU: two gloo ranks, each with its own replica
seed, agree on the slowest rank's time and report whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2503_07526_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = replicas.dist_env()
        seed = replicas.replica_seed(1, r)
        t_local = 2.0 + r  # rank 1 is the slow one
        t_max = replicas.max_over_ranks(t_local, dist)
        rate = replicas.weak_scaling_rate(1000, 50, w, t_max)
        seeds = [None] * w
        dist.all_gather_object(seeds, seed)
        out.put((r, w, local, seeds, t_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_distinct_seeds():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, seeds, t_max, rate) in enumerate(res):
        assert (rank, w, local) == (r, world, r)
        assert seeds == [1, 2]
        assert t_max == 3.0  # max over ranks, not the local time
        assert rate == pytest.approx(world * 1000 * 50 / 3.0)


def test_single_process_identity():
    assert replicas.max_over_ranks(1.25) == 1.25
    assert replicas.weak_scaling_rate(10, 3, 1, 2.0) == 15.0
    with pytest.raises(ValueError):
        replicas.weak_scaling_rate(10, 3, 1, 0.0)
