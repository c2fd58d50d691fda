"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with
its own timing; the job's time is the slowest rank's and its throughput
counts the units of every rank (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    local_ms = [120.0, 80.0][rank]
    t = bench.max_over_ranks(local_ms)
    rate = bench.job_rate(10, ws, t / 1e3)
    dist.barrier()
    q.put((r, ws, local, t, rate))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k, (r, ws, local, t, rate) in enumerate(out):
        assert (r, ws, local) == (k, 2, k)
        assert t == 120.0                       # the slowest rank's time
        assert rate == pytest.approx(2 * 10 / 0.12)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(20, 1, 0.5) == 40.0
