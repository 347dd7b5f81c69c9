"""The benchmark's multi-rank reduction (replicas on N GPUs) on CPU with gloo, world size 2."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r measured (10 + r) ms for its replica; everyone must agree on the max
    t = bench.max_over_ranks(10.0 + rank, torch.device("cpu"))
    q.put((rank, t, bench.whole_job_value(bytes_per_rank=1e9, ms=t, world=world)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    # value = bytes of all replicas / slowest replica's time, in GB/s
    assert res[0][2] == pytest.approx(2 * 1e9 / 11e-3 / 1e9)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_value(bytes_per_rank=2e9, ms=1.0, world=1) == pytest.approx(2000.0)
