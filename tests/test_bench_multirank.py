"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2): the
timed value uses the maximum time over ranks and the sum of their work; the
reference arm runs on rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    q.put((rank, bench.reduce_max_sum(10.0 + rank, 5.0 * (rank + 1), "cpu")))
    dist.destroy_process_group()


def test_reduce_max_sum_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == (11.0, 15.0)


def test_reduce_is_identity_without_process_group():
    import bench
    assert bench.reduce_max_sum(3.5, 7, "cpu") == (3.5, 7.0)


def test_reference_arm_exits_on_nonzero_ranks(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup = 2, 1, 0

    assert bench.run_reference(A()) == 0
