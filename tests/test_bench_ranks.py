"""Multi-rank host logic of bench.py on CPU: two gloo ranks (the GPU runs use one
process per GPU with NCCL; the reduction and the aggregate formula are the same)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) ms for the step loop and (10 - r) ms per kernel launch
    got = bench.max_over_ranks([rank + 1.0, 10.0 - rank], "cpu", dist)
    value = bench.aggregate_mlups(world, 1000, 50, got[0])
    out.put((rank, got, value))
    dist.barrier()
    dist.destroy_process_group()


def test_timing_is_max_over_ranks_and_value_is_whole_job():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [2.0, 10.0]
        # 2 replicas x 1000 nodes x 50 steps in 2 ms
        assert value == pytest.approx(2 * 1000 * 50 / 2e-3 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], "cpu", None) == [3.0, 4.0]
    assert bench.aggregate_mlups(1, 16777216, 100, 30.0) == pytest.approx(16777216 * 100 / 0.03 / 1e6)
