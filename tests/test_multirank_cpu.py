"""The multi-rank bench path on CPU: two gloo ranks (replicas) agree on the
slowest rank's timed region and on the whole-job sweeps/s."""
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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = 100.0 + 50.0 * rank               # rank 1 is the slow one
        tot = bench.max_over_ranks(mine, dist)
        q.put((rank, tot, bench.job_value(20, ws, tot), bench.dist_env()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, tot, value, env in out:
        assert tot == 150.0
        assert abs(value - 20 * 2 / 0.150) < 1e-9
        assert env == (2, rank, 0)
