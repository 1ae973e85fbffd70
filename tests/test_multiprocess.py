"""The N > 1 bench path on CPU: world-size-2 gloo ranks run the same
whole-job timing reduction bench.py uses under torchrun (independent
replicas, maximum step time over ranks, aggregate value over ranks)."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 1.0 + rank            # rank 1 is the slow replica
    job = bench.job_timing(ms, world, dist, device="cpu")
    val = bench.job_value(1e9, world, job)
    dist.barrier()
    q.put((rank, job, val))
    dist.destroy_process_group()


def test_two_rank_job_timing_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job, val in res:
        assert job == 2.0                      # maximum over ranks
        assert abs(val - 2 * 1e9 / 2e-3 / 1e9) < 1e-9   # both replicas' bytes over the job time


def test_single_rank_is_identity():
    import bench
    assert bench.job_timing(3.5, 1, None) == 3.5
    assert bench.job_value(2e9, 1, 1.0) == 2000.0
