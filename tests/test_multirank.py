"""The N > 1 path of bench.py on CPU: two gloo ranks (rendezvous on 127.0.0.1) check the
cross-rank timing rule (the job's time is its slowest rank's, every rank sees it) and the
whole-job throughput of N replicas (units of all ranks / that time), and that the
reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + 0.5 * rank            # the last rank is the slowest
        mx = bench.max_over_ranks(t_local, "cpu", dist)
        thr = bench.job_throughput(100.0, t_local, world, "cpu", dist)
        assert bench.dist_env() == (rank, rank, world)
        q.put((rank, mx, thr))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_throughput():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        results = sorted(q.get(timeout=180) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    slowest = 1.0 + 0.5 * (world - 1)
    for rank, mx, thr in results:
        assert mx == pytest.approx(slowest)
        assert thr == pytest.approx(100.0 * world / slowest)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    args = type("Args", (), dict(workload="ngon32_small", steps=1, warmup=0, gpus=2))
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.reference_arm(args, rank=1, world=2) is None
    assert out.getvalue() == ""
