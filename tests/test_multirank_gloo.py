"""The N-rank bench path on CPU with two gloo ranks: every rank times its replica, the job takes
the slowest rank's time (max over ranks) and counts the nodes of all replicas; the reference arm
runs on rank 0 alone."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
        total = bench.slowest_rank_ms(local_ms, dist, torch, "cpu")
        rate = bench.job_rate(w, 1000, 20, total)
        out.put((r, w, total, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_count_all_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for r, w, total, rate in res:
        assert w == 2
        assert total == 15.0                  # max over ranks
        assert rate == pytest.approx(2 * 1000 * 20 / 15e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    calls = []
    monkeypatch.setattr(bench, "run_oracle", lambda *a, **k: calls.append(a) or ([1.0], 1))
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup = "c2", 1, 0
    bench.run_reference(A())
    assert calls == []                        # rank 1 exits without work
