"""The multi-process path of bench.py on CPU: two gloo ranks (replicas, one
per GPU on a real node) agree on the slowest rank's time and report the
whole-job throughput; the reference arm prints on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 1.5 + rank  # rank 1 is the slow replica
        dist.barrier()
        t_max = bench.max_over_ranks(elapsed, dist)
        q.put((rank, t_max, bench.replica_value(300.0, world, t_max), bench._dist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_agree_on_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]
    assert [o[2] for o in out] == [240.0, 240.0]  # 2 ranks x 300 units / 2.5 s
    assert [o[3] for o in out] == [(0, 2, 0), (1, 2, 1)]


def test_single_process_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.replica_value(10.0, 1, 2.0) == 5.0


def test_reference_arm_is_silent_off_rank_0(capsys, monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        scale, steps, warmup, gpus = 10, 1, 0, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
