"""Multi-process (replica) logic of bench.py on CPU with the gloo backend,
world size 2: max-over-ranks timing, summed work, and the reference arm's
rank-0-only behaviour."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tot, its = bench.aggregate(dist, 1.0 + rank, 10 * (rank + 1), "cpu")
        q.put((rank, tot, its))
    finally:
        dist.destroy_process_group()


def test_aggregate_gloo_world2():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tot, its in got:
        assert tot == 2.0          # the slowest rank's time
        assert its == 30.0         # all ranks' iterations


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(None, 3.5, 7, "cpu") == (3.5, 7)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0

    bench.run_reference(A())
    assert capsys.readouterr().out == ""
