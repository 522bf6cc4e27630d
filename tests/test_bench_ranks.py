"""The multi-rank path of bench.py (replicas, one independent series per rank)
on CPU with the gloo backend, world size 2: the job's time is the slowest
rank's and the per-step figure divides by all ranks' steps."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r spent 100 + 50 r ms on 4 steps
    v = bench.aggregate_ms_per_step(100.0 + 50.0 * rank, 4, world, dist)
    m = bench.max_over_ranks(3.0 - rank, dist)
    out[rank] = (v, m)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        v, m = out[r]
        assert abs(v - 150.0 / (4 * 2)) < 1e-12
        assert m == 3.0


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_ms_per_step(80.0, 4, 1, None) == 20.0
    assert bench.max_over_ranks(2.5, None) == 2.5


def test_roofline_bytes_follow_the_accounting():
    """The bench's byte counts against hand-worked values.  One cycle of k = 2
    Arnoldi steps on N points, FP32 (s = 4):
    three-sweep CGS2 accounting: steps j = 0, 1 move s N (3(j+1) + 7) = 10 s N
    and 13 s N; x += V y adds (k s + 16) N = 24 N; the FP64 true residual 32 N.
    Two-pass: steps move s N (2j + 6) = 6 s N and 8 s N; x += V y s N k + 16 N;
    the restart 16 N + s N; the final residual check 16 N + s N."""
    import bench
    N, s = 1000, 4
    res = {"iters": 2, "cycles": 1}
    assert bench.algorithmic_bytes(res, N, 30, s) == (10 + 13) * s * N + 24 * N + 32 * N
    assert bench.algorithmic_bytes(res, N, 30, s, kappa=True) == \
        (10 + 13) * s * N + 2 * 4 * N + 24 * N + 32 * N
    assert bench.two_pass_bytes(res, N, 30, s) == \
        (6 + 8) * s * N + (2 * s * N + 16 * N) + (16 * N + s * N) + (16 * N + s * N)
    # two cycles: a full one of m = 3 steps, then 1 step
    res = {"iters": 4, "cycles": 2}
    per = lambda k: sum(s * N * (3 * (j + 1) + 7) for j in range(k)) + (k * s + 16) * N + 32 * N  # noqa: E731
    assert bench.algorithmic_bytes(res, N, 3, s) == per(3) + per(1)
