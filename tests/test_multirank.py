"""Host logic of the multi-rank benchmark path on CPU: two gloo ranks, each with
its own replica, reduce their timings to the maximum and report the whole-job
throughput (weak scaling, no data-path collective)."""
import os

import pytest


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # the slower rank sets the job time
    m = bench.reduce_max(ms, dist, "cpu")
    v = bench.whole_job_mlups(1_000_000, 100, m, world)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_sum_the_work():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    # 2 ranks x 1e6 nodes x 100 steps in 15 ms
    assert out[0][2] == pytest.approx(2 * 1e6 * 100 / 15e-3 / 1e6)
    assert out[0][2] == out[1][2]


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.whole_job_mlups(2_097_152, 200, 116.0, 1) == pytest.approx(2_097_152 * 200 / 0.116 / 1e6)
