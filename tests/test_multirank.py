"""Host logic of the multi-rank benchmark path on CPU: gloo ranks, each building
and advancing its own replica of the workload, reduce their timings to the
maximum and report the whole-job throughput (weak scaling, no data-path
collective).  The oracle's FP64 step stands in for the GPU step."""
import os
import time

import pytest


def _tiny_workload():
    from paper_2607_06794_b300 import Config, workloads
    c = Config(32, 24, 16, prec="fp32", cx=15.5, cy=11.5, cz=-0.5, a=13, b=10, c=12, width=1.0,
               theta_deg=80.0, J0=1e-4, evap_start=0, top_bc=1, max_beads=64, eps_coh=0.006,
               xi=0.05, seed=77)
    return workloads.Workload("tiny_replica", [c], [None], [(3, 6.0)], 10)


def _rank(rank, world, port, q, delay):
    try:
        _replica(rank, world, port, q, delay)
    except BaseException as e:  # report instead of leaving the parent waiting
        q.put((rank, repr(e)))
        raise


def _replica(rank, world, port, q, delay):
    import torch.distributed as dist

    import bench
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "1"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _tiny_workload()
    wires = bench.wire_placement(wl)  # every rank builds the same replica
    p, fR, fB, cot, beads = bench.oracle_workload(wl, wires)
    acc = oracle.Acc()
    steps = 3
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        assert oracle.step(p, fR, fB, cot, acc, beads) == 0
    if rank == world - 1:
        time.sleep(delay)  # the slow rank sets the job time
    ms_local = (time.perf_counter() - t0) * 1e3
    dist.barrier()
    ms, value = bench.job_throughput(ms_local, wl.nodes, steps, world, dist, "cpu")
    q.put((rank, ms_local, ms, value, wl.nodes, beads.n, float(fR.sum())))
    dist.destroy_process_group()


def test_gloo_replicas_reduce_to_the_slowest_and_sum_the_work():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    world, delay = 2, 0.3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q, delay)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=300) for _ in ps)
    assert all(len(o) > 2 for o in out), out
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    ms_all = [o[1] for o in out]
    # every rank reports the slowest rank's time and the same whole-job number
    assert [o[2] for o in out] == [max(ms_all)] * world
    assert max(ms_all) >= delay * 1e3
    nodes, steps = out[0][4], 3
    assert nodes == 32 * 24 * 16
    assert out[0][3] == pytest.approx(world * nodes * steps / (max(ms_all) * 1e-3) / 1e6)
    assert out[0][3] == out[1][3]
    # the replicas are identical: same wires, same state after the same steps
    assert out[0][5] == out[1][5] == 9
    assert out[0][6] == out[1][6]


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.whole_job_mlups(2_097_152, 200, 116.0, 1) == pytest.approx(2_097_152 * 200 / 0.116 / 1e6)
    assert bench.job_throughput(4.0, 1000, 10, 1, None, "cpu") == (4.0, pytest.approx(1000 * 10 / 4e-3 / 1e6))


def test_bench_host_helpers_run_on_the_current_sources():
    """The bench's host-side helpers that need no GPU: the kernel-source hash that keys
    the committed traffic figures, the peak lookup and the launch count per step."""
    import bench
    from paper_2607_06794_b300 import workloads
    h = bench.kernel_hash()
    assert len(h) == 12 and h == bench.kernel_hash()
    peak, kind = bench.peaks()
    assert peak > 1000.0 and kind in ("measured", "fallback")
    assert bench.launches_per_step(workloads.droplet_c5("fp32")) == 2 + 4 + 5
    assert bench.launches_per_step(workloads.droplet_c1()) == 2
