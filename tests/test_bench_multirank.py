"""bench.py's multi-rank path on CPU: two gloo ranks (one per process), slowest-rank timing and
the whole-job throughput; no GPU and no collective on the data path."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0 + 5.0 * rank, 3.0 - rank]
    red = bench.reduce_max(ms, world, "cpu")
    out[rank] = (red, bench.aggregate_throughput(red[0], world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        red, value = out[r]
        assert red == [15.0, 3.0]
        assert value == pytest.approx(2 * 1000.0 / 15.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.aggregate_throughput(20.0, 1) == pytest.approx(50.0)


def test_bench_workloads_name_the_seeded_configurations():
    """Every --workload of bench.py builds one of the seeded workloads, with its N, M, S, gamma."""
    import bench
    from paper_2105_08806_gb300 import workloads as W
    expect = {"2d-hard-spheres": (2, 64, 32), "2d-maxwell": (2, 16, 8), "3d-bkw": (3, 16, 32),
              "3d-bimaxwell": (3, 24, 32)}
    assert bench.HEADLINE == "2d-hard-spheres" and set(bench.WORKLOADS) == set(expect)
    for name, (ctor, desc) in bench.WORKLOADS.items():
        w = getattr(W, ctor)()
        assert (w.d, w.N, w.M) == expect[name], name
        assert f"N={w.N}" in desc and f"M={w.M}" in desc
