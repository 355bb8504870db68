"""Host logic of bench.py: the max-over-ranks timing of a multi-rank run,
exercised with two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.aggregate_time(1.0 + rank * 0.5, dist)
    out[rank] = t
    dist.destroy_process_group()


def test_slowest_rank_time_with_two_gloo_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 1.5


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_time(2.25, None) == 2.25
    a = bench.parse(["--steps", "7", "--batch-steps", "0"])
    assert a.steps == 7 and a.batch_steps == 0 and a.gpus == 1


def test_traffic_of_the_roofline_kernel_comes_from_the_committed_capture():
    """The bench line's roofline `traffic` is read from profiles/traffic.txt
    (DRAM bytes per launch of one ncu capture of the current kernel)."""
    import bench
    t = bench.traffic_from_profiles("cheb", "channel_512x96")
    assert t is not None and 20e6 < t < 30e6      # ~ the 27.6 MB algorithmic
    assert bench.traffic_from_profiles("cheb", "no_such_workload") is None
