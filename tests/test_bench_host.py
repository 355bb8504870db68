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


def test_roofline_kernel_traffic_is_recorded():
    """The default roofline kernel of the bench line has a committed DRAM
    traffic figure (ncu capture of the CGS2 update pass on the channel)."""
    import bench
    a = bench.parse([])
    t = bench.traffic_from_profiles(a.roofline_kernel, "channel_512x96")
    assert a.roofline_kernel == "cgs_upd" and t is not None and 25e6 < t < 35e6


class _FakeFs:
    """Stands in for the binding: records the smoother calls."""

    def __init__(self):
        self.calls = []

    def fs_autotune_smoother(self, prob, candidates, nsteps=3):
        self.calls.append(("fixed", list(candidates), nsteps))
        return {"best": {"cheb_ratio": candidates[0][0]}}

    def fs_tune_smoother(self, prob, nsteps=3, degrees=(), ratios=()):
        self.calls.append(("tune", tuple(degrees), tuple(ratios), nsteps))
        return {"cheb_ratio": ratios[0]}


def test_smoother_set_up_tuned_or_fixed():
    import bench

    class S:
        prob = None

    assert bench.parse_ratios("4, 6,,12") == (4, 6, 12)
    fake = _FakeFs()
    saved = bench.FIXED_SMOOTHER
    try:
        bench.FIXED_SMOOTHER = None
        assert bench.tune_smoother(fake, S, (), 5) is None      # tuning switched off
        bench.tune_smoother(fake, S, (6, 12), 5)
        assert fake.calls[-1] == ("tune", bench.SMOOTHER_DEGREES, (6, 12), 5)
        bench.FIXED_SMOOTHER = (1, 2, 16)                       # --smoother 1,2,16
        bench.tune_smoother(fake, S, (6, 12), 5)
        assert fake.calls[-1] == ("fixed", [(16, 1, 2)], 1)
    finally:
        bench.FIXED_SMOOTHER = saved
