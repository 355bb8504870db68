"""The continuous-batching request loop: requests admitted as slots and
memory free up, several requests resident at once, and each
request's result the same alone and in the mix (bit for bit for requests
in the deterministic mode: assembly and every reduction of the solve sum in
a fixed order, so a request's arithmetic does not depend on what else runs) and the same as the oracle's steps of
that request (within the parity tolerance, 1e-9 relative L2); the
admission estimate bounds the measured footprint of large 2D and 3D
requests too."""
import time

import numpy as np
import pytest

import fs_workloads as W
from tests.gpu_helpers import oracle_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX = [(W.unit_square(12, nu=1.0 / 50, jitter=0.0, dt=1e-3), 4),
       (W.cube(4, nu=1.0 / 20, jitter=0.0, dt=1e-3), 3),
       (W.unit_square(20, nu=1.0 / 900, jitter=0.0, dt=1e-3), 5),
       (W.unit_square(7, nu=1.0, jitter=0.0, dt=1e-3), 6),
       (W.cube(3, nu=1.0 / 300, jitter=0.0, dt=1e-3), 2)]


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25403_gb300 import build
    build.build()
    from paper_2605_25403_gb300 import fs as mod
    return mod


def _run(fs, reqs, budget, slots, keep=True, watch=None):
    srv = fs.Server(budget, slots)
    try:
        t0 = time.perf_counter()
        ids = [srv.submit(wl, n, 0.0, keep_state=keep, deterministic=True) for wl, n in reqs]
        done = {}
        while len(done) < len(ids):
            srv.progress(time.perf_counter() - t0)
            for r in srv.completed():
                done[r["id"]] = r
            if watch is not None:
                watch(srv.status())
            assert time.perf_counter() - t0 < 300
        states = [srv.take_state(i) for i in ids] if keep else None
        return [done[i] for i in ids], states
    finally:
        srv.close()


def test_results_same_alone_and_in_the_mix(fs):
    alone = []
    for wl, n in MIX:
        res, st = _run(fs, [(wl, n)], 8 << 30, 1)
        assert res[0]["status"] == 0
        alone.append(st[0])
    seen = []
    res, mixed = _run(fs, MIX, 8 << 30, len(MIX), watch=lambda s: seen.append(s))
    for (wl, n), r, xa, xm in zip(MIX, res, alone, mixed):
        assert r["status"] == 0 and r["nsteps"] == n
        assert np.array_equal(xm, xa), (wl.name, rel_l2(xm, xa))
        P = oracle_problem(wl)
        for _ in range(n):
            P.step()
        assert rel_l2(xm, P.x) <= 1e-9, (wl.name, rel_l2(xm, P.x))
    # the mix was resident at once (whether one request's steps end before
    # another's set-up does depends on their speeds, so that is not tested)
    assert max(s["resident"] for s in seen) >= 2


def test_admission_respects_budget_and_slots(fs):
    reqs = [(W.unit_square(16, nu=1.0 / 100, jitter=0.0, dt=1e-3), 3) for _ in range(6)]
    est = fs.fs_server_estimate_bytes(reqs[0][0])
    seen = []
    budget = int(2.5 * est)  # room for two requests at a time
    res, _ = _run(fs, reqs, budget, 4, keep=False, watch=lambda s: seen.append(s))
    assert all(r["status"] == 0 for r in res)
    assert max(s["resident"] for s in seen) <= 2
    assert max(s["bytes_reserved"] for s in seen) <= budget
    # the estimate bounds the measured footprint
    assert all(r["device_bytes"] <= est for r in res)
    # FIFO admission
    adm = [r["admitted"] for r in res]
    assert adm == sorted(adm)


@pytest.mark.parametrize("wl", [W.unit_square(512, jitter=0.0, nu=1e-3, dt=1e-3),
                                W.cube(48, jitter=0.0, nu=1e-3, dt=1e-3)],
                         ids=lambda w: w.name)
def test_estimate_bounds_footprint_of_large_requests(fs, wl):
    """The largest sizes of the serving workload (2D N = 512: 2.36M DOF; 3D
    N = 48: 2.86M DOF, with its dense coarsest levels): the measured device
    footprint of one served request stays within its admission estimate, and
    the reservation it holds while resident is the estimate."""
    est = fs.fs_server_estimate_bytes(wl)
    seen = []
    res, _ = _run(fs, [(wl, 1)], 150 << 30, 1, keep=False, watch=lambda s: seen.append(s))
    assert res[0]["status"] == 0
    assert 0 < res[0]["device_bytes"] <= est, (res[0]["device_bytes"], est)
    assert max(s["bytes_reserved"] for s in seen) == est
