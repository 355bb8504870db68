"""Batched instances (one problem over a union of independent meshes): each
instance's result equals its solo run within the parity tolerance (1e-9
relative L2; the instance keeps its own Arnoldi process and convergence
test, but shares the multigrid's Chebyshev bounds and depth with the batch,
so the iterates differ at the solver-tolerance level) and the oracle, and
the non-blocking step API gives the same states as the blocking one."""
import numpy as np
import pytest

import fs_workloads as W
from tests.gpu_helpers import oracle_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BATCH = [W.unit_square(6, nu=1.0, jitter=0.0, dt=1e-3),
         W.unit_square(9, nu=0.05, jitter=0.0, dt=1e-3),
         W.unit_square(13, nu=1 / 500, jitter=0.0, dt=1e-3)]


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25403_gb300 import build
    build.build()
    from paper_2605_25403_gb300 import fs as mod
    return mod


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32_refine"])
def test_batch_matches_solo_and_oracle(fs, prec):
    steps = 3
    B = fs.Stepper.from_workloads(BATCH, precision=prec)
    try:
        fs.fs_step(B.prob, steps)
        xb, tb = B.state()
        stats = fs.fs_instance_stats(B.prob)
        assert all(s["status"] == 0 and s["rel_res"] <= 1e-12 for s in stats)
        for i, wl in enumerate(BATCH):
            S = fs.Stepper.from_workload(wl, precision=prec)
            try:
                fs.fs_step(S.prob, steps)
                xs, ts = S.state()
            finally:
                S.close()
            xi = B.instance_state(xb, i)
            assert xi.shape == xs.shape
            assert rel_l2(xi, xs) <= 1e-9, (i, rel_l2(xi, xs))
            P = oracle_problem(wl)
            for _ in range(steps):
                P.step()
            assert rel_l2(xi, P.x) <= 1e-9, (i, rel_l2(xi, P.x))
    finally:
        B.close()


def test_async_step_api_matches_blocking(fs):
    wl = W.unit_square(10, jitter=0.05, seed=1)
    A = fs.Stepper.from_workload(wl)
    Bs = fs.Stepper.from_workload(wl)
    try:
        fs.fs_step(A.prob, 3)
        fs.fs_step_begin(Bs.prob, 3)
        polls = 0
        while True:
            done, rc = fs.fs_step_poll(Bs.prob, wait=False)
            polls += 1
            if done:
                break
        assert rc == 0 and polls >= 1
        xa, ta = A.state()
        xb, tb = Bs.state()
        assert ta == tb
        assert rel_l2(xb, xa) <= 1e-12
    finally:
        A.close()
        Bs.close()
