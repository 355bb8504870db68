"""Free-running solution parity at large sizes: the CUDA path, stepped through
the C ABI exactly as the benchmark steps it, against the oracle's own solve
of the same steps (relative L2 <= 1e-9 at every step).

  * channel 512x96 (445,411 DOF), the benchmark workload: 2 steps from the
    impulsive start, FP32 inner solves with FP64 refinement and the plain
    FP64 path; the oracle takes the sparse direct solve (ILU(0)-GMRES
    stagnates on this do-nothing saddle-point system);
  * cube 16^3 (112,724 DOF, jitter 0.05h): 5 steps, both precisions, the
    oracle's ILU(0)-GMRES;
  * a batch whose first instance is the hardest corner of the batched
    workload (N = 128, Re = 2000), beside a viscous-dominated one (N = 16,
    Re = 1) and a middle one: 3 steps, each instance against its own oracle
    run.

The oracle runs on the host inside the test (about a minute per channel
step on one core).
"""
import time

import numpy as np
import pytest

import fs_workloads as W
from tests.gpu_helpers import oracle_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25403_gb300 import build
    build.build()
    from paper_2605_25403_gb300 import fs as mod
    return mod


def _free_running(fs, wl, steps, method):
    S = {p: fs.Stepper.from_workload(wl, precision=p) for p in (1, 0)}
    try:
        P = oracle_problem(wl)
        for p in S:
            assert rel_l2(S[p].state()[0], P.x) <= 1e-14
        errs = []
        for k in range(steps):
            t0 = time.time()
            P.step(method=method)
            t_or = time.time() - t0
            row = {}
            for p, st in S.items():
                s = fs.fs_step(st.prob, 1)[0]
                assert s["status"] == 0 and s["rel_res"] <= 1e-12, (p, k, s)
                x, t = st.state()
                assert abs(t - P.t) < 1e-14
                row[p] = rel_l2(x, P.x)
            errs.append(row)
            print(f"{wl.name} step {k}: rel L2 fp32+refine {row[1]:.2e} fp64 {row[0]:.2e}"
                  f" (oracle {t_or:.1f} s)")
        for k, row in enumerate(errs):
            for p, e in row.items():
                assert e <= 1e-9, (wl.name, k, p, e)
    finally:
        for st in S.values():
            st.close()


def test_channel_512x96_free_running_vs_oracle(fs):
    _free_running(fs, W.C2, 2, "lu")


def test_cube_16_free_running_vs_oracle(fs):
    _free_running(fs, W.cube(16), 5, "auto")


HARD_BATCH = [W.unit_square(128, nu=1 / 2000.0, dt=1e-3, jitter=0.0),
              W.unit_square(16, nu=1.0, dt=1e-3, jitter=0.0),
              W.unit_square(37, nu=1 / 150.0, dt=1e-3, jitter=0.0)]


@pytest.mark.parametrize("prec", [1, 0], ids=["fp32_refine", "fp64"])
def test_batch_hard_corner_vs_oracle(fs, prec):
    steps = 3
    B = fs.Stepper.from_workloads(HARD_BATCH, precision=prec)
    try:
        Ps = [oracle_problem(w) for w in HARD_BATCH]
        for k in range(steps):
            fs.fs_step(B.prob, 1)
            stats = fs.fs_instance_stats(B.prob)
            assert all(s["status"] == 0 and s["rel_res"] <= 1e-12 for s in stats), stats
            xb, tb = B.state()
            for i, P in enumerate(Ps):
                P.step(method="lu")
                e = rel_l2(B.instance_state(xb, i), P.x)
                print(f"batch instance {i} ({HARD_BATCH[i].name}, nu {HARD_BATCH[i].nu:.2e})"
                      f" step {k}: rel L2 {e:.2e}, {stats[i]['iters']} iterations")
                assert e <= 1e-9, (i, k, e)
    finally:
        B.close()


def test_batch_n256_re2000_vs_oracle(fs):
    """The extreme corner of the batched workload, N = 256 (592,387 DOF) at
    Re = 2000, inside a batch beside a small viscous instance: one step of
    both precisions against the oracle's sparse direct solve of the same
    step (about a minute on one core)."""
    wls = [W.unit_square(256, nu=1 / 2000.0, dt=1e-3, jitter=0.0),
           W.unit_square(16, nu=1.0, dt=1e-3, jitter=0.0)]
    Bs = {p: fs.Stepper.from_workloads(wls, precision=p) for p in (1, 0)}
    try:
        Ps = [oracle_problem(w) for w in wls]
        for P in Ps:
            P.step(method="lu")
        for p, B in Bs.items():
            fs.fs_step(B.prob, 1)
            stats = fs.fs_instance_stats(B.prob)
            assert all(s["status"] == 0 and s["rel_res"] <= 1e-12 for s in stats), (p, stats)
            xb, _ = B.state()
            for i, P in enumerate(Ps):
                e = rel_l2(B.instance_state(xb, i), P.x)
                print(f"precision {p} instance {i} ({wls[i].name}): rel L2 {e:.2e}, "
                      f"{stats[i]['iters']} iterations")
                assert e <= 1e-9, (p, i, e)
    finally:
        for B in Bs.values():
            B.close()
