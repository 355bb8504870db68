"""Incremental pressure-correction stepping on the GPU (paper Sec. 2.2.1,
IPCS; the Sec. 4.1 table "IPCS convergence analysis") against the oracle's
IPCS step, stage by stage solved exactly there and by CG here (Jacobi for
the velocity stages, one multigrid V-cycle per iteration for the pressure
stage): relative L2 <= 1e-9 at every step, free-running; the pressure
stage's iteration count stays flat under refinement; exact discrete steady
states are kept; boundary set-ups the scheme does not cover are refused."""
import numpy as np
import pytest

import fs_workloads as W
from oracle import oracle as O
from tests.gpu_helpers import oracle_problem, poly_oseen, rel_l2

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


CASES = [W.unit_square(8, nu=1.0, dt=0.01).with_(steps=5),
         W.unit_square(32, nu=1.0 / 50, dt=5e-3, jitter=0.05, seed=4).with_(steps=3),
         W.cube(3, nu=0.1, dt=0.01, jitter=0.1, seed=2).with_(steps=3)]


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_ipcs_steps_match_oracle(fs, wl):
    S = fs.Stepper.from_workload(wl)
    try:
        P = oracle_problem(wl)
        for k in range(wl.steps):
            st = fs.fs_step_ipcs(S.prob, 1)[0]
            assert st["status"] == 0 and max(st["rel_res"]) <= 1e-11, st
            O.ipcs_step(P)
            x, t = S.state()
            assert abs(t - P.t) < 1e-14
            e = rel_l2(x, P.x)
            print(f"{wl.name} IPCS step {k}: rel L2 {e:.2e}, CG iterations {st['iters']}")
            assert e <= 1e-9, (k, e)
    finally:
        S.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_pressure_stage_iterations_flat_in_mesh_size(fs, prec):
    # Jacobi CG needs O(n) iterations on the pressure Poisson problem (248 at
    # 32 x 32 to 1e-13); the V-cycle preconditioner keeps the count bounded.
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    its = {}
    for n in (16, 64, 128):
        wl = W.unit_square(n, nu=1.0 / 50, dt=5e-3, jitter=0.05, seed=4)
        S = fs.Stepper.from_workload(wl, precision=p)
        try:
            st = fs.fs_step_ipcs(S.prob, 2)
            assert all(s["status"] == 0 for s in st), st
            its[n] = max(s["iters"][1] for s in st)
        finally:
            S.close()
    print(prec, "pressure CG iterations by n:", its)
    assert max(its.values()) <= 40, its
    assert its[128] <= its[16] + 16, its


@pytest.mark.parametrize("dim,n", [(2, (5, 4)), (3, (2, 3, 2))])
def test_ipcs_keeps_exact_discrete_steady_state(fs, dim, n):
    wl = poly_oseen(dim, n)
    S = fs.Stepper.from_workload(wl)
    try:
        x0, _ = S.state()
        fs.fs_step_ipcs(S.prob, 3)
        x, _ = S.state()
        assert np.abs(x - x0).max() <= 1e-10 * max(1.0, np.abs(x0).max())
    finally:
        S.close()


def test_ipcs_refuses_natural_boundaries(fs):
    S = fs.Stepper.from_workload(W.channel(16, 4))
    try:
        with pytest.raises(fs.FsError, match="UNSUPPORTED"):
            fs.fs_step_ipcs(S.prob, 1)
    finally:
        S.close()
