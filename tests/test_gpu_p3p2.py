"""Taylor-Hood P3/P2 on the GPU (paper Sec. 4.1, the P3-P2 experiment,
stepped by IPCS as in the paper) against the P3/P2 oracle: sizes and the
initial interpolant, free-running IPCS steps within 1e-9 relative L2, the
exact P3 x P2 steady state kept, and the calls a P3/P2 problem does not
support refused."""
import numpy as np
import pytest

import fs_workloads as W
from oracle import p3p2 as Q
from tests.gpu_helpers import rel_l2

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


def _oracle(wl):
    return Q.Problem3(n=wl.n, problem=wl.problem, nu=wl.nu, dt=wl.dt, jitter=wl.jitter,
                      seed=wl.seed, wconst=wl.wconst)


CASES = [W.unit_square(8, nu=1.0, dt=0.01).with_(steps=5),
         W.unit_square(16, nu=0.02, dt=5e-3, jitter=0.05, seed=4).with_(steps=3)]


@pytest.mark.parametrize("wl", CASES, ids=lambda w: w.name)
def test_p3p2_ipcs_steps_match_oracle(fs, wl):
    S = fs.Stepper.from_workload_p3(wl)
    try:
        P = _oracle(wl)
        assert S.info["n_p3"] == P.n3 and S.info["n_p2_pressure"] == P.np_
        x0, _ = S.state()
        assert rel_l2(x0, P.x) <= 1e-14
        for k in range(wl.steps):
            st = fs.fs_step_ipcs(S.prob, 1)[0]
            assert st["status"] == 0 and max(st["rel_res"]) <= 1e-11, st
            P.ipcs_step()
            x, t = S.state()
            assert abs(t - P.t) < 1e-14
            e = rel_l2(x, P.x)
            print(f"P3/P2 {wl.name} IPCS step {k}: rel L2 {e:.2e}, CG iterations {st['iters']}")
            assert e <= 1e-9, (k, e)
    finally:
        S.close()


def test_p3p2_keeps_exact_steady_state(fs):
    wl = W.Workload(name="poly3", dim=2, n=(5, 4), lo=(0.0, 0.0), hi=(1.0, 1.0),
                    problem=W.POLY3, nu=0.7, dt=0.05, steps=3, jitter=0.1, seed=9,
                    side_mask=0x0F, pin_p0=True, wconst=(1.0, 0.5))
    S = fs.Stepper.from_workload_p3(wl)
    try:
        x0, _ = S.state()
        fs.fs_step_ipcs(S.prob, 3)
        x, _ = S.state()
        assert np.abs(x - x0).max() <= 1e-10 * np.abs(x0).max()
    finally:
        S.close()


def test_p3p2_refuses_the_coupled_calls(fs):
    S = fs.Stepper.from_workload_p3(W.unit_square(4))
    try:
        with pytest.raises(fs.FsError, match="UNSUPPORTED"):
            fs.fs_step(S.prob, 1)
        with pytest.raises(fs.FsError, match="UNSUPPORTED"):
            fs.fs_step_picard(S.prob, 1)
    finally:
        S.close()
    with pytest.raises(fs.FsError, match="UNSUPPORTED"):
        fs.Stepper.from_workload_p3(W.cube(2))
