"""Starting guesses of the time steps.  fs_step starts every solve from the
polynomial extrapolation of the state history: the converged states are
those of solves started from the latest state (within the solver
tolerance), with fewer inner iterations on a run that is smooth in time.  A
state set at the current time continues the history; one set at another
time starts a new history."""
import numpy as np
import pytest

import fs_workloads as W
from tests.gpu_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the Sec. 4.1 solution (smooth in time) on a 24x24 square
WL = W.unit_square(24, nu=1e-2, jitter=0.0, dt=1e-3)
NSTEPS = 6


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25403_gb300 import build
    build.build()
    from paper_2605_25403_gb300 import fs as mod
    return mod


def _stepped(fs, before_last=None):
    """NSTEPS steps through fs_step; `before_last(S)` runs before the last."""
    S = fs.Stepper.from_workload(WL, precision=fs.FS_PREC_FP64)
    try:
        iters = []
        for k in range(NSTEPS):
            if k == NSTEPS - 1 and before_last is not None:
                before_last(S)
            st = fs.fs_step(S.prob, 1)[0]
            assert st["status"] == 0
            iters.append(st["iters"])
        x, t = fs.fs_get_state(S.prob)
        return iters, x, t
    finally:
        S.close()


def test_history_cuts_iterations_not_the_solution(fs):
    iters, x, t = _stepped(fs)
    # the same steps with every solve started from the latest state:
    # assemble, then fs_solve from the state (fs_solve does not extrapolate)
    S = fs.Stepper.from_workload(WL, precision=fs.FS_PREC_FP64)
    try:
        plain = []
        for _ in range(NSTEPS):
            xn, tn = fs.fs_get_state(S.prob)
            fs.fs_assemble_step(S.prob, tn + WL.dt)
            st = fs.fs_solve(S.prob)
            assert st["status"] == 0
            plain.append(st["iters"])
            xs, _ = fs.fs_get_state(S.prob)
            fs.fs_set_state(S.prob, xs, tn + WL.dt)
        xp, tp = fs.fs_get_state(S.prob)
    finally:
        S.close()
    assert abs(tp - t) <= 1e-15
    assert rel_l2(x, xp) <= 1e-9, rel_l2(x, xp)
    # the first step has no history; the later ones start closer
    assert iters[0] == pytest.approx(plain[0], abs=1)
    assert sum(iters[2:]) < sum(plain[2:]), (iters, plain)


def test_state_set_at_the_current_time_keeps_the_history(fs):
    iters, x, _ = _stepped(fs)

    def same_time(S):
        xs, ts = fs.fs_get_state(S.prob)
        fs.fs_set_state(S.prob, xs, ts)

    kept, xk, _ = _stepped(fs, same_time)
    assert abs(kept[-1] - iters[-1]) <= 1, (kept, iters)
    assert rel_l2(xk, x) <= 1e-9


def test_state_set_at_another_time_starts_a_new_history(fs):
    iters, _, _ = _stepped(fs)

    def other_time(S):
        xs, ts = fs.fs_get_state(S.prob)
        fs.fs_set_state(S.prob, xs, ts + 0.5 * WL.dt)

    fresh, _, _ = _stepped(fs, other_time)
    # the last solve starts from the state alone, as a first step does
    assert fresh[-1] > iters[-1], (fresh, iters)
