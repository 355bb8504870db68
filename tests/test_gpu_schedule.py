"""Execution schedules of the multigrid preconditioner.

The coarse levels can run as separate kernels or inside one cluster kernel,
and the SpMV and smoothing passes can issue 4, 6 or 8 matrix slots per
thread at a time (fs_set_schedule).  Every form evaluates the same per-row
formulas, so a schedule changes launch counts and timing, not the solution:
the preconditioner outputs differ at most by rounding (FMA contraction may differ
between the two compiled forms), and the two solves then stop at different
iterates that both meet rtol = 1e-14, so the step results agree to the
conditioning times rtol.  Bars: FP64 1e-11 (the preconditioner differs by
FP64 rounding only, which the FP64 Krylov iterates follow closely); FP32
inner solves with FP64 refinement 1e-9, the parity bar (batched and solo
solves of the same instance already differ by about 1e-10 there).
fs_autotune times the candidates and installs the fastest.
"""
TOL = {"fp64": 1e-11, "fp32_refine": 1e-9}
import numpy as np
import pytest

import fs_workloads as W
from tests.gpu_helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (tail rows velocity, tail rows pressure, SpMV group, smoothing group,
#  coarse-level smoother degree, serialised launches, persistent preconditioner,
#  finest-level smoother degree, Chebyshev interval ratio, Schur-complement form)
SCHEDULES = [(0, 0, 0, 0, 0, 0, 0, 0, 0, 0), (65536, 65536, 8, 6, 0, 0, 0, 0, 0, 0),
             (4096, 16384, 4, 4, 0, 1, 0, 0, 0, 0), (16384, 0, 6, 6, 0, 0, 0, 0, 0, 0),
             (0, 0, 0, 0, 0, 0, 1, 0, 0, 0), (0, 0, 6, 0, 0, 1, 1, 0, 8, 0)]
KEYS = ("tail_rows_velocity", "tail_rows_pressure", "spmv_group", "smooth_group",
        "coarse_degree", "serial_launches", "persistent_precond", "fine_degree", "cheb_ratio",
        "schur")
PERSISTENT = (0, 0, 0, 0, 0, 0, 1, 0, 0, 0)


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_25403_gb300 import build
    build.build()
    from paper_2605_25403_gb300 import fs as mod
    return mod


def _run(fs, make, sched, prec, nsteps=2, iters=False):
    S = make(prec)
    try:
        fs.fs_set_schedule(S.prob, *sched)
        assert fs.fs_get_schedule(S.prob) == dict(zip(KEYS, sched))
        st = fs.fs_step(S.prob, nsteps)
        assert all(s["status"] == 0 for s in st)
        x = S.state()[0]
        return (x, [s["iters"] for s in st]) if iters else x
    finally:
        S.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_schedules_agree_single(fs, prec):
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    wl = W.channel(64, 16)
    xs = [_run(fs, lambda q: fs.Stepper.from_workload(wl, precision=q), sc, p)
          for sc in SCHEDULES]
    for x in xs[1:]:
        assert rel_l2(x, xs[0]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_schedules_agree_batch(fs, prec):
    """A batch: level 0 of the hierarchies is in instance-block order, so the
    fused kernel's result goes through the block-order map."""
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    wls = [W.unit_square(12, jitter=0.1, seed=1), W.unit_square(20, jitter=0.1, seed=2),
           W.unit_square(9, jitter=0.1, seed=3)]
    make = lambda q: fs.Stepper.from_workloads(wls, precision=q)
    xs = [_run(fs, make, sc, p) for sc in SCHEDULES[:2] + [PERSISTENT]]
    for x in xs[1:]:
        assert rel_l2(x, xs[0]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_persistent_preconditioner_3d_and_batch_with_retirement(fs, prec):
    """The persistent form on 3D rows (three components padded to four) and on
    a batch whose instances converge at different iterations (a small
    viscous square and a larger one at Re = 500): items of a converged
    instance are skipped while the others continue."""
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    wl = W.cube(6, jitter=0.05)
    make = lambda q: fs.Stepper.from_workload(wl, precision=q)
    x0 = _run(fs, make, SCHEDULES[0], p)
    x1 = _run(fs, make, PERSISTENT, p)
    assert rel_l2(x1, x0) <= TOL[prec]
    wls = [W.unit_square(8, jitter=0.1, seed=4),
           W.unit_square(48, nu=1.0 / 500.0), W.unit_square(16, jitter=0.1, seed=5)]
    make = lambda q: fs.Stepper.from_workloads(wls, precision=q)
    x0, i0 = _run(fs, make, SCHEDULES[0], p, nsteps=3, iters=True)
    x1, i1 = _run(fs, make, PERSISTENT, p, nsteps=3, iters=True)
    print(prec, "iterations per step, per pass / persistent:", i0, i1)
    assert rel_l2(x1, x0) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_coarse_degree_two_reaches_the_same_solution(fs, prec):
    """Degree-2 smoothing below the finest level (the default) is a
    different preconditioner from degree 3: the iterates change, the solution
    does not beyond the parity bar.  Both meshes have a smoothed level
    between the finest and the dense coarsest one."""
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    for wl in (W.channel(64, 16), W.cube(10, jitter=0.05)):
        make = lambda q: fs.Stepper.from_workload(wl, precision=q)
        x3, i3 = _run(fs, make, (0, 0, 0, 0, 3, 0, 0, 0, 0, 0), p, iters=True)
        x2, i2 = _run(fs, make, (0, 0, 0, 0, 2, 0, 0, 0, 0, 0), p, iters=True)
        print(wl.name, prec, "iterations per step, degree 3 / 2:", i3, i2)
        assert not np.array_equal(x2, x3)  # the knob reaches the V-cycle
        assert rel_l2(x2, x3) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_fine_degree_two_reaches_the_same_solution(fs, prec):
    """Degree 2 on the finest level of both hierarchies (the default) against
    degree 3, per-pass and in the persistent form and in the fused cluster
    tail when that covers every level: the solution agrees within the parity
    bar, and the persistent and tail forms agree with the per-pass one."""
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    for wl in (W.channel(64, 16), W.cube(10, jitter=0.05)):
        make = lambda q: fs.Stepper.from_workload(wl, precision=q)
        x3, i3 = _run(fs, make, (0, 0, 0, 0, 0, 0, 0, 3, 0, 0), p, iters=True)
        x2, i2 = _run(fs, make, (0, 0, 0, 0, 0, 0, 0, 2, 0, 0), p, iters=True)
        xp = _run(fs, make, (0, 0, 0, 0, 0, 0, 1, 2, 0, 0), p)
        xt = _run(fs, make, (1 << 30, 1 << 30, 0, 0, 0, 0, 0, 2, 0, 0), p)
        print(wl.name, prec, "iterations per step, finest degree 3 / 2:", i3, i2)
        assert not np.array_equal(x2, x3)
        assert rel_l2(x2, x3) <= 1e-9
        assert rel_l2(xp, x2) <= TOL[prec] and rel_l2(xt, x2) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_chebyshev_interval_reaches_the_same_solution(fs, prec):
    """Another smoothing interval is another preconditioner: the iterates
    change, the solution stays within the parity bar; the persistent form
    rebuilds its work-list with the new coefficients and agrees with the
    per-pass form at the same interval."""
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    wl = W.channel(64, 16)
    make = lambda q: fs.Stepper.from_workload(wl, precision=q)
    x8, i8 = _run(fs, make, (0, 0, 0, 0, 0, 0, 0, 0, 8, 0), p, iters=True)
    x12, i12 = _run(fs, make, (0, 0, 0, 0, 0, 0, 0, 0, 12, 0), p, iters=True)
    # degree 1 on every level (the restriction's or load's first step alone)
    x1, i1 = _run(fs, make, (0, 0, 0, 0, 1, 0, 0, 1, 8, 0), p, iters=True)
    print(prec, "iterations per step, degree 1:", i1)
    assert rel_l2(x1, x8) <= 1e-9
    S = make(p)
    try:
        # the persistent work-list is built at ratio 8 first, then replaced
        fs.fs_set_schedule(S.prob, 0, 0, persistent_precond=1)
        fs.fs_set_schedule(S.prob, 0, 0, persistent_precond=1, cheb_ratio=12)
        st = fs.fs_step(S.prob, 2)
        assert all(s["status"] == 0 for s in st)
        xp12 = S.state()[0]
    finally:
        S.close()
    print(prec, "iterations per step, ratio 8 / 12:", i8, i12)
    assert not np.array_equal(x8, x12)
    assert rel_l2(x12, x8) <= 1e-9
    assert rel_l2(xp12, x12) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_convection_diffusion_schur_reaches_the_same_solution(fs, prec):
    """The pressure convection-diffusion Schur part is another preconditioner:
    the solution agrees with the Cahouet-Chabard one within the parity bar,
    on the channel (do-nothing outflow, fixed outflow rows), a jittered cube,
    and a batch (per-instance viscosity and a pinned vertex per instance)."""
    p = fs.FS_PREC_FP64 if prec == "fp64" else fs.FS_PREC_FP32_REFINE
    cases = [(W.channel(64, 16), lambda w, q: fs.Stepper.from_workload(w, precision=q)),
             (W.cube(8, jitter=0.05), lambda w, q: fs.Stepper.from_workload(w, precision=q)),
             ([W.unit_square(12, nu=1 / 500.0, dt=1e-3), W.unit_square(20, nu=0.1, dt=1e-3)],
              lambda w, q: fs.Stepper.from_workloads(w, precision=q))]
    for wl, mk in cases:
        make = lambda q: mk(wl, q)
        xc, ic = _run(fs, make, (0, 0, 0, 0, 0, 0, 0, 0, 0, 0), p, nsteps=3, iters=True)
        xp, ip = _run(fs, make, (0, 0, 0, 0, 0, 0, 0, 0, 0, 1), p, nsteps=3, iters=True)
        print(prec, "iterations per step, Cahouet-Chabard / convection-diffusion:", ic, ip)
        assert not np.array_equal(xc, xp)
        assert rel_l2(xp, xc) <= 1e-9
    S = fs.Stepper.from_workload(W.channel(64, 16), precision=p)
    try:
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, persistent_precond=1, schur=1)
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, schur=2)
        # switched on after the first step: the assembled system's pressure
        # convection is built from the state at once
        fs.fs_step(S.prob, 1)
        fs.fs_set_schedule(S.prob, 0, 0, schur=1)
        st = fs.fs_step(S.prob, 2)
        assert all(s["status"] == 0 for s in st)
    finally:
        S.close()


def test_autotune_smoother_restores_the_state(fs):
    S = fs.Stepper.from_workload(W.channel(64, 16), precision=fs.FS_PREC_FP32_REFINE)
    try:
        fs.fs_step(S.prob, 2)
        x0, t0 = S.state()
        rep = fs.fs_tune_smoother(S.prob, nsteps=2, degrees=((2, 2), (1, 1)), ratios=(6, 12))
        print(rep)
        assert rep["cheb_ratio"] in (6, 12)
        assert (rep["coarse_degree"], rep["fine_degree"]) in ((2, 2), (1, 1))
        for part in ("degrees", "ratios"):
            assert all(m > 0 for m in rep[part]["ms_per_step"])
            assert all(i > 0 for i in rep[part]["iters_per_step"])
        assert fs.fs_get_schedule(S.prob) == rep["ratios"]["best"]
        x1, t1 = S.state()
        assert t1 == t0 and np.array_equal(x0, x1)
        st = fs.fs_step(S.prob, 1)[0]
        assert st["status"] == 0 and st["rel_res"] <= 1e-12
        with pytest.raises(fs.FsError):
            fs.fs_autotune_smoother(S.prob, [(1, 0, 0)], nsteps=1)
        with pytest.raises(fs.FsError):
            fs.fs_autotune_smoother(S.prob, [(0, 4, 0)], nsteps=1)
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, cheb_ratio=100)
    finally:
        S.close()


def test_autotune_installs_a_candidate(fs):
    S = fs.Stepper.from_workload(W.channel(64, 16), precision=fs.FS_PREC_FP32_REFINE)
    try:
        x0, t0 = S.state()
        rep = fs.fs_autotune(S.prob, reps=3)
        assert rep["candidates"] >= 2 and 0 < rep["best_ms"] <= rep["default_ms"]
        assert rep["persistent_ms"] > 0  # the persistent form was timed too
        assert 0 < rep["spmv_best_ms"] <= rep["spmv_default_ms"]
        assert fs.fs_get_schedule(S.prob) == rep["best"]
        x1, t1 = S.state()
        assert t1 == t0 and np.array_equal(x0, x1)  # state untouched
        st = fs.fs_step(S.prob, 1)[0]
        assert st["status"] == 0 and st["rel_res"] <= 1e-12
        ms, _ = fs.fs_profile_kernel(S.prob, fs.FS_KERNEL_PRECOND, reps=3)
        assert ms > 0
        # one CGS2 step on the Krylov scratch, then the next step solves as
        # before (the solve rebuilds its basis and cycle state)
        ms, by = fs.fs_profile_kernel(S.prob, fs.FS_KERNEL_CGS, reps=3)
        assert ms > 0 and by == (3 * 15 + 8) * S.info["n_dof"] * 4
        st = fs.fs_step(S.prob, 1)[0]
        assert st["status"] == 0 and st["rel_res"] <= 1e-12
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, -1, 0)
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, spmv_group=5)
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, smooth_group=8)
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, serial_launches=2)
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, persistent_precond=2)
        with pytest.raises(fs.FsError):
            fs.fs_set_schedule(S.prob, 0, 0, fine_degree=4)
    finally:
        S.close()
