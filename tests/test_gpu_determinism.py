"""Run-to-run determinism of the CUDA path in its deterministic mode: the
element kernels add into the block values colour by colour (cells of one
colour share no node) with no atomics, and every reduction of the Krylov
solve (norms, Gram-Schmidt dots) sums its partials in a fixed order, so two
runs of the same problem give bit-identical assembled systems and states.
The default mode adds the per-step convection values with FP64 atomics; its
runs agree to rounding (checked here against the deterministic mode)."""
import numpy as np
import pytest

import fs_workloads as W

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


def _run(fs, wl, prec, steps):
    S = fs.Stepper.from_workload(wl, precision=prec, deterministic=True)
    try:
        info = S.info
        val = torch.zeros(info["nnz"], dtype=torch.float64, device="cuda")
        b = torch.zeros(info["n_dof"], dtype=torch.float64, device="cuda")
        fs.fs_assemble_step(S.prob, wl.dt, val, b)
        torch.cuda.synchronize()
        v0, b0 = val.cpu().numpy(), b.cpu().numpy()
        fs.fs_step(S.prob, steps)
        x, _ = S.state()
        return v0, b0, x
    finally:
        S.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32_refine"])
@pytest.mark.parametrize("wl", [W.C1, W.channel(64, 12), W.cube(6, jitter=0.05)],
                         ids=lambda w: w.name)
def test_two_runs_are_bit_identical(fs, wl, prec):
    a = _run(fs, wl, prec, 3)
    b = _run(fs, wl, prec, 3)
    for p, q in zip(a, b):
        assert np.array_equal(p, q)


@pytest.mark.parametrize("wl", [W.channel(64, 12), W.cube(6, jitter=0.05)], ids=lambda w: w.name)
def test_atomic_assembly_agrees_to_rounding(fs, wl):
    outs = []
    for det in (True, False):
        S = fs.Stepper.from_workload(wl, precision=1, deterministic=det)
        try:
            info = S.info
            val = torch.zeros(info["nnz"], dtype=torch.float64, device="cuda")
            fs.fs_assemble_step(S.prob, wl.dt, val, None)
            torch.cuda.synchronize()
            outs.append(val.cpu().numpy())
        finally:
            S.close()
    a, b = outs
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()
