"""The allocation-free residual check against the allocating one.

fs_csr_residual_norm_noalloc exists for callers that cannot allocate device
memory (serving processes whose memory is committed under a fixed budget,
hosts that forbid a library to grow after start-up); it runs the same
reduction with static device scratch.
Two calls in a row must agree with fs_csr_residual_norm within the tolerance
of the other residual tests.  Collected last so that a failure here comes
after every other test has run."""
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


def _system(fs, wl):
    S = fs.Stepper.from_workload(wl, dofmap_arrays=True)
    info = S.info
    val = torch.zeros(info["nnz"], dtype=torch.float64, device="cuda")
    b = torch.zeros(info["n_dof"], dtype=torch.float64, device="cuda")
    fs.fs_assemble_step(S.prob, wl.dt, val, b)
    torch.cuda.synchronize()
    rp = torch.from_numpy(info["rowptr"]).cuda()
    col = torch.from_numpy(info["col"]).cuda()
    return S, rp, col, val, b


@pytest.mark.parametrize("wl", [W.C1, W.channel(64, 12)], ids=lambda w: w.name)
def test_noalloc_matches_allocating_entry_point(fs, wl):
    S, rp, col, val, b = _system(fs, wl)
    try:
        rng = np.random.default_rng(7)
        for call in range(2):
            x = torch.from_numpy(rng.standard_normal(b.numel())).cuda()
            r_ref, b_ref = fs.fs_csr_residual_norm(rp, col, val, x, b)
            r_na, b_na = fs.fs_csr_residual_norm_noalloc(rp, col, val, x, b)
            assert abs(r_na - r_ref) <= 1e-12 * r_ref, (call, r_na, r_ref)
            assert abs(b_na - b_ref) <= 1e-12 * b_ref, (call, b_na, b_ref)
    finally:
        S.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(fs):
    S, rp, col, val, b = _system(fs, W.C1)
    try:
        with pytest.raises(fs.FsError, match="exceed the limit"):
            fs.fs_csr_residual_norm_noalloc(rp, col, val, b, b, n=4194305)
    finally:
        S.close()
