"""Parity at the benchmark sizes (channel 512x96, 445,411 DOF; cube 48^3,
2,855,668 DOF) in the configuration bench.py times.  The oracle cannot solve
these systems in test time, so it checks them one row at a time:

  * sampled rows of the GPU-assembled monolithic system (values and right-hand
    side; the velocity rows of every sampled node and the pressure rows of
    every sampled vertex, B entries and b_p included) against the same rows
    computed by the oracle from the elements that contain the sampled nodes
    (1e-12 of the row's largest entry);
  * after one solved step: the global FP64 residual of the GPU solution with
    the GPU's exported system (<= 1e-12 relative, fs_csr_residual_norm), and
    the residual of sampled rows recomputed by the oracle (the solution
    satisfies the oracle's equations to the same level).
"""
import numpy as np
import pytest

import fs_workloads as W
from oracle import oracle as O
from tests.gpu_helpers import oracle_problem

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


def _sample_nodes(P, k=24, seed=0):
    rng = np.random.default_rng(seed)
    nodes = set(rng.choice(P.n2, k, replace=False).tolist())
    nodes |= {0, P.nv - 1, P.nv, P.n2 - 1}          # corners, first/last edge
    nodes |= set(np.where(P.mask)[0][:3].tolist())  # Dirichlet rows
    nodes |= set(rng.choice(P.nv, 8, replace=False).tolist())  # pressure rows
    return sorted(nodes)


def _gather_rows(rp, rows, val_dev):
    out = {}
    for r in rows:
        a, b = int(rp[r]), int(rp[r + 1])
        out[r] = (a, b, val_dev[a:b].cpu().numpy())
    return out


@pytest.mark.parametrize("prec", [1, 0], ids=["fp32_refine", "fp64"])
@pytest.mark.parametrize("wl", [W.C2, W.C3], ids=lambda w: w.name)
def test_fullsize_sampled_rows_and_residual(fs, wl, prec):
    S = fs.Stepper.from_workload(wl, precision=prec, dofmap_arrays=True)
    try:
        info = S.info
        rp = info["rowptr"]
        col = info["col"]
        P = oracle_problem(wl.with_(jitter=wl.jitter))
        assert P.ndof == info["n_dof"]
        val = torch.zeros(info["nnz"], dtype=torch.float64, device="cuda")
        b = torch.zeros(info["n_dof"], dtype=torch.float64, device="cuda")
        fs.fs_assemble_step(S.prob, wl.dt, val, b)
        torch.cuda.synchronize()
        nodes = _sample_nodes(P)
        rows_ref, rhs_ref = O.assemble_rows(P, nodes)
        got = _gather_rows(rp, rows_ref.keys(), val)
        bh = b.cpu().numpy()
        for r, ref in rows_ref.items():
            a, e, v = got[r]
            cols = col[a:e]
            scale = max(abs(x) for x in ref.values())
            refv = np.array([ref.get(int(c), 0.0) for c in cols])
            # every oracle entry is in the GPU row and every GPU entry is matched
            assert set(ref) <= set(int(c) for c in cols)
            assert np.abs(v - refv).max() <= 1e-12 * scale, r
            assert abs(bh[r] - rhs_ref[r]) <= 1e-12 * max(abs(rhs_ref[r]), np.abs(bh).max() * 1e-6)
        # one solved step
        st = fs.fs_solve(S.prob)
        assert st["status"] == 0 and st["rel_res"] <= 1e-12
        x = torch.zeros(info["n_dof"], dtype=torch.float64, device="cuda")
        fs.fs_get_state(S.prob, x)
        t = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).cuda()
        rn, bn = fs.fs_csr_residual_norm(t(rp), t(col), val, x, b)
        assert rn <= 1e-12 * bn
        xh = x.cpu().numpy()
        for r, ref in rows_ref.items():
            ax = sum(v * xh[c] for c, v in ref.items())
            assert abs(rhs_ref[r] - ax) <= 1e-9 * max(1.0, abs(rhs_ref[r])) * max(1.0, np.abs(xh).max())
    finally:
        S.close()
