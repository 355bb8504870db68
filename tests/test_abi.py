"""CPU tests of the C-ABI library: it loads, exports every symbol that
include/fs.h declares, and its host-side mesh / DOF map / CSR pattern are
bit-exact against the oracle (no GPU needed: these calls touch no device)."""
import os
import re

import numpy as np
import pytest

import fs_workloads as W
from oracle import oracle as O
from tests.gpu_helpers import oracle_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fs():
    from paper_2605_25403_gb300 import build
    build.build()
    from paper_2605_25403_gb300 import fs as mod
    return mod


def test_library_exports_every_declared_symbol(fs):
    hdrs = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))
            if h.endswith(".h")]
    declared = set()
    for h in hdrs:
        txt = open(h).read()
        declared |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fs_[a-z_0-9]+)\s*\(",
                                   txt, re.M))
    assert declared, "no declarations found"
    import ctypes
    lib = ctypes.CDLL(fs.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(fs.EXPORTED) <= declared


@pytest.mark.parametrize("wl", [W.C1, W.cube(3), W.channel(16, 6), W.cube(2, jitter=0.2, seed=5),
                                W.unit_square(7, jitter=0.0)], ids=lambda w: w.name)
def test_dofmap_and_pattern_bitexact(fs, wl):
    mesh = fs.fs_mesh_create(wl.dim, wl.n, wl.lo, wl.hi, wl.jitter, wl.seed, wl.side_mask)
    try:
        d = fs.fs_dof_map(mesh)
    finally:
        fs.fs_mesh_destroy(mesh)
    P = oracle_problem(wl)
    rp, col, _ = O.assemble(wl.dim, P.nv, P.n2, P.c2d, P.p2xyz, None, 1.0, 1.0)
    assert d["n_dof"] == P.ndof == wl.ndof
    assert np.array_equal(d["coords"], P.coords)      # bit-exact FP64 coordinates
    assert np.array_equal(d["cell2dof"], P.c2d)
    assert np.array_equal(d["rowptr"], rp)
    assert np.array_equal(d["col"], col)
    assert np.array_equal(d["dirichlet"], P.mask)
    assert d["nnz"] == rp[-1]


def test_config_sizes(fs):
    """The documented sizes of the benchmark configurations."""
    for wl, ndof, nnz in ((W.C1, 659, 11415), (W.C2, 445411, 8329191)):
        mesh = fs.fs_mesh_create(wl.dim, wl.n, wl.lo, wl.hi, wl.jitter, wl.seed, wl.side_mask)
        d = fs.fs_dof_map(mesh, arrays=False)
        fs.fs_mesh_destroy(mesh)
        assert (d["n_dof"], d["nnz"]) == (ndof, nnz)


def test_invalid_arguments(fs):
    with pytest.raises(fs.FsError, match="INVALID_ARG"):
        fs.fs_mesh_create(4, (2, 2, 2), (0, 0, 0), (1, 1, 1))
    with pytest.raises(fs.FsError, match="INVALID_ARG"):
        fs.fs_mesh_create(2, (0, 2), (0, 0), (1, 1))
    with pytest.raises(fs.FsError, match="INVALID_ARG"):
        fs.fs_mesh_create(2, (2, 2), (0, 0), (1, 1), jitter=0.3)


def test_batch_mesh_is_union_of_instances(fs):
    """A batched mesh numbers the instances' meshes as one mesh: instance
    vertices consecutive, then all edge nodes, then cells; mapped back, each
    piece is bit-exact against the oracle's mesh of that instance."""
    wls = [W.unit_square(3), W.unit_square(5, jitter=0.1, seed=2), W.channel(6, 2)]
    mesh = fs.fs_mesh_create_batch([(w.dim, w.n, w.lo, w.hi, w.jitter, w.seed, w.side_mask)
                                    for w in wls])
    try:
        d = fs.fs_dof_map(mesh)
        off = fs.fs_mesh_instances(mesh)
    finally:
        fs.fs_mesh_destroy(mesh)
    nv_total = d["n_vert"]
    assert off.shape == (3, 6)
    for i, wl in enumerate(wls):
        P = oracle_problem(wl)
        v0, nv, e0, ne, c0, nc = (int(a) for a in off[i])
        assert (nv, ne, nc) == (P.nv, P.n2 - P.nv, P.cells.shape[0])
        assert np.array_equal(d["coords"][v0:v0 + nv], P.coords)
        g = d["cell2dof"][c0:c0 + nc].astype(np.int64)
        local = np.where(g < nv_total, g - v0, g - e0 + nv)
        assert np.array_equal(local, P.c2d)
        dmask = np.concatenate([d["dirichlet"][v0:v0 + nv], d["dirichlet"][e0:e0 + ne]])
        assert np.array_equal(dmask, P.mask)


def test_server_estimate_and_rejection(fs):
    """The admission estimate grows with the mesh and a request larger than
    the whole budget is refused at submission (host-side, no device work)."""
    small = fs.fs_server_estimate_bytes(W.unit_square(16))
    big = fs.fs_server_estimate_bytes(W.unit_square(64))
    cube = fs.fs_server_estimate_bytes(W.cube(16))
    assert 0 < small < big < cube
    srv = fs.Server(small // 2, 2)
    try:
        with pytest.raises(fs.FsError, match="OOM"):
            srv.submit(W.unit_square(16), 1, 0.0)
        assert srv.status() == {"queued": 0, "resident": 0, "bytes_reserved": 0}
    finally:
        srv.close()


def test_server_estimate_covers_history_and_dense_coarsest(fs):
    """A request of at least 100,000 P2 nodes keeps coarsest levels of up to
    3,500 rows in 3D and 2,000 in 2D (dense FP32 inverses, made through an
    FP64 workspace at set-up) and four previous states for the steps'
    starting guesses: the admission estimate counts them with the Krylov
    basis."""
    for wl, nc in ((W.C3, 3500), (W.C2, 2000)):
        est = fs.fs_server_estimate_bytes(wl)
        krylov = 4 * 61 * wl.ndof          # V (31 vectors) and Z (30), FP32
        history = 8 * 4 * wl.ndof          # previous states, FP64
        dense = (2 * 4 + 16) * nc ** 2     # two FP32 inverses + the set-up workspace
        assert est >= krylov + history + dense
