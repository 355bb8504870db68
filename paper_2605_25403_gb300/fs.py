"""Thin ctypes binding of libfs (include/fs.h): argument marshalling only.

Every function keeps the C name.  Device buffers are torch CUDA tensors (their
data pointers are passed through); host buffers are numpy arrays.  There is no
fallback: importing this module fails when libfs.so has not been built, and
every call raises FsError on a non-zero status.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2605_25403_gb300.build` "
        "(the CUDA path has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

_i32, _i64, _u64, _d, _int = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
_P = ctypes.POINTER
_vp = ctypes.c_void_p

FS_OK = 0
STATUS = {0: "FS_OK", 1: "FS_ERR_INVALID_ARG", 2: "FS_ERR_INVALID_MESH", 3: "FS_ERR_OOM",
          4: "FS_ERR_CUDA", 5: "FS_ERR_NOT_CONVERGED", 6: "FS_ERR_NUMERIC",
          7: "FS_ERR_TIMEOUT", 8: "FS_ERR_BUSY", 9: "FS_ERR_UNSUPPORTED"}
FS_PREC_FP64, FS_PREC_FP32_REFINE = 0, 1
FS_PROBLEM_UNSTEADY_BENCH, FS_PROBLEM_STEADY_POLY, FS_PROBLEM_CHANNEL, FS_PROBLEM_CUBE, \
    FS_PROBLEM_POLY_OSEEN = range(5)


class FsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.fs_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")


class fs_mesh_desc(ctypes.Structure):
    _fields_ = [("dim", _int), ("n", _int * 3), ("lo", _d * 3), ("hi", _d * 3),
                ("jitter", _d), ("seed", _u64), ("dirichlet_sides", _int)]


class fs_dofmap_info(ctypes.Structure):
    _fields_ = [("dim", _int), ("nloc", _int), ("n_vert", _i64), ("n_edge", _i64),
                ("n_p2", _i64), ("n_cell", _i64), ("n_dof", _i64), ("nnz", _i64),
                ("nnz_a", _i64), ("nnz_b", _i64)]


class fs_problem_desc(ctypes.Structure):
    _fields_ = [("problem", _int), ("nu", _d), ("dt", _d), ("t0", _d), ("precision", _int),
                ("pin_pressure", _int), ("init", _int), ("wconst", _d * 3)]


class fs_solve_opts(ctypes.Structure):
    _fields_ = [("restart", _int), ("max_iter", _int), ("rtol", _d), ("inner_rtol", _d),
                ("max_refine", _int), ("use_graph", _int)]


class fs_solve_stats(ctypes.Structure):
    _fields_ = [("iters", _int), ("refinements", _int), ("status", _int), ("cycles", _int),
                ("rel_res", _d)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib.fs_last_error.restype = ctypes.c_char_p
_lib.fs_last_error.argtypes = []
_lib.fs_default_solve_opts.restype = None
_lib.fs_default_solve_opts.argtypes = [_P(fs_solve_opts)]
_lib.fs_mesh_create.argtypes = [_P(fs_mesh_desc), _P(_vp)]
_lib.fs_mesh_destroy.argtypes = [_vp]
_lib.fs_dof_map.argtypes = [_vp, _P(fs_dofmap_info), _vp, _vp, _vp, _vp, _vp]
_lib.fs_problem_create.argtypes = [_vp, _P(fs_problem_desc), _vp, _P(_vp)]
_lib.fs_problem_destroy.argtypes = [_vp]
_lib.fs_assemble_step.argtypes = [_vp, _d, _vp, _vp]
_lib.fs_solve.argtypes = [_vp, _P(fs_solve_opts), _vp, _P(fs_solve_stats)]
_lib.fs_step.argtypes = [_vp, _int, _P(fs_solve_opts), _P(fs_solve_stats)]
_lib.fs_apply_operator.argtypes = [_vp, _vp, _vp]
_lib.fs_get_state.argtypes = [_vp, _vp, _int, _P(_d)]
_lib.fs_set_state.argtypes = [_vp, _vp, _int, _d]
_lib.fs_problem_device_bytes.restype = _i64
_lib.fs_problem_device_bytes.argtypes = [_vp]
_lib.fs_csr_residual_norm.restype = _int
_lib.fs_csr_residual_norm.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _P(_d), _vp]
_lib.fs_csr_residual_norm_noalloc.restype = _int
_lib.fs_csr_residual_norm_noalloc.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _P(_d), _vp]
_lib.fs_launch_count.restype = _i64
_lib.fs_launch_count.argtypes = []
_lib.fs_profile_kernel.restype = _int
_lib.fs_profile_kernel.argtypes = [_vp, _int, _int, _P(_d), _P(_d)]
for _name in ("fs_mesh_create", "fs_mesh_destroy", "fs_dof_map", "fs_problem_create",
              "fs_problem_destroy", "fs_assemble_step", "fs_solve", "fs_step",
              "fs_apply_operator", "fs_get_state", "fs_set_state"):
    getattr(_lib, _name).restype = _int

EXPORTED = ["fs_mesh_create", "fs_mesh_destroy", "fs_dof_map", "fs_problem_create",
            "fs_problem_destroy", "fs_assemble_step", "fs_solve", "fs_step",
            "fs_apply_operator", "fs_get_state", "fs_set_state", "fs_problem_device_bytes",
            "fs_default_solve_opts", "fs_last_error", "fs_launch_count",
            "fs_profile_kernel", "fs_csr_residual_norm", "fs_csr_residual_norm_noalloc"]
FS_KERNEL_SPMV, FS_KERNEL_SPMV_FP64, FS_KERNEL_CHEB, FS_KERNEL_ASSEMBLE_CONV = range(4)


def _check(rc, where):
    if rc != FS_OK:
        raise FsError(rc, where)


def _dptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
def fs_mesh_create(dim, n, lo, hi, jitter=0.0, seed=0, dirichlet_sides=0x3F):
    d = fs_mesh_desc()
    d.dim = dim
    for a in range(3):
        d.n[a] = int(n[a]) if a < len(n) else 1
        d.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        d.hi[a] = float(hi[a]) if a < len(hi) else 1.0
    d.jitter = float(jitter)
    d.seed = int(seed) & (2**64 - 1)
    d.dirichlet_sides = int(dirichlet_sides)
    h = _vp()
    _check(_lib.fs_mesh_create(ctypes.byref(d), ctypes.byref(h)), "fs_mesh_create")
    return h


def fs_mesh_destroy(mesh):
    _check(_lib.fs_mesh_destroy(mesh), "fs_mesh_destroy")


def fs_dof_map(mesh, arrays=True):
    info = fs_dofmap_info()
    _check(_lib.fs_dof_map(mesh, ctypes.byref(info), None, None, None, None, None), "fs_dof_map")
    out = {k: getattr(info, k) for k, _ in info._fields_}
    if arrays:
        coords = np.zeros((info.n_vert, info.dim))
        c2d = np.zeros((info.n_cell, info.nloc), np.int32)
        rp = np.zeros(info.n_dof + 1, np.int64)
        col = np.zeros(info.nnz, np.int32)
        dirich = np.zeros(info.n_p2, np.uint8)
        _check(_lib.fs_dof_map(mesh, ctypes.byref(info), _hptr(coords), _hptr(c2d), _hptr(rp),
                               _hptr(col), _hptr(dirich)), "fs_dof_map")
        out.update(coords=coords, cell2dof=c2d, rowptr=rp, col=col, dirichlet=dirich)
    return out


def fs_default_solve_opts(**kw):
    o = fs_solve_opts()
    _lib.fs_default_solve_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def fs_problem_create(mesh, problem, nu, dt, t0=0.0, precision=FS_PREC_FP64, pin_pressure=1,
                      init=0, wconst=(0.0, 0.0, 0.0), stream=None):
    d = fs_problem_desc()
    d.problem, d.nu, d.dt, d.t0 = int(problem), float(nu), float(dt), float(t0)
    d.precision, d.pin_pressure, d.init = int(precision), int(pin_pressure), int(init)
    for a in range(3):
        d.wconst[a] = float(wconst[a]) if a < len(wconst) else 0.0
    h = _vp()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(_lib.fs_problem_create(mesh, ctypes.byref(d), s, ctypes.byref(h)), "fs_problem_create")
    _state_sizes[h.value] = fs_dof_map(mesh, arrays=False)["n_dof"]
    return h


def fs_problem_destroy(prob):
    _state_sizes.pop(prob.value, None)
    _check(_lib.fs_problem_destroy(prob), "fs_problem_destroy")


def fs_problem_device_bytes(prob):
    return int(_lib.fs_problem_device_bytes(prob))


def fs_assemble_step(prob, t_next, val_out=None, b_out=None):
    _check(_lib.fs_assemble_step(prob, float(t_next), _dptr(val_out), _dptr(b_out)),
           "fs_assemble_step")


def fs_solve(prob, opts=None, x=None, raise_on_error=True):
    st = fs_solve_stats()
    o = opts if opts is not None else fs_default_solve_opts()
    rc = _lib.fs_solve(prob, ctypes.byref(o), _dptr(x), ctypes.byref(st))
    if raise_on_error:
        _check(rc, "fs_solve")
    return st.as_dict()


def fs_step(prob, nsteps, opts=None, raise_on_error=True):
    stats = (fs_solve_stats * max(nsteps, 1))()
    o = opts if opts is not None else fs_default_solve_opts()
    rc = _lib.fs_step(prob, int(nsteps), ctypes.byref(o), stats)
    if raise_on_error:
        _check(rc, "fs_step")
    return [stats[i].as_dict() for i in range(nsteps)]


def fs_apply_operator(prob, x, y):
    _check(_lib.fs_apply_operator(prob, _dptr(x), _dptr(y)), "fs_apply_operator")


def fs_get_state(prob, out=None):
    """Host copy (numpy) of the state when out is None, else into the CUDA
    tensor `out`.  Returns (x, t)."""
    t = _d()
    if out is None:
        x = np.zeros(_state_len(prob))
        _check(_lib.fs_get_state(prob, _hptr(x), 1, ctypes.byref(t)), "fs_get_state")
        return x, t.value
    _check(_lib.fs_get_state(prob, _dptr(out), 0, ctypes.byref(t)), "fs_get_state")
    return out, t.value


_state_sizes = {}


def _state_len(prob):
    return _state_sizes[prob.value]


def fs_csr_residual_norm(rowptr, col, val, x, b, stream=None):
    """(||b - A x||_2, ||b||_2) of a monolithic CSR system held in CUDA
    tensors (rowptr int64, col int32, val/x/b float64)."""
    out = (_d * 2)()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(_lib.fs_csr_residual_norm(rowptr.numel() - 1, _dptr(rowptr), _dptr(col), _dptr(val),
                                     _dptr(x), _dptr(b), out, s), "fs_csr_residual_norm")
    return out[0], out[1]


def fs_csr_residual_norm_noalloc(rowptr, col, val, x, b, stream=None, n=None):
    """Same as fs_csr_residual_norm through the allocation-free entry point
    (static device scratch; for callers that cannot allocate).  `n`
    overrides the row count (only to exercise the size check)."""
    out = (_d * 2)()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    rows = rowptr.numel() - 1 if n is None else int(n)
    _check(_lib.fs_csr_residual_norm_noalloc(rows, _dptr(rowptr), _dptr(col), _dptr(val),
                                             _dptr(x), _dptr(b), out, s),
           "fs_csr_residual_norm_noalloc")
    return out[0], out[1]


def fs_launch_count():
    return int(_lib.fs_launch_count())


def fs_profile_kernel(prob, kernel, reps=20):
    """(mean ms per launch, algorithmic bytes per launch) of one hot kernel."""
    ms, by = _d(), _d()
    _check(_lib.fs_profile_kernel(prob, int(kernel), int(reps), ctypes.byref(ms),
                                  ctypes.byref(by)), "fs_profile_kernel")
    return ms.value, by.value


def fs_set_state(prob, x, t):
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, np.float64)
        _check(_lib.fs_set_state(prob, _hptr(x), 1, float(t)), "fs_set_state")
    else:
        _check(_lib.fs_set_state(prob, _dptr(x), 0, float(t)), "fs_set_state")


# ---------------------------------------------------------------------------
# Convenience wrapper: one problem built from a workload description
# ---------------------------------------------------------------------------
_KIND = {0: FS_PROBLEM_UNSTEADY_BENCH, 1: FS_PROBLEM_STEADY_POLY, 2: FS_PROBLEM_CHANNEL,
         3: FS_PROBLEM_CUBE, 4: FS_PROBLEM_POLY_OSEEN}


@dataclass
class Stepper:
    mesh: object
    prob: object
    info: dict

    @classmethod
    def from_workload(cls, wl, precision=FS_PREC_FP64, stream=None, dofmap_arrays=False):
        mesh = fs_mesh_create(wl.dim, wl.n, wl.lo, wl.hi, wl.jitter, wl.seed, wl.side_mask)
        info = fs_dof_map(mesh, arrays=dofmap_arrays)
        prob = fs_problem_create(mesh, _KIND[wl.problem], wl.nu, wl.dt, 0.0, precision,
                                 1 if wl.pin_p0 else 0, 1 if wl.init == "zero_interior" else 0,
                                 wl.wconst or (0.0, 0.0, 0.0), stream)
        return cls(mesh, prob, info)

    def state(self):
        return fs_get_state(self.prob)

    def close(self):
        if self.prob is not None:
            fs_problem_destroy(self.prob)
            self.prob = None
        if self.mesh is not None:
            fs_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
