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
    FS_PROBLEM_POLY_OSEEN, FS_PROBLEM_POLY_OSEEN_T, FS_PROBLEM_POLY3 = range(7)


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
                ("pin_pressure", _int), ("init", _int), ("wconst", _d * 3),
                ("deterministic", _int)]


class fs_solve_opts(ctypes.Structure):
    _fields_ = [("restart", _int), ("max_iter", _int), ("rtol", _d), ("inner_rtol", _d),
                ("max_refine", _int), ("use_graph", _int)]


class fs_solve_stats(ctypes.Structure):
    _fields_ = [("iters", _int), ("refinements", _int), ("status", _int), ("cycles", _int),
                ("rel_res", _d)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fs_picard_stats(ctypes.Structure):
    _fields_ = [("picard_iters", _int), ("krylov_iters", _int), ("status", _int),
                ("update", _d), ("rel_res", _d)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fs_ipcs_stats(ctypes.Structure):
    _fields_ = [("iters", _int * 3), ("status", _int), ("rel_res", _d * 3)]

    def as_dict(self):
        return {"iters": list(self.iters), "status": self.status,
                "rel_res": list(self.rel_res)}


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
_lib.fs_step_picard.argtypes = [_vp, _int, _P(fs_solve_opts), _d, _int, _P(fs_picard_stats)]
_lib.fs_solve_steady.argtypes = [_vp, _P(fs_solve_opts), _d, _int, _P(fs_picard_stats)]
_lib.fs_step_ipcs.argtypes = [_vp, _int, _d, _int, _P(fs_ipcs_stats)]
_lib.fs_problem_create_p3.argtypes = [_vp, _P(fs_problem_desc), _vp, _P(_vp)]
_lib.fs_problem_sizes.argtypes = [_vp, _P(_i64)]
_lib.fs_apply_operator.argtypes = [_vp, _vp, _vp]
_lib.fs_get_state.argtypes = [_vp, _vp, _int, _P(_d)]
_lib.fs_set_state.argtypes = [_vp, _vp, _int, _d]
_lib.fs_problem_device_bytes.restype = _i64
_lib.fs_problem_device_bytes.argtypes = [_vp]
_lib.fs_mesh_create_batch.restype = _int
_lib.fs_mesh_create_batch.argtypes = [_vp, _int, _P(_vp)]
_lib.fs_mesh_instances.restype = _int
_lib.fs_mesh_instances.argtypes = [_vp, _vp]
_lib.fs_problem_create_batch.restype = _int
_lib.fs_problem_create_batch.argtypes = [_vp, _vp, _int, _vp, _P(_vp)]
_lib.fs_step_begin.restype = _int
_lib.fs_step_begin.argtypes = [_vp, _int, _P(fs_solve_opts)]
_lib.fs_step_poll.restype = _int
_lib.fs_step_poll.argtypes = [_vp, _int, _P(_int)]
_lib.fs_instance_stats.restype = _int
_lib.fs_instance_stats.argtypes = [_vp, _vp]
class fs_server_desc(ctypes.Structure):
    _fields_ = [("hbm_budget", _i64), ("max_slots", _int), ("setup_threads", _int)]


class fs_schedule(ctypes.Structure):
    _fields_ = [("tail_rows_velocity", _i64), ("tail_rows_pressure", _i64),
                ("spmv_group", _int), ("smooth_group", _int), ("coarse_degree", _int),
                ("serial_launches", _int), ("persistent_precond", _int),
                ("fine_degree", _int), ("cheb_ratio", _int), ("schur", _int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fs_tune_report(ctypes.Structure):
    _fields_ = [("candidates", _int), ("default_ms", _d), ("best_ms", _d),
                ("spmv_default_ms", _d), ("spmv_best_ms", _d), ("best", fs_schedule),
                ("persistent_ms", _d)]

    def as_dict(self):
        return {"candidates": self.candidates, "default_ms": self.default_ms,
                "best_ms": self.best_ms, "spmv_default_ms": self.spmv_default_ms,
                "spmv_best_ms": self.spmv_best_ms, "best": self.best.as_dict(),
                "persistent_ms": self.persistent_ms}


class fs_request_result(ctypes.Structure):
    _fields_ = [("id", _i64), ("status", _int), ("nsteps", _int), ("iters", _int),
                ("arrival", _d), ("admitted", _d), ("started", _d), ("finished", _d),
                ("device_bytes", _i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib.fs_server_create.restype = _int
_lib.fs_server_create.argtypes = [_P(fs_server_desc), _P(_vp)]
_lib.fs_server_destroy.restype = _int
_lib.fs_server_destroy.argtypes = [_vp]
_lib.fs_server_submit.restype = _int
_lib.fs_server_submit.argtypes = [_vp, _P(fs_mesh_desc), _P(fs_problem_desc), _int, _d, _int,
                                  _P(_i64)]
_lib.fs_server_progress.restype = _int
_lib.fs_server_progress.argtypes = [_vp, _d, _P(_int)]
_lib.fs_server_pop_completed.restype = _int
_lib.fs_server_pop_completed.argtypes = [_vp, _vp, _int, _P(_int)]
_lib.fs_server_take_state.restype = _int
_lib.fs_server_take_state.argtypes = [_vp, _i64, _vp, _i64]
_lib.fs_server_status.restype = _int
_lib.fs_server_status.argtypes = [_vp, _P(_int), _P(_int), _P(_i64)]
_lib.fs_server_estimate_bytes.restype = _i64
_lib.fs_server_estimate_bytes.argtypes = [_P(fs_mesh_desc), _int]
_lib.fs_csr_residual_norm.restype = _int
_lib.fs_csr_residual_norm.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _P(_d), _vp]
_lib.fs_csr_residual_norm_noalloc.restype = _int
_lib.fs_csr_residual_norm_noalloc.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _P(_d), _vp]
_lib.fs_launch_count.restype = _i64
_lib.fs_launch_count.argtypes = []
_lib.fs_profile_kernel.restype = _int
_lib.fs_profile_kernel.argtypes = [_vp, _int, _int, _P(_d), _P(_d)]
_lib.fs_get_schedule.restype = _int
_lib.fs_get_schedule.argtypes = [_vp, _P(fs_schedule)]
_lib.fs_autotune_smoother.restype = _int
_lib.fs_autotune_smoother.argtypes = [_vp, _int, _P(ctypes.c_int32), _int, _P(_d), _P(_d),
                                      _P(fs_schedule)]
_lib.fs_set_schedule.restype = _int
_lib.fs_set_schedule.argtypes = [_vp, _P(fs_schedule)]
_lib.fs_autotune.restype = _int
_lib.fs_autotune.argtypes = [_vp, _int, _P(fs_tune_report)]
for _name in ("fs_mesh_create", "fs_mesh_destroy", "fs_dof_map", "fs_problem_create",
              "fs_problem_destroy", "fs_assemble_step", "fs_solve", "fs_step",
              "fs_apply_operator", "fs_get_state", "fs_set_state"):
    getattr(_lib, _name).restype = _int

EXPORTED = ["fs_mesh_create", "fs_mesh_destroy", "fs_dof_map", "fs_problem_create",
            "fs_problem_destroy", "fs_assemble_step", "fs_solve", "fs_step",
            "fs_apply_operator", "fs_get_state", "fs_set_state", "fs_problem_device_bytes",
            "fs_default_solve_opts", "fs_last_error", "fs_launch_count",
            "fs_profile_kernel", "fs_csr_residual_norm", "fs_csr_residual_norm_noalloc",
            "fs_mesh_create_batch", "fs_mesh_instances", "fs_problem_create_batch",
            "fs_step_begin", "fs_step_poll", "fs_instance_stats", "fs_server_create",
            "fs_server_destroy", "fs_server_submit", "fs_server_progress",
            "fs_server_pop_completed", "fs_server_take_state", "fs_server_status",
            "fs_server_estimate_bytes", "fs_get_schedule", "fs_set_schedule", "fs_autotune",
            "fs_autotune_smoother",
            "fs_step_picard", "fs_solve_steady", "fs_step_ipcs", "fs_problem_create_p3",
            "fs_problem_sizes"]
(FS_KERNEL_SPMV, FS_KERNEL_SPMV_FP64, FS_KERNEL_CHEB, FS_KERNEL_ASSEMBLE_CONV,
 FS_KERNEL_PRECOND, FS_KERNEL_CGS, FS_KERNEL_CGS_DOT, FS_KERNEL_CGS_UPD,
 FS_KERNEL_CGS_FIN) = range(9)
FS_PROFILE_COLD_L2 = 0x100


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
def _mesh_desc(dim, n, lo, hi, jitter=0.0, seed=0, dirichlet_sides=0x3F):
    d = fs_mesh_desc()
    d.dim = dim
    for a in range(3):
        d.n[a] = int(n[a]) if a < len(n) else 1
        d.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        d.hi[a] = float(hi[a]) if a < len(hi) else 1.0
    d.jitter = float(jitter)
    d.seed = int(seed) & (2**64 - 1)
    d.dirichlet_sides = int(dirichlet_sides)
    return d


def fs_mesh_create_batch(descs):
    """descs: list of (dim, n, lo, hi, jitter, seed, dirichlet_sides)."""
    arr = (fs_mesh_desc * len(descs))(*[_mesh_desc(*d) for d in descs])
    h = _vp()
    _check(_lib.fs_mesh_create_batch(arr, len(descs), ctypes.byref(h)), "fs_mesh_create_batch")
    return h


def fs_mesh_instances(mesh):
    """(count x 6) int64 array: first vertex, vertex count, first edge node,
    edge node count, first cell, cell count of every instance."""
    n = _lib.fs_mesh_instances(mesh, None)
    if n < 0:
        raise FsError(-n, "fs_mesh_instances")
    out = np.zeros((n, 6), np.int64)
    _lib.fs_mesh_instances(mesh, _hptr(out))
    return out


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


def _problem_desc(problem, nu, dt, t0=0.0, precision=FS_PREC_FP64, pin_pressure=1, init=0,
                  wconst=(0.0, 0.0, 0.0), deterministic=0):
    d = fs_problem_desc()
    d.problem, d.nu, d.dt, d.t0 = int(problem), float(nu), float(dt), float(t0)
    d.precision, d.pin_pressure, d.init = int(precision), int(pin_pressure), int(init)
    for a in range(3):
        d.wconst[a] = float(wconst[a]) if a < len(wconst) else 0.0
    d.deterministic = int(bool(deterministic))
    return d


def fs_problem_create_batch(mesh, descs, stream=None):
    """descs: list of keyword dicts for _problem_desc, one per instance."""
    arr = (fs_problem_desc * len(descs))(*[_problem_desc(**d) for d in descs])
    h = _vp()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(_lib.fs_problem_create_batch(mesh, arr, len(descs), s, ctypes.byref(h)),
           "fs_problem_create_batch")
    _state_sizes[h.value] = fs_dof_map(mesh, arrays=False)["n_dof"]
    _instance_counts[h.value] = len(descs)
    return h


def fs_step_begin(prob, nsteps, opts=None):
    o = opts if opts is not None else fs_default_solve_opts()
    _check(_lib.fs_step_begin(prob, int(nsteps), ctypes.byref(o)), "fs_step_begin")


def fs_step_poll(prob, wait=False, raise_on_error=True):
    """(done, status)."""
    done = _int(0)
    rc = _lib.fs_step_poll(prob, 1 if wait else 0, ctypes.byref(done))
    if raise_on_error and rc != FS_OK:
        raise FsError(rc, "fs_step_poll")
    return bool(done.value), rc


def fs_instance_stats(prob):
    n = _instance_counts.get(prob.value, 1)
    arr = (fs_solve_stats * n)()
    _check(_lib.fs_instance_stats(prob, arr), "fs_instance_stats")
    return [arr[i].as_dict() for i in range(n)]


_instance_counts = {}


def fs_problem_sizes(prob):
    """(velocity nodes per component, pressure nodes, n_dof)."""
    out = (_i64 * 3)()
    _check(_lib.fs_problem_sizes(prob, out), "fs_problem_sizes")
    return tuple(int(v) for v in out)


def fs_problem_create_p3(mesh, problem, nu, dt, t0=0.0, pin_pressure=1, init=0,
                         wconst=(0.0, 0.0, 0.0), stream=None):
    """A Taylor-Hood P3/P2 problem on a 2D mesh (stepped by fs_step_ipcs)."""
    d = _problem_desc(problem, nu, dt, t0, FS_PREC_FP64, pin_pressure, init, wconst)
    h = _vp()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(_lib.fs_problem_create_p3(mesh, ctypes.byref(d), s, ctypes.byref(h)),
           "fs_problem_create_p3")
    _state_sizes[h.value] = fs_problem_sizes(h)[2]
    _instance_counts[h.value] = 1
    return h


def fs_problem_create(mesh, problem, nu, dt, t0=0.0, precision=FS_PREC_FP64, pin_pressure=1,
                      init=0, wconst=(0.0, 0.0, 0.0), stream=None, deterministic=0):
    d = _problem_desc(problem, nu, dt, t0, precision, pin_pressure, init, wconst, deterministic)
    h = _vp()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(_lib.fs_problem_create(mesh, ctypes.byref(d), s, ctypes.byref(h)), "fs_problem_create")
    _state_sizes[h.value] = fs_dof_map(mesh, arrays=False)["n_dof"]
    _instance_counts[h.value] = int(_lib.fs_mesh_instances(mesh, None))
    return h


def fs_problem_destroy(prob):
    _state_sizes.pop(prob.value, None)
    _instance_counts.pop(prob.value, None)
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


def fs_step_picard(prob, nsteps, nl_tol=1e-10, max_picard=50, opts=None, raise_on_error=True):
    """nsteps time steps, each Picard-iterated to nl_tol; per-step stats."""
    stats = (fs_picard_stats * max(nsteps, 1))()
    o = opts if opts is not None else fs_default_solve_opts()
    rc = _lib.fs_step_picard(prob, int(nsteps), ctypes.byref(o), float(nl_tol), int(max_picard),
                             stats)
    if raise_on_error:
        _check(rc, "fs_step_picard")
    return [stats[i].as_dict() for i in range(nsteps)]


def fs_solve_steady(prob, nl_tol=1e-10, max_picard=50, opts=None, raise_on_error=True):
    """Picard iteration of a steady problem (created with dt = inf)."""
    st = fs_picard_stats()
    o = opts if opts is not None else fs_default_solve_opts()
    rc = _lib.fs_solve_steady(prob, ctypes.byref(o), float(nl_tol), int(max_picard),
                              ctypes.byref(st))
    if raise_on_error:
        _check(rc, "fs_solve_steady")
    return st.as_dict()


def fs_step_ipcs(prob, nsteps, rtol=1e-13, max_iter=20000, raise_on_error=True):
    """nsteps incremental pressure-correction steps; per-step stats."""
    stats = (fs_ipcs_stats * max(nsteps, 1))()
    rc = _lib.fs_step_ipcs(prob, int(nsteps), float(rtol), int(max_iter), stats)
    if raise_on_error:
        _check(rc, "fs_step_ipcs")
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


def fs_get_schedule(prob):
    sc = fs_schedule()
    _check(_lib.fs_get_schedule(prob, ctypes.byref(sc)), "fs_get_schedule")
    return sc.as_dict()


def fs_set_schedule(prob, tail_rows_velocity, tail_rows_pressure, spmv_group=0, smooth_group=0,
                    coarse_degree=0, serial_launches=0, persistent_precond=0, fine_degree=0,
                    cheb_ratio=0, schur=0):
    sc = fs_schedule(int(tail_rows_velocity), int(tail_rows_pressure), int(spmv_group),
                     int(smooth_group), int(coarse_degree), int(serial_launches),
                     int(persistent_precond), int(fine_degree), int(cheb_ratio), int(schur))
    _check(_lib.fs_set_schedule(prob, ctypes.byref(sc)), "fs_set_schedule")


def fs_autotune(prob, reps=10):
    """Times the preconditioner under every candidate schedule, installs
    the fastest and returns the report as a dict."""
    r = fs_tune_report()
    _check(_lib.fs_autotune(prob, int(reps), ctypes.byref(r)), "fs_autotune")
    return r.as_dict()


def fs_autotune_smoother(prob, candidates, nsteps=3):
    """Times `nsteps` steps from the current state under each candidate
    (cheb_ratio, coarse_degree, fine_degree) (0 keeps the installed value),
    installs the fastest and restores the state; returns the trials and the
    installed schedule."""
    n = len(candidates)
    flat = [int(v) for c in candidates for v in c]
    cc = (ctypes.c_int32 * (3 * n))(*flat)
    ms = (_d * n)()
    it = (_d * n)()
    best = fs_schedule()
    _check(_lib.fs_autotune_smoother(prob, int(nsteps), cc, n, ms, it, ctypes.byref(best)),
           "fs_autotune_smoother")
    return {"candidates": [list(c) for c in candidates], "ms_per_step": list(ms),
            "iters_per_step": list(it), "best": best.as_dict()}


def fs_tune_smoother(prob, nsteps=3, degrees=((2, 2), (1, 2), (2, 1), (1, 1)),
                     ratios=(4, 6, 8, 12, 16)):
    """The smoother picked field by field: the degree pairs (coarse, finest)
    at the installed interval, then the interval at the chosen degrees."""
    d = fs_autotune_smoother(prob, [(0, c, f) for c, f in degrees], nsteps) if degrees else None
    r = fs_autotune_smoother(prob, [(q, 0, 0) for q in ratios], nsteps) if ratios else None
    sc = fs_get_schedule(prob)
    return {"degrees": d, "ratios": r, "cheb_ratio": sc["cheb_ratio"],
            "coarse_degree": sc["coarse_degree"], "fine_degree": sc["fine_degree"]}


def fs_profile_kernel(prob, kernel, reps=20, cold=False):
    """(mean ms per launch, algorithmic bytes per launch) of one hot kernel;
    cold=True times each launch after the L2 was filled with other data."""
    ms, by = _d(), _d()
    kid = int(kernel) | (FS_PROFILE_COLD_L2 if cold else 0)
    _check(_lib.fs_profile_kernel(prob, kid, int(reps), ctypes.byref(ms),
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
         3: FS_PROBLEM_CUBE, 4: FS_PROBLEM_POLY_OSEEN, 5: FS_PROBLEM_POLY_OSEEN_T,
         6: FS_PROBLEM_POLY3}


@dataclass
class Stepper:
    mesh: object
    prob: object
    info: dict

    @classmethod
    def from_workload(cls, wl, precision=FS_PREC_FP64, stream=None, dofmap_arrays=False,
                      deterministic=False):
        mesh = fs_mesh_create(wl.dim, wl.n, wl.lo, wl.hi, wl.jitter, wl.seed, wl.side_mask)
        info = fs_dof_map(mesh, arrays=dofmap_arrays)
        prob = fs_problem_create(mesh, _KIND[wl.problem], wl.nu, wl.dt, 0.0, precision,
                                 1 if wl.pin_p0 else 0, 1 if wl.init == "zero_interior" else 0,
                                 wl.wconst or (0.0, 0.0, 0.0), stream, deterministic)
        return cls(mesh, prob, info)

    @classmethod
    def from_workload_p3(cls, wl, stream=None):
        """A Taylor-Hood P3/P2 problem on the workload's 2D mesh."""
        mesh = fs_mesh_create(wl.dim, wl.n, wl.lo, wl.hi, wl.jitter, wl.seed, wl.side_mask)
        prob = fs_problem_create_p3(mesh, _KIND[wl.problem], wl.nu, wl.dt, 0.0,
                                    1 if wl.pin_p0 else 0,
                                    1 if wl.init == "zero_interior" else 0,
                                    wl.wconst or (0.0, 0.0, 0.0), stream)
        n3, np_, ndof = fs_problem_sizes(prob)
        return cls(mesh, prob, {"n_p3": n3, "n_p2_pressure": np_, "n_dof": ndof})

    @classmethod
    def from_workloads(cls, wls, precision=FS_PREC_FP64, stream=None):
        """One batched problem over several independent workloads (same dim,
        problem kind and dt; nu may differ)."""
        mesh = fs_mesh_create_batch([(w.dim, w.n, w.lo, w.hi, w.jitter, w.seed, w.side_mask)
                                     for w in wls])
        info = fs_dof_map(mesh, arrays=False)
        prob = fs_problem_create_batch(mesh, [dict(
            problem=_KIND[w.problem], nu=w.nu, dt=w.dt, precision=precision,
            pin_pressure=1 if w.pin_p0 else 0, init=1 if w.init == "zero_interior" else 0,
            wconst=w.wconst or (0.0, 0.0, 0.0)) for w in wls], stream)
        info["instances"] = fs_mesh_instances(mesh)
        return cls(mesh, prob, info)

    def instance_state(self, x, i):
        """Instance i's entries of a union state vector, in its own layout
        [u_x | u_y | (u_z) | p]."""
        v0, nv, e0, ne = (int(a) for a in self.info["instances"][i][:4])
        n2, d = self.info["n_p2"], self.info["dim"]
        parts = []
        for c in range(d):
            parts += [x[c * n2 + v0:c * n2 + v0 + nv], x[c * n2 + e0:c * n2 + e0 + ne]]
        parts.append(x[d * n2 + v0:d * n2 + v0 + nv])
        return np.concatenate(parts)

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


# ---------------------------------------------------------------------------
# Continuous-batching request loop
# ---------------------------------------------------------------------------
class Server:
    """Thin wrapper of the fs_server_* calls (the scheduler itself is native)."""

    def __init__(self, hbm_budget, max_slots, setup_threads=4):
        d = fs_server_desc(int(hbm_budget), int(max_slots), int(setup_threads))
        self.h = _vp()
        _check(_lib.fs_server_create(ctypes.byref(d), ctypes.byref(self.h)), "fs_server_create")
        self.ndof = {}

    def submit(self, wl, nsteps, arrival, precision=FS_PREC_FP32_REFINE, keep_state=False,
               deterministic=False):
        md = _mesh_desc(wl.dim, wl.n, wl.lo, wl.hi, wl.jitter, wl.seed, wl.side_mask)
        pd = _problem_desc(_KIND[wl.problem], wl.nu, wl.dt, 0.0, precision,
                           1 if wl.pin_p0 else 0, 1 if wl.init == "zero_interior" else 0,
                           wl.wconst or (0.0, 0.0, 0.0), deterministic)
        rid = _i64()
        _check(_lib.fs_server_submit(self.h, ctypes.byref(md), ctypes.byref(pd), int(nsteps),
                                     float(arrival), 1 if keep_state else 0, ctypes.byref(rid)),
               "fs_server_submit")
        self.ndof[rid.value] = wl.ndof
        return rid.value

    def progress(self, now):
        n = _int(0)
        _check(_lib.fs_server_progress(self.h, float(now), ctypes.byref(n)), "fs_server_progress")
        return n.value

    def completed(self, max_n=4096):
        arr = (fs_request_result * max_n)()
        n = _int(0)
        _check(_lib.fs_server_pop_completed(self.h, arr, max_n, ctypes.byref(n)),
               "fs_server_pop_completed")
        return [arr[i].as_dict() for i in range(n.value)]

    def take_state(self, rid):
        x = np.zeros(self.ndof[rid])
        _check(_lib.fs_server_take_state(self.h, int(rid), _hptr(x), x.shape[0]),
               "fs_server_take_state")
        return x

    def status(self):
        q, r, b = _int(0), _int(0), _i64(0)
        _check(_lib.fs_server_status(self.h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)),
               "fs_server_status")
        return {"queued": q.value, "resident": r.value, "bytes_reserved": b.value}

    def close(self):
        if self.h:
            _lib.fs_server_destroy(self.h)
            self.h = None


def fs_server_estimate_bytes(wl, precision=FS_PREC_FP32_REFINE):
    md = _mesh_desc(wl.dim, wl.n, wl.lo, wl.hi, wl.jitter, wl.seed, wl.side_mask)
    return int(_lib.fs_server_estimate_bytes(ctypes.byref(md), int(precision)))
