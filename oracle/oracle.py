"""The oracle: a plain, slow FP64 CPU reference for the Taylor-Hood P2/P1
backward-Euler Oseen step of the paper (Sec. 2.2.1, the Oseen linearisation
equation, with V_h = [P_2]^d, Q_h = P_1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  It shares no code with the CUDA path: the heavy loops live in
``fs_oracle.c`` (plain C, compiled by ``build()`` below) and the rest is
numpy.  Inputs come from ``fs_workloads`` (shapes and seeds only).

Parity pins (what fixes this code independently of itself) live in
``tests/test_oracle_pins.py``; the one function that has no pin is noted in
its docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fs_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

# problem ids (mirrors the enum in fs_oracle.c)
JOHN, STEADY_POLY, CHANNEL, CUBE, POLY_OSEEN, POLY_OSEEN_T, POLY3 = 0, 1, 2, 3, 4, 5, 6

_P = ctypes.POINTER
_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile fs_oracle.c into a shared library (gcc, -O2, no FP contraction
    so that mesh coordinates are bit-identical on x86 and Arm hosts)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_uniform.restype = _d
        L.or_uniform.argtypes = [_u64, _u64]
        L.or_mesh_nvert.restype = _i64
        L.or_mesh_nvert.argtypes = [_int, _P(_int)]
        L.or_mesh_ncell.restype = _i64
        L.or_mesh_ncell.argtypes = [_int, _P(_int)]
        L.or_mesh.restype = _int
        L.or_mesh.argtypes = [_int, _P(_int), _P(_d), _P(_d), _d, _u64,
                              _P(_d), _P(_i32)]
        L.or_dofmap.restype = _i64
        L.or_dofmap.argtypes = [_int, _i64, _i64, _P(_i32), _P(_i32), _P(_i32)]
        L.or_p2_coords.restype = None
        L.or_p2_coords.argtypes = [_int, _i64, _i64, _P(_d), _P(_i32), _P(_d)]
        L.or_dirichlet_mask.restype = None
        L.or_dirichlet_mask.argtypes = [_int, _P(_int), _int, _i64, _i64,
                                        _P(_i32), _P(ctypes.c_uint8)]
        L.or_exact_many.restype = None
        L.or_exact_many.argtypes = [_int, _int, _d, _d, _P(_d), _i64, _P(_d),
                                    _P(_d), _P(_d), _P(_d)]
        L.or_ref_tensors.restype = None
        L.or_ref_tensors.argtypes = [_int, _P(_d), _P(_d), _P(_d), _P(_d)]
        L.or_element.restype = _d
        L.or_element.argtypes = [_int, _P(_d), _P(_d), _d, _d] + [_P(_d)] * 7
        L.or_assemble_capacity.restype = _i64
        L.or_assemble_capacity.argtypes = [_int, _i64, _i64]
        L.or_assemble.restype = _i64
        L.or_assemble.argtypes = [_int, _i64, _i64, _i64, _P(_i32), _P(_d),
                                  _P(_d), _d, _d, _P(_i64), _P(_i32), _P(_d)]
        L.or_rhs.restype = None
        L.or_rhs.argtypes = [_int, _i64, _i64, _i64, _P(_i32), _P(_d), _P(_d),
                             _int, _d, _d, _P(_d), _d, _P(_d)]
        L.or_apply_bc.restype = None
        L.or_apply_bc.argtypes = [_int, _i64, _i64, _P(_i64), _P(_i32), _P(_d),
                                  _P(_d), _P(ctypes.c_uint8), _P(_d), _int, _d,
                                  _d, _P(_d), _int]
        L.or_spmv.restype = None
        L.or_spmv.argtypes = [_i64, _P(_i64), _P(_i32), _P(_d), _P(_d), _P(_d)]
        L.or_dense_solve.restype = _int
        L.or_dense_solve.argtypes = [_i64, _P(_d), _P(_d)]
        L.or_gmres_ilu0.restype = _int
        L.or_gmres_ilu0.argtypes = [_i64, _P(_i64), _P(_i32), _P(_d), _P(_d),
                                    _P(_d), _int, _int, _d, _P(_int), _P(_d)]
        _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data_as(_P(ctype))


def _ivec(n):
    return (_int * 3)(*(list(n) + [1] * (3 - len(n))))


def _dvec(v):
    return (_d * 3)(*(list(v) + [0.0] * (3 - len(v))))


# --------------------------------------------------------------------------
# Mesh, DOF map, boundary
# --------------------------------------------------------------------------
def uniform(seed: int, key: int) -> float:
    """SplitMix64(seed ^ key) >> 11, scaled to [0, 1)."""
    return lib().or_uniform(seed & (2**64 - 1), key & (2**64 - 1))


def mesh(dim, n, lo, hi, jitter=0.0, seed=0):
    """Structured simplicial mesh (2 triangles per square along v00-v11, or
    6 Kuhn tetrahedra per cube) with seeded jitter of interior vertices."""
    L = lib()
    nv = L.or_mesh_nvert(dim, _ivec(n))
    nc = L.or_mesh_ncell(dim, _ivec(n))
    coords = np.zeros((nv, dim), np.float64)
    cells = np.zeros((nc, dim + 1), np.int32)
    rc = L.or_mesh(dim, _ivec(n), _dvec(lo), _dvec(hi), float(jitter),
                   seed & (2**64 - 1), _ptr(coords, _d), _ptr(cells, _i32))
    if rc:
        raise ValueError("bad mesh description")
    return coords, cells


def dofmap(dim, nv, cells):
    """Edges (sorted unique vertex pairs) and the P2 cell-to-node map."""
    L = lib()
    nc = cells.shape[0]
    ne = L.or_dofmap(dim, nv, nc, _ptr(cells, _i32), None, None)
    edges = np.zeros((ne, 2), np.int32)
    nloc = 6 if dim == 2 else 10
    c2d = np.zeros((nc, nloc), np.int32)
    L.or_dofmap(dim, nv, nc, _ptr(cells, _i32), _ptr(edges, _i32),
                _ptr(c2d, _i32))
    return edges, c2d


def p2_coords(dim, coords, edges):
    out = np.zeros((coords.shape[0] + edges.shape[0], dim), np.float64)
    lib().or_p2_coords(dim, coords.shape[0], edges.shape[0],
                       _ptr(coords, _d), _ptr(edges, _i32), _ptr(out, _d))
    return out


def dirichlet_mask(dim, n, side_mask, nv, edges):
    mask = np.zeros(nv + edges.shape[0], np.uint8)
    lib().or_dirichlet_mask(dim, _ivec(n), side_mask, nv, edges.shape[0],
                            _ptr(edges, _i32), _ptr(mask, ctypes.c_uint8))
    return mask


def exact(problem, dim, t, nu, x, wconst=None):
    """Exact (u, p, f) at points x (npts x dim)."""
    x = np.ascontiguousarray(x, np.float64)
    npts = x.shape[0]
    u = np.zeros((npts, dim))
    p = np.zeros(npts)
    f = np.zeros((npts, dim))
    wc = None if wconst is None else np.ascontiguousarray(wconst, np.float64)
    lib().or_exact_many(problem, dim, float(t), float(nu), _ptr(wc, _d), npts,
                        _ptr(x, _d), _ptr(u, _d), _ptr(p, _d), _ptr(f, _d))
    return u, p, f


# --------------------------------------------------------------------------
# Element level
# --------------------------------------------------------------------------
def ref_tensors(dim):
    """Means over the simplex of the P2 basis products (exact)."""
    nloc, nb = (6, 3) if dim == 2 else (10, 4)
    M = np.zeros((nloc, nloc))
    K = np.zeros((nloc, nloc, nb, nb))
    N = np.zeros((nloc, nloc, nloc, nb))
    B = np.zeros((nb, nloc, nb))
    lib().or_ref_tensors(dim, _ptr(M, _d), _ptr(K, _d), _ptr(N, _d), _ptr(B, _d))
    return M, K, N, B


def element(dim, xv, w=None, mass_coef=0.0, nu=1.0):
    """Element matrices on one simplex (vertex coords (d+1) x d)."""
    nloc, nb = (6, 3) if dim == 2 else (10, 4)
    xv = np.ascontiguousarray(xv, np.float64)
    wv = None if w is None else np.ascontiguousarray(w, np.float64)
    out = {k: np.zeros((nloc, nloc)) for k in ("A", "M", "K", "N")}
    out["B"] = np.zeros((dim, nb, nloc))
    out["Kp"] = np.zeros((nb, nb))
    out["Mp"] = np.zeros((nb, nb))
    det = lib().or_element(dim, _ptr(xv, _d), _ptr(wv, _d), float(mass_coef),
                           float(nu), *(_ptr(out[k], _d) for k in
                                        ("A", "M", "K", "N", "B", "Kp", "Mp")))
    out["det"] = det
    return out


# --------------------------------------------------------------------------
# Global level
# --------------------------------------------------------------------------
def assemble(dim, nv, n2, c2d, p2xyz, w, mass_coef, nu):
    """Monolithic CSR (int64 rowptr, int32 col, f64 val) of the Oseen
    saddle-point matrix before boundary conditions."""
    L = lib()
    nc = c2d.shape[0]
    ndof = dim * n2 + nv
    cap = L.or_assemble_capacity(dim, nc, nv)
    rowptr = np.zeros(ndof + 1, np.int64)
    col = np.zeros(cap, np.int32)
    val = np.zeros(cap, np.float64)
    wv = None if w is None else np.ascontiguousarray(w, np.float64)
    nnz = L.or_assemble(dim, nv, n2, nc, _ptr(c2d, _i32), _ptr(p2xyz, _d),
                        _ptr(wv, _d), float(mass_coef), float(nu),
                        _ptr(rowptr, _i64), _ptr(col, _i32), _ptr(val, _d))
    return rowptr, col[:nnz].copy(), val[:nnz].copy()


def rhs(dim, nv, n2, c2d, p2xyz, u_prev, problem, t, nu, inv_dt, wconst=None):
    b = np.zeros(dim * n2 + nv)
    up = None if u_prev is None else np.ascontiguousarray(u_prev, np.float64)
    wc = None if wconst is None else np.ascontiguousarray(wconst, np.float64)
    lib().or_rhs(dim, nv, n2, c2d.shape[0], _ptr(c2d, _i32), _ptr(p2xyz, _d),
                 _ptr(up, _d), problem, float(t), float(nu), _ptr(wc, _d),
                 float(inv_dt), _ptr(b, _d))
    return b


def apply_bc(dim, nv, n2, rowptr, col, val, b, mask, p2xyz, problem, t, nu,
             pin_p0, wconst=None):
    wc = None if wconst is None else np.ascontiguousarray(wconst, np.float64)
    lib().or_apply_bc(dim, nv, n2, _ptr(rowptr, _i64), _ptr(col, _i32),
                      _ptr(val, _d), _ptr(b, _d), _ptr(mask, ctypes.c_uint8),
                      _ptr(p2xyz, _d), problem, float(t), float(nu),
                      _ptr(wc, _d), int(bool(pin_p0)))


def spmv(rowptr, col, val, x):
    y = np.zeros(rowptr.shape[0] - 1)
    x = np.ascontiguousarray(x, np.float64)
    lib().or_spmv(y.shape[0], _ptr(rowptr, _i64), _ptr(col, _i32),
                  _ptr(val, _d), _ptr(x, _d), _ptr(y, _d))
    return y


def csr_to_dense(rowptr, col, val):
    n = rowptr.shape[0] - 1
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    np.add.at(A, (rows, col), val)
    return A


def dense_solve(A, b):
    """Dense LU with partial pivoting (plain C loops)."""
    A = np.array(A, np.float64, order="C")
    x = np.array(b, np.float64)
    if lib().or_dense_solve(x.shape[0], _ptr(A, _d), _ptr(x, _d)):
        raise np.linalg.LinAlgError("singular matrix")
    return x


def gmres_ilu0(rowptr, col, val, b, x0=None, restart=200, maxit=20000,
               rtol=1e-14):
    n = rowptr.shape[0] - 1
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    it = _int(0)
    rr = _d(0)
    rc = lib().or_gmres_ilu0(n, _ptr(rowptr, _i64), _ptr(col, _i32),
                             _ptr(val, _d), _ptr(b, _d), _ptr(x, _d), restart,
                             maxit, rtol, ctypes.byref(it), ctypes.byref(rr))
    return x, rc, it.value, rr.value


def sparse_lu_solve(rowptr, col, val, b, max_refine=4):
    """Sparse direct solve: scipy's SuperLU factorisation (a library
    primitive, COLAMD column ordering) followed by FP64 iterative refinement
    x += LU^-1 (b - A x) with the residual from the oracle's own CSR product,
    for as long as the true residual keeps falling.  Returns (x, relres).
    Used for systems where ILU(0)-GMRES stagnates (the do-nothing channel)."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spl
    n = rowptr.shape[0] - 1
    b = np.ascontiguousarray(b, np.float64)
    A = sps.csr_matrix((val, col, rowptr), shape=(n, n)).tocsc()
    lu = spl.splu(A, permc_spec="COLAMD")
    del A
    x = lu.solve(b)
    bn = max(np.linalg.norm(b), 1e-300)
    rr = np.linalg.norm(b - spmv(rowptr, col, val, x)) / bn
    for _ in range(max_refine):
        r = b - spmv(rowptr, col, val, x)
        xn = x + lu.solve(r)
        rn = np.linalg.norm(b - spmv(rowptr, col, val, xn)) / bn
        if not rn < rr:
            break
        x, rr = xn, rn
    return x, rr


def solve(rowptr, col, val, b, x0=None, dense_max=1500, rtol=1e-14,
          method="auto"):
    """Exact-as-possible solve: dense LU for small systems, otherwise
    ILU(0)-GMRES to a true relative residual of rtol (a stagnation at the
    rounding floor within 100 rtol is accepted; where GMRES fails the sparse
    direct solve takes over); method="lu" takes the sparse direct solve with
    refinement directly."""
    n = rowptr.shape[0] - 1
    if n <= dense_max:
        return dense_solve(csr_to_dense(rowptr, col, val), b)
    if method == "lu":
        x, rr = sparse_lu_solve(rowptr, col, val, b)
        if not rr <= 100 * rtol:
            raise RuntimeError(f"oracle sparse LU residual {rr:.3e}")
        return x
    x, rc, it, rr = gmres_ilu0(rowptr, col, val, b, x0=x0, rtol=rtol)
    if rc == 3 and rr <= 100 * rtol:
        rc = 0
    if rc != 0:
        # ILU(0) stagnates on some saddle-point systems (do-nothing outflow,
        # convection-dominated flows): fall back to the direct solve
        x, rr = sparse_lu_solve(rowptr, col, val, b)
        if not rr <= 100 * rtol:
            raise RuntimeError(f"oracle solve failed: GMRES rc={rc} it={it}, "
                               f"sparse LU relres={rr:.3e}")
    return x


# --------------------------------------------------------------------------
# Quadrature for error norms: Stroud conical product rule built from
# Gauss-Jacobi nodes (Golub-Welsch), exact for degree 2q-1.
# --------------------------------------------------------------------------
def gauss_jacobi01(q, alpha):
    """Nodes/weights on [0,1] for the weight (1-s)^alpha (Golub-Welsch)."""
    a, b = float(alpha), 0.0
    k = np.arange(q, dtype=np.float64)
    # recurrence of monic Jacobi polynomials P^(a,b) on [-1,1]
    diag = np.zeros(q)
    off = np.zeros(max(q - 1, 0))
    for i in range(q):
        den = (2 * i + a + b) * (2 * i + a + b + 2)
        diag[i] = (b * b - a * a) / den if den != 0 else (b - a) / (a + b + 2)
    for i in range(1, q):
        num = 4 * i * (i + a) * (i + b) * (i + a + b)
        den = (2 * i + a + b) ** 2 * (2 * i + a + b + 1) * (2 * i + a + b - 1)
        off[i - 1] = np.sqrt(num / den)
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(J)
    mu0 = 2.0 ** (a + b + 1) / (a + b + 1)  # int_{-1}^{1} (1-x)^a dx for b=0
    w = mu0 * V[0, :] ** 2
    del k
    # map to [0,1]: s = (1+x)/2, (1-s) = (1-x)/2 -> factor 2^-(a+1)
    return (1 + x) / 2, w / 2.0 ** (a + b + 1)


def simplex_rule(dim, q=8):
    """Barycentric points (npts x (d+1)) and weights summing to 1/d!."""
    if dim == 2:
        s, ws = gauss_jacobi01(q, 1)
        t, wt = gauss_jacobi01(q, 0)
        S, T = np.meshgrid(s, t, indexing="ij")
        W = np.outer(ws, wt)
        xi, eta = S, T * (1 - S)
        lam = np.stack([1 - xi - eta, xi, eta], -1).reshape(-1, 3)
        return lam, W.reshape(-1)
    s, ws = gauss_jacobi01(q, 2)
    t, wt = gauss_jacobi01(q, 1)
    r, wr = gauss_jacobi01(q, 0)
    S, T, R = np.meshgrid(s, t, r, indexing="ij")
    W = ws[:, None, None] * wt[None, :, None] * wr[None, None, :]
    xi = S
    eta = T * (1 - S)
    zeta = R * (1 - S) * (1 - T)
    lam = np.stack([1 - xi - eta - zeta, xi, eta, zeta], -1).reshape(-1, 4)
    return lam, W.reshape(-1)


def p2_basis_values(dim, lam):
    """P2 basis (npts x nloc) at barycentric points, local order of the
    DOF map (vertices, then edges)."""
    edges = [(1, 2), (2, 0), (0, 1)] if dim == 2 else \
        [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    cols = [lam[:, v] * (2 * lam[:, v] - 1) for v in range(dim + 1)]
    cols += [4 * lam[:, a] * lam[:, b] for a, b in edges]
    return np.stack(cols, -1)


def l2_errors(dim, coords, cells, c2d, u, p, problem, t, nu, q=8,
              wconst=None):
    """||u - u_h||_{L2} and ||(p - p_h) - mean||_{L2} over the mesh."""
    lam, wq = simplex_rule(dim, q)
    phi = p2_basis_values(dim, lam)
    nb = dim + 1
    xv = coords[cells]                                     # nc x nb x d
    J = np.stack([xv[:, r + 1] - xv[:, 0] for r in range(dim)], -1)
    vol = np.abs(np.linalg.det(J)) * (1.0 if dim == 2 else 1.0)
    X = np.einsum("qr,crd->cqd", lam, xv)                  # nc x nq x d
    ue, pe, _ = exact(problem, dim, t, nu, X.reshape(-1, dim), wconst)
    ue = ue.reshape(X.shape)
    pe = pe.reshape(X.shape[:2])
    n2 = u.shape[0] // dim
    uh = np.stack([np.einsum("qi,ci->cq", phi, u[a * n2:(a + 1) * n2][c2d])
                   for a in range(dim)], -1)
    ph = np.einsum("qr,cr->cq", lam, p[cells])
    wts = vol[:, None] * wq[None, :]     # |det J| * w (w sums to 1/d!)
    eu = np.sqrt(np.sum(wts[..., None] * (uh - ue) ** 2))
    ep = ph - pe
    area = np.sum(wts)
    mean = np.sum(wts * ep) / area
    epn = np.sqrt(np.sum(wts * (ep - mean) ** 2))
    del nb
    return eu, epn


# --------------------------------------------------------------------------
# The time stepper
# --------------------------------------------------------------------------
@dataclass
class Problem:
    """One Taylor-Hood P2/P1 Oseen stepping problem on a structured mesh."""
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    problem: int
    nu: float
    dt: float
    jitter: float = 0.0
    seed: int = 0
    side_mask: int = 0x3F
    pin_p0: bool = True
    wconst: tuple | None = None     # constant convecting field (Oseen test)
    init: str = "exact"             # "exact": I_h u(0); "zero_interior"
    t0: float = 0.0
    state: dict = field(default_factory=dict)

    def __post_init__(self):
        d = self.dim
        self.coords, self.cells = mesh(d, self.n, self.lo, self.hi,
                                       self.jitter, self.seed)
        self.nv = self.coords.shape[0]
        self.edges, self.c2d = dofmap(d, self.nv, self.cells)
        self.n2 = self.nv + self.edges.shape[0]
        self.ndof = d * self.n2 + self.nv
        self.p2xyz = p2_coords(d, self.coords, self.edges)
        sm = self.side_mask & (0xF if d == 2 else 0x3F)
        self.mask = dirichlet_mask(d, self.n, sm, self.nv, self.edges)
        self.t = self.t0
        u0, p0, _ = exact(self.problem, d, self.t, self.nu, self.p2xyz,
                          self.wconst)
        if self.init == "zero_interior":
            u0 = u0 * self.mask[:, None]
        self.u = np.ascontiguousarray(u0.T.reshape(-1))   # component-blocked
        self.p = p0[:self.nv].copy()

    @property
    def x(self):
        return np.concatenate([self.u, self.p])

    def system(self, t_next, u_prev=None, w=None, mass_coef=None):
        """Assembled Oseen system (CSR, b) at t_next with BCs applied."""
        d = self.dim
        mc = 1.0 / self.dt if mass_coef is None else mass_coef
        up = self.u if u_prev is None else u_prev
        if w is None:
            if self.wconst is not None:
                w = np.repeat(np.asarray(self.wconst, np.float64), self.n2)
            else:
                w = up
        rp, col, val = assemble(d, self.nv, self.n2, self.c2d, self.p2xyz, w,
                                mc, self.nu)
        b = rhs(d, self.nv, self.n2, self.c2d, self.p2xyz,
                up if mc != 0.0 else None, self.problem, t_next, self.nu, mc,
                self.wconst)
        apply_bc(d, self.nv, self.n2, rp, col, val, b, self.mask, self.p2xyz,
                 self.problem, t_next, self.nu, self.pin_p0, self.wconst)
        return rp, col, val, b

    def step(self, rtol=1e-14, method="auto"):
        t1 = self.t + self.dt
        rp, col, val, b = self.system(t1)
        x = solve(rp, col, val, b, x0=self.x, rtol=rtol, method=method)
        self.u = x[:self.dim * self.n2].copy()
        self.p = x[self.dim * self.n2:].copy()
        self.t = t1
        return x

    def errors(self, q=8):
        return l2_errors(self.dim, self.coords, self.cells, self.c2d, self.u,
                         self.p, self.problem, self.t, self.nu, q,
                         self.wconst)


def steady_picard(prob: Problem, tol=1e-12, maxit=50):
    """Steady Oseen/Picard iteration (mass term dropped): w <- u_h until
    the update is below tol.  Used for the steady example of Sec. 3.3."""
    for it in range(maxit):
        rp, col, val, b = prob.system(prob.t, u_prev=None, w=prob.u,
                                      mass_coef=0.0)
        x = solve(rp, col, val, b, x0=prob.x)
        du = np.linalg.norm(x[:prob.dim * prob.n2] - prob.u)
        prob.u = x[:prob.dim * prob.n2].copy()
        prob.p = x[prob.dim * prob.n2:].copy()
        if du <= tol * max(1.0, np.linalg.norm(prob.u)):
            return it + 1
    return maxit


def picard_step(prob: Problem, tol=1e-12, maxit=50, method="auto"):
    """One backward-Euler step of the nonlinear system, solved by Picard
    iteration (Sec. 2.2.1: the convection term linearised around the latest
    iterate, ((u^k . grad) u^{k+1}, v); Sec. 3.3: iterate until the update is
    below tol).  The first iterate convects with u^n; every iterate keeps u^n
    in the load.  Stops when ||u^{k+1} - u^k|| <= tol max(1, ||u^{k+1}||).
    Returns the number of linear solves."""
    t1 = prob.t + prob.dt
    un = prob.u.copy()
    w = prob.u.copy()
    nvel = prob.dim * prob.n2
    for it in range(maxit):
        rp, col, val, b = prob.system(t1, u_prev=un, w=w)
        x = solve(rp, col, val, b, x0=prob.x, method=method)
        unew = x[:nvel]
        du = np.linalg.norm(unew - w)
        prob.u = unew.copy()
        prob.p = x[nvel:].copy()
        w = prob.u.copy()
        if du <= tol * max(1.0, np.linalg.norm(prob.u)):
            prob.t = t1
            return it + 1
    prob.t = t1
    return maxit


def _blocks(prob, w, mass_coef):
    """The blocks of the assembled (pre-boundary-condition) Oseen matrix as
    scipy CSR matrices: A (velocity-velocity, all components), the
    divergence block B (pressure rows, velocity columns; +B in the
    continuity rows, -B^T in the momentum rows) and, from the P1 element
    matrices, the pressure Laplacian K_p."""
    import scipy.sparse as sps
    d, n2, nv = prob.dim, prob.n2, prob.nv
    nvel = d * n2
    rp, col, val = assemble(d, nv, n2, prob.c2d, prob.p2xyz, w, mass_coef, prob.nu)
    K = sps.csr_matrix((val, col, rp), shape=(nvel + nv, nvel + nv))
    A = K[:nvel, :nvel].tocsr()
    B = K[nvel:, :nvel].tocsr()
    rows, cols, vals = [], [], []
    nb = d + 1
    for c in range(prob.c2d.shape[0]):
        g = prob.c2d[c, :nb]
        E = element(d, prob.p2xyz[g], None, 0.0, 1.0)
        for i in range(nb):
            for j in range(nb):
                rows.append(g[i])
                cols.append(g[j])
                vals.append(E["Kp"][i, j])
    Kp = sps.csr_matrix((vals, (rows, cols)), shape=(nv, nv))
    return A, B, Kp


def _solve_rows_replaced(Mat, rhs, fixed, values):
    """Solve Mat x = rhs with the rows of the `fixed` unknowns replaced by
    identity rows holding `values` (columns kept), by the sparse direct
    solve with FP64 refinement."""
    import scipy.sparse as sps
    Mat = sps.csr_matrix(Mat)
    keep = np.ones(Mat.shape[0])
    keep[fixed] = 0.0
    D = sps.diags(keep)
    Mat = (D @ Mat + sps.diags(1.0 - keep)).tocsr()
    Mat.sort_indices()
    b = rhs.copy()
    b[fixed] = values
    x, rr = sparse_lu_solve(Mat.indptr.astype(np.int64), Mat.indices.astype(np.int32),
                            Mat.data.astype(np.float64), b)
    if not rr <= 1e-12:
        raise RuntimeError(f"oracle IPCS sub-solve residual {rr:.3e}")
    return x


def ipcs_step(prob: Problem):
    """One step of the incremental pressure-correction scheme (Sec. 2.2.1,
    IPCS, density rho = 1), in the paper's three stages:

    1. tentative velocity u*: (u* - u^n)/dt + ((w . grad) u^n, v)
       + nu (grad u*, grad v) - (p^n, div v) = (f^{n+1}, v), with the
       convection explicit (w = u^n, or the constant field of the
       polynomial problems) and u* = u_D(t^{n+1}) on Dirichlet nodes;
    2. pressure increment dp = p^{n+1} - p^n:
       (grad dp, grad q) = -(1/dt) (div u*, q); the sign is the one that
       makes stage 3 remove the divergence (the printed right-hand side
       has the opposite sign, which contradicts the paper's own stage 3);
       the pinned vertex 0 takes dp = p_exact(x_0, t^{n+1}) - p^n(x_0);
    3. velocity correction: (u^{n+1} - u*, v)/dt = -(grad dp, v), i.e.
       M u^{n+1} = M u* + dt B^T dp on interior rows (v vanishes on the
       Dirichlet boundary, so (grad dp, v) = -(dp, div v)), u^{n+1} = u_D
       on Dirichlet nodes.

    Each stage's linear system is solved exactly (sparse direct).  Needs a
    velocity Dirichlet condition on the whole boundary and the pressure
    pin.  Returns the state vector."""
    d, n2, nv = prob.dim, prob.n2, prob.nv
    nvel = d * n2
    t1 = prob.t + prob.dt
    inv_dt = 1.0 / prob.dt
    w = (np.repeat(np.asarray(prob.wconst, np.float64), n2)
         if prob.wconst is not None else prob.u)
    Aosn, B, Kp = _blocks(prob, w, inv_dt)          # M/dt + nu K + N(w)
    Astk, _, _ = _blocks(prob, None, inv_dt)         # M/dt + nu K
    Mass, _, _ = _blocks(prob, None, 1.0)
    Mass = Mass - _blocks(prob, None, 0.0)[0]        # M (all components)
    Nw = Aosn - Astk
    # load: M (u^n / dt + I_h f^{n+1}), b_p = 0
    bfull = rhs(d, nv, n2, prob.c2d, prob.p2xyz, prob.u, prob.problem, t1, prob.nu,
                inv_dt, prob.wconst)
    dir_nodes = np.where(prob.mask)[0]
    dir_rows = np.concatenate([a * n2 + dir_nodes for a in range(d)])
    wc = None if prob.wconst is None else np.asarray(prob.wconst, np.float64)
    ue, _, _ = exact(prob.problem, d, t1, prob.nu, prob.p2xyz[dir_nodes], wc)
    dir_vals = np.concatenate([ue[:, a] for a in range(d)])
    # stage 1
    r1 = bfull[:nvel] - Nw @ prob.u + B.T @ prob.p
    ustar = _solve_rows_replaced(Astk, r1, dir_rows, dir_vals)
    # stage 2
    r2 = -inv_dt * (B @ ustar)
    fixed, fval = [], []
    if prob.pin_p0:
        _, pe, _ = exact(prob.problem, d, t1, prob.nu, prob.p2xyz[0:1], wc)
        fixed, fval = [0], [pe[0] - prob.p[0]]
    dp = _solve_rows_replaced(Kp, r2, np.array(fixed, int), np.array(fval))
    # stage 3
    r3 = Mass @ ustar + prob.dt * (B.T @ dp)
    unew = _solve_rows_replaced(Mass, r3, dir_rows, dir_vals)
    prob.u = unew
    prob.p = prob.p + dp
    prob.t = t1
    return prob.x


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)


def assemble_rows(prob: Problem, nodes, w=None, mass_coef=None, t_next=None):
    """Rows of the monolithic system (after boundary conditions) for a sample
    of P2 nodes, computed from the elements that contain them (paper
    Sec. 2.2.1, the Oseen equation; rows in the layout of ``assemble``):
    for every sampled node its d velocity rows, and for every sampled vertex
    also its pressure row (+B entries, the explicit diagonal, b_p = 0; the
    pinned row of vertex 0 becomes an identity row holding p_exact).
    Returns {global row: {global col: value}} and {global row: rhs}.
    Used to check full-size systems one row at a time; pinned against
    ``assemble`` + ``apply_bc`` + ``rhs`` on whole meshes."""
    d, n2, nv = prob.dim, prob.n2, prob.nv
    mc = 1.0 / prob.dt if mass_coef is None else mass_coef
    t1 = prob.t + prob.dt if t_next is None else t_next
    if w is None:
        w = (np.repeat(np.asarray(prob.wconst, np.float64), n2)
             if prob.wconst is not None else prob.u)
    nodes = np.asarray(nodes)
    want = set(int(i) for i in nodes)
    cells = np.where(np.isin(prob.c2d, nodes).any(1))[0]
    rows, rhs = {}, {}
    nb = d + 1
    wc = None if prob.wconst is None else np.asarray(prob.wconst, np.float64)
    for gi in sorted(want):
        if gi < nv:                       # pressure row: explicit diagonal
            r = d * n2 + gi
            rows[r] = {r: 0.0}
            rhs[r] = 0.0
    for c in cells:
        g = prob.c2d[c]
        xv = prob.p2xyz[g[:nb]]
        wl = np.stack([w[a * n2 + g] for a in range(d)], 1)
        E = element(d, xv, wl, mc, prob.nu)
        _, _, fj = exact(prob.problem, d, t1, prob.nu, prob.p2xyz[g], wc)
        for i, gi in enumerate(g):
            if int(gi) not in want:
                continue
            for a in range(d):
                r = a * n2 + int(gi)
                row = rows.setdefault(r, {})
                for j, gj in enumerate(g):
                    row[a * n2 + int(gj)] = row.get(a * n2 + int(gj), 0.0) + E["A"][i, j]
                for q in range(nb):
                    cp = d * n2 + int(g[q])
                    row[cp] = row.get(cp, 0.0) - E["B"][a, q, i]
                gl = (mc * prob.u[a * n2 + g] if mc != 0.0 else 0.0) + fj[:, a]
                rhs[r] = rhs.get(r, 0.0) + float(E["M"][i] @ gl)
        for q in range(nb):
            if int(g[q]) not in want:
                continue
            row = rows[d * n2 + int(g[q])]
            for a in range(d):
                for j, gj in enumerate(g):
                    cu = a * n2 + int(gj)
                    row[cu] = row.get(cu, 0.0) + E["B"][a, q, j]
    # boundary rows
    for gi in want:
        if prob.mask[gi]:
            u, _, _ = exact(prob.problem, d, t1, prob.nu, prob.p2xyz[gi:gi + 1], wc)
            for a in range(d):
                r = a * n2 + gi
                rows[r] = {cc: (1.0 if cc == r else 0.0) for cc in rows[r]}
                rhs[r] = u[0, a]
    if prob.pin_p0 and 0 in want:
        r = d * n2
        _, p, _ = exact(prob.problem, d, t1, prob.nu, prob.p2xyz[0:1], wc)
        rows[r] = {cc: (1.0 if cc == r else 0.0) for cc in rows[r]}
        rhs[r] = float(p[0])
    return rows, rhs
