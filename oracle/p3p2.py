"""The oracle for the Taylor-Hood P3/P2 pair on triangles (paper Sec. 4.1,
the P3-P2 convergence table: higher-order spaces solved by IPCS), in plain
numpy/scipy and FP64.

TEST INFRASTRUCTURE ONLY: only ``tests/`` may import this module.  It shares
no code with the CUDA path.  Element integrals are exact: every integrand is
expanded in barycentric monomials and integrated by
    int_K l0^a l1^b l2^c = a! b! c! 2! |K| / (a + b + c + 2)!.
Meshes, the P2 DOF map and the manufactured fields come from ``oracle.py``.

Numbering (reading 18 of the design notes): velocity P3 nodes are the
vertices, then two nodes per edge in the lexicographic order of the edges
(the one nearer the edge's smaller vertex id first), then one interior node
per cell; pressure P2 nodes are the vertices, then one node per edge (the P2
numbering of ``oracle.py``).  Local P3 order: vertices 0, 1, 2; for each of
the edges (1,2), (2,0), (0,1) the node nearer its first vertex, then the
other; the interior node.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from oracle import oracle as O

EDGES = [(1, 2), (2, 0), (0, 1)]


# --------------------------------------------------------------------------
# barycentric polynomials: {(a0, a1, a2): coefficient}
# --------------------------------------------------------------------------
def _mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
            out[e] = out.get(e, 0) + ca * cb
    return {e: c for e, c in out.items() if c != 0}


def _add(*ps):
    out = {}
    for p in ps:
        for e, c in p.items():
            out[e] = out.get(e, 0) + c
    return {e: c for e, c in out.items() if c != 0}


def _scale(p, s):
    return {e: c * s for e, c in p.items()}


def _lam(r):
    e = [0, 0, 0]
    e[r] = 1
    return {tuple(e): Fraction(1)}


def _const(c):
    return {(0, 0, 0): Fraction(c)}


def _dlam(p, r):
    """d p / d lambda_r."""
    out = {}
    for e, c in p.items():
        if e[r] > 0:
            f = list(e)
            f[r] -= 1
            out[tuple(f)] = out.get(tuple(f), 0) + c * e[r]
    return out


def _mean(p):
    """Integral over the simplex divided by its area (exact, rational)."""
    s = Fraction(0)
    for (a, b, c), v in p.items():
        s += v * Fraction(math.factorial(a) * math.factorial(b) * math.factorial(c) * 2,
                          math.factorial(a + b + c + 2))
    return s


def p3_basis():
    """The ten P3 Lagrange functions in the local order of the module."""
    L = [_lam(r) for r in range(3)]
    out = []
    for v in range(3):   # (1/2) l (3l - 1)(3l - 2)
        t = _mul(_mul(L[v], _add(_scale(L[v], 3), _const(-1))),
                 _add(_scale(L[v], 3), _const(-2)))
        out.append(_scale(t, Fraction(1, 2)))
    for a, b in EDGES:   # (9/2) l_a l_b (3 l_a - 1), then (3 l_b - 1)
        for near in (a, b):
            t = _mul(_mul(L[a], L[b]), _add(_scale(L[near], 3), _const(-1)))
            out.append(_scale(t, Fraction(9, 2)))
    out.append(_scale(_mul(_mul(L[0], L[1]), L[2]), 27))
    return out


def p2_basis():
    L = [_lam(r) for r in range(3)]
    out = [_mul(L[v], _add(_scale(L[v], 2), _const(-1))) for v in range(3)]
    out += [_scale(_mul(L[a], L[b]), 4) for a, b in EDGES]
    return out


def _node_bary():
    """Barycentric coordinates of the P3 nodes (local order)."""
    pts = [tuple(1.0 if r == v else 0.0 for r in range(3)) for v in range(3)]
    for a, b in EDGES:
        for near in (a, b):
            far = b if near == a else a
            l = [0.0, 0.0, 0.0]
            l[near], l[far] = 2.0 / 3.0, 1.0 / 3.0
            pts.append(tuple(l))
    pts.append((1.0 / 3.0,) * 3)
    return np.array(pts)


class _Ref:
    """Reference integrals (means over the simplex), computed once."""

    def __init__(self):
        P3, P2 = p3_basis(), p2_basis()
        self.mass = np.array([[float(_mean(_mul(a, b))) for b in P3] for a in P3])
        d3 = [[_dlam(f, r) for r in range(3)] for f in P3]
        d2 = [[_dlam(f, r) for r in range(3)] for f in P2]
        # stiff[i, j, r, s] = mean(d_r phi_i d_s phi_j)
        self.stiff = np.array([[[[float(_mean(_mul(d3[i][r], d3[j][s]))) for s in range(3)]
                                 for r in range(3)] for j in range(10)] for i in range(10)])
        # conv[i, k, j, r] = mean(phi_i phi_k d_r phi_j)
        pk = [[_mul(P3[i], P3[k]) for k in range(10)] for i in range(10)]
        self.conv = np.array([[[[float(_mean(_mul(pk[i][k], d3[j][r]))) for r in range(3)]
                                for j in range(10)] for k in range(10)] for i in range(10)])
        # div[q, j, r] = mean(psi_q d_r phi_j)
        self.div = np.array([[[float(_mean(_mul(P2[q], d3[j][r]))) for r in range(3)]
                              for j in range(10)] for q in range(6)])
        # pstiff[q, s, r, t] = mean(d_r psi_q d_t psi_s)
        self.pstiff = np.array([[[[float(_mean(_mul(d2[q][r], d2[s][t]))) for t in range(3)]
                                  for r in range(3)] for s in range(6)] for q in range(6)])


_REF = None


def ref():
    global _REF
    if _REF is None:
        _REF = _Ref()
    return _REF


def element(xv, w=None, mass_coef=0.0, nu=1.0):
    """P3/P2 element matrices on one triangle (vertex coordinates 3 x 2):
    M, K, N(w) (10 x 10; w: P3 nodal values 10 x 2, or None), A = mass_coef M
    + nu K + N(w), B (2 x 6 x 10, B[c, q, j] = int psi_q d_c phi_j) and Kp
    (6 x 6 P2 stiffness).  Returns a dict (and |K| as "area")."""
    R = ref()
    xv = np.asarray(xv, np.float64)
    J = np.stack([xv[1] - xv[0], xv[2] - xv[0]], 1)          # columns e1, e2
    det = np.linalg.det(J)
    Ji = np.linalg.inv(J)
    g = np.zeros((3, 2))
    g[1:] = Ji                                              # grad l_1, grad l_2
    g[0] = -g[1] - g[2]
    area = abs(det) / 2.0
    G = g @ g.T                                             # grad l_r . grad l_s
    M = area * R.mass
    K = area * np.einsum("ijrs,rs->ij", R.stiff, G)
    N = np.zeros((10, 10))
    if w is not None:
        cw = np.asarray(w) @ g.T                            # (w_k . grad l_r)
        N = area * np.einsum("ikjr,kr->ij", R.conv, cw)
    B = area * np.einsum("qjr,rc->cqj", R.div, g)
    Kp = area * np.einsum("qsrt,rt->qs", R.pstiff, G)
    return {"M": M, "K": K, "N": N, "A": mass_coef * M + nu * K + N, "B": B, "Kp": Kp,
            "area": area}


# --------------------------------------------------------------------------
# DOF maps
# --------------------------------------------------------------------------
def p3_dofmap(coords, cells, edges, c2d2):
    """P3 cell-to-node map (ncell x 10), node coordinates and the number of
    nodes, from the P2 map (vertices, then edges ranked lexicographically)."""
    nv, ne, nc = coords.shape[0], edges.shape[0], cells.shape[0]
    c2d3 = np.zeros((nc, 10), np.int64)
    c2d3[:, :3] = cells
    for le, (a, b) in enumerate(EDGES):
        r = c2d2[:, 3 + le] - nv                       # edge rank
        va, vb = cells[:, a], cells[:, b]
        lo_first = va < vb                             # node nearer a is the one
        c2d3[:, 3 + 2 * le] = nv + 2 * r + np.where(lo_first, 0, 1)
        c2d3[:, 4 + 2 * le] = nv + 2 * r + np.where(lo_first, 1, 0)
    c2d3[:, 9] = nv + 2 * ne + np.arange(nc)
    n3 = nv + 2 * ne + nc
    xyz = np.zeros((n3, 2))
    lam = _node_bary()
    for c in range(nc):
        X = coords[cells[c]]
        xyz[c2d3[c]] = lam @ X
    return c2d3, xyz, n3


@dataclass
class Problem3:
    """A P3/P2 problem on the structured triangle mesh of oracle.py, all
    sides Dirichlet, pressure vertex 0 pinned."""
    n: tuple
    problem: int
    nu: float
    dt: float
    jitter: float = 0.0
    seed: int = 0
    wconst: tuple | None = None
    t0: float = 0.0
    state: dict = field(default_factory=dict)

    def __post_init__(self):
        self.coords, self.cells = O.mesh(2, self.n, (0.0, 0.0), (1.0, 1.0), self.jitter,
                                         self.seed)
        self.nv = self.coords.shape[0]
        self.edges, self.c2d2 = O.dofmap(2, self.nv, self.cells)
        self.np_ = self.nv + self.edges.shape[0]              # P2 pressure nodes
        self.c2d3, self.xyz3, self.n3 = p3_dofmap(self.coords, self.cells, self.edges,
                                                  self.c2d2)
        mask2 = O.dirichlet_mask(2, self.n, 0xF, self.nv, self.edges)
        m3 = np.zeros(self.n3, np.uint8)
        m3[:self.nv] = mask2[:self.nv]
        ne = self.edges.shape[0]
        m3[self.nv:self.nv + 2 * ne] = np.repeat(mask2[self.nv:], 2)
        self.mask = m3
        self.ndof = 2 * self.n3 + self.np_
        self.t = self.t0
        u0, p0 = self.exact_state(self.t)
        self.u, self.p = u0, p0

    def _wc(self):
        return None if self.wconst is None else np.asarray(self.wconst, np.float64)

    def exact_state(self, t):
        u, _, _ = O.exact(self.problem, 2, t, self.nu, self.xyz3, self._wc())
        p2xyz = O.p2_coords(2, self.coords, self.edges)
        _, p, _ = O.exact(self.problem, 2, t, self.nu, p2xyz, self._wc())
        return np.ascontiguousarray(u.T.reshape(-1)), p

    @property
    def x(self):
        return np.concatenate([self.u, self.p])

    def _geometry(self):
        """Per-cell barycentric gradients (nc x 3 x 2) and areas."""
        if "geom" not in self.state:
            xv = self.coords[self.cells]
            J = np.stack([xv[:, 1] - xv[:, 0], xv[:, 2] - xv[:, 0]], -1)
            g = np.zeros((xv.shape[0], 3, 2))
            g[:, 1:] = np.linalg.inv(J)
            g[:, 0] = -g[:, 1] - g[:, 2]
            self.state["geom"] = (g, np.abs(np.linalg.det(J)) / 2.0)
        return self.state["geom"]

    def blocks(self, w, mass_coef):
        """Scalar velocity block (mass_coef M + nu K + N(w)), the mass M, the
        divergence block B (P2 rows, 2 n3 columns) and the P2 Laplacian, as
        scipy CSR matrices (no boundary conditions).  The element matrices
        of ``element`` for every cell at once."""
        import scipy.sparse as sps
        R = ref()
        n3, np_, nc = self.n3, self.np_, self.cells.shape[0]
        g, area = self._geometry()
        G = np.einsum("crd,csd->crs", g, g)
        M = area[:, None, None] * R.mass[None]
        K = area[:, None, None] * np.einsum("ijrs,crs->cij", R.stiff, G)
        A = mass_coef * M + self.nu * K
        if w is not None:
            wl = np.stack([w[self.c2d3], w[n3 + self.c2d3]], -1)      # nc x 10 x 2
            cw = np.einsum("ckd,crd->ckr", wl, g)
            A = A + area[:, None, None] * np.einsum("ikjr,ckr->cij", R.conv, cw)
        B = area[:, None, None, None] * np.einsum("qjr,crd->cdqj", R.div, g)
        Kp = area[:, None, None] * np.einsum("qsrt,crt->cqs", R.pstiff, G)
        g3, g2 = self.c2d3, self.c2d2
        rA = np.repeat(g3, 10, axis=1).reshape(-1)
        cA = np.tile(g3, (1, 10)).reshape(-1)
        Am = sps.csr_matrix((A.reshape(-1), (rA, cA)), shape=(n3, n3))
        Mm = sps.csr_matrix((M.reshape(-1), (rA, cA)), shape=(n3, n3))
        rB = np.repeat(g2, 10, axis=1).reshape(-1)
        cB = np.tile(g3, (1, 6)).reshape(-1)
        Bm = sps.hstack([sps.csr_matrix((B[:, a].reshape(-1), (rB, cB)), shape=(np_, n3))
                         for a in range(2)]).tocsr()
        rK = np.repeat(g2, 6, axis=1).reshape(-1)
        cK = np.tile(g2, (1, 6)).reshape(-1)
        Km = sps.csr_matrix((Kp.reshape(-1), (rK, cK)), shape=(np_, np_))
        return Am, Mm, Bm, Km

    def load(self, t, u_prev, inv_dt, M):
        """b_u = M (inv_dt u_prev + I_h f(t)) per component (P3 interpolant)."""
        _, _, f = O.exact(self.problem, 2, t, self.nu, self.xyz3, self._wc())
        n3 = self.n3
        return np.concatenate([M @ (inv_dt * u_prev[a * n3:(a + 1) * n3] + f[:, a])
                               for a in range(2)])

    def _dirichlet(self, t):
        nodes = np.where(self.mask)[0]
        u, _, _ = O.exact(self.problem, 2, t, self.nu, self.xyz3[nodes], self._wc())
        rows = np.concatenate([nodes, self.n3 + nodes])
        return rows, np.concatenate([u[:, 0], u[:, 1]])

    def _pin(self, t):
        _, p, _ = O.exact(self.problem, 2, t, self.nu, self.coords[0:1], self._wc())
        return float(p[0])

    def _w(self):
        if self.wconst is not None:
            return np.concatenate([np.full(self.n3, self.wconst[0]),
                                   np.full(self.n3, self.wconst[1])])
        return self.u

    def coupled_step(self):
        """The backward-Euler Oseen step (Sec. 2.2.1) with P3/P2 elements:
        the monolithic system [[A, -B^T], [B, 0]] with w = u^n, Dirichlet
        rows and the pin replaced, solved exactly."""
        import scipy.sparse as sps
        t1 = self.t + self.dt
        A, M, B, _ = self.blocks(self._w(), 1.0 / self.dt)
        n3 = self.n3
        Av = sps.block_diag([A, A])
        K = sps.bmat([[Av, -B.T], [B, sps.csr_matrix((self.np_, self.np_))]]).tocsr()
        b = np.concatenate([self.load(t1, self.u, 1.0 / self.dt, M), np.zeros(self.np_)])
        rows, vals = self._dirichlet(t1)
        fixed = np.concatenate([rows, [2 * n3]])
        values = np.concatenate([vals, [self._pin(t1)]])
        x = O._solve_rows_replaced(K, b, fixed, values)
        self.u, self.p, self.t = x[:2 * n3].copy(), x[2 * n3:].copy(), t1
        return self.x

    def ipcs_step(self):
        """One incremental pressure-correction step (Sec. 2.2.1, IPCS; the
        three stages and readings of oracle.ipcs_step) with P3/P2 blocks."""
        import scipy.sparse as sps
        t1 = self.t + self.dt
        inv_dt = 1.0 / self.dt
        n3 = self.n3
        Aosn, M, B, Kp = self.blocks(self._w(), inv_dt)
        Astk, _, _, _ = self.blocks(None, inv_dt)
        Nw = sps.block_diag([Aosn - Astk, Aosn - Astk]).tocsr()
        Av = sps.block_diag([Astk, Astk]).tocsr()
        Mv = sps.block_diag([M, M]).tocsr()
        rows, vals = self._dirichlet(t1)
        r1 = self.load(t1, self.u, inv_dt, M) - Nw @ self.u + B.T @ self.p
        ustar = O._solve_rows_replaced(Av, r1, rows, vals)
        r2 = -inv_dt * (B @ ustar)
        dp = O._solve_rows_replaced(Kp, r2, np.array([0]),
                                    np.array([self._pin(t1) - self.p[0]]))
        r3 = Mv @ ustar + self.dt * (B.T @ dp)
        self.u = O._solve_rows_replaced(Mv, r3, rows, vals)
        self.p = self.p + dp
        self.t = t1
        return self.x

    def errors(self, q=10):
        """||u - u_h|| and ||(p - p_h) - mean|| (Stroud rule of oracle.py)."""
        lam, wq = O.simplex_rule(2, q)
        phi3 = np.stack([_eval(f, lam) for f in p3_basis()], -1)
        phi2 = np.stack([_eval(f, lam) for f in p2_basis()], -1)
        xv = self.coords[self.cells]
        J = np.stack([xv[:, 1] - xv[:, 0], xv[:, 2] - xv[:, 0]], -1)
        vol = np.abs(np.linalg.det(J))
        X = np.einsum("qr,crd->cqd", lam, xv)
        ue, pe, _ = O.exact(self.problem, 2, self.t, self.nu, X.reshape(-1, 2), self._wc())
        ue = ue.reshape(X.shape)
        pe = pe.reshape(X.shape[:2])
        n3 = self.n3
        uh = np.stack([np.einsum("qi,ci->cq", phi3, self.u[a * n3:(a + 1) * n3][self.c2d3])
                       for a in range(2)], -1)
        ph = np.einsum("qi,ci->cq", phi2, self.p[self.c2d2])
        wts = vol[:, None] * wq[None, :]
        eu = np.sqrt(np.sum(wts[..., None] * (uh - ue) ** 2))
        ep = ph - pe
        mean = np.sum(wts * ep) / np.sum(wts)
        return eu, np.sqrt(np.sum(wts * (ep - mean) ** 2))


def _eval(poly, lam):
    out = np.zeros(lam.shape[0])
    for (a, b, c), v in poly.items():
        out += float(v) * lam[:, 0] ** a * lam[:, 1] ** b * lam[:, 2] ** c
    return out
