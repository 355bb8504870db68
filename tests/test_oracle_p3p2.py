"""Pins of the P3/P2 oracle (oracle/p3p2.py) to things other than itself:
element matrices against sympy integrals of a Lagrange basis built here
from its interpolation conditions (not from the oracle's barycentric
formulas), invariants, exact discrete steady states, consistency of IPCS
with the coupled step, and the rates of the paper's P3-P2 table."""
import json
import math
import os

import numpy as np
import pytest

import fs_workloads as W
from oracle import oracle as O
from oracle import p3p2 as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "p3p2_table.json")


def _lagrange_basis(sp, X, Y, nodes, degree):
    """Lagrange basis of P_degree on the given nodes (sympy rationals), by
    solving the Vandermonde system of the monomials x^a y^b, a + b <= degree."""
    mons = [X ** a * Y ** b for d in range(degree + 1) for a in range(d, -1, -1)
            for b in [d - a]]
    V = sp.Matrix([[m.subs({X: px, Y: py}) for m in mons] for px, py in nodes])
    C = V.inv()
    return [sp.expand(sum(C[k, i] * mons[k] for k in range(len(mons))))
            for i in range(len(nodes))]


def test_p3p2_element_matrices_vs_sympy():
    sp = pytest.importorskip("sympy")
    from fractions import Fraction as F
    X, Y, S, T = sp.symbols("x y s t")
    verts = [(F(1, 10), F(1, 20)), (F(11, 10), F(-1, 5)), (F(3, 10), F(9, 10))]
    P = [sp.Matrix([sp.Rational(v[0].numerator, v[0].denominator),
                    sp.Rational(v[1].numerator, v[1].denominator)]) for v in verts]
    lerp = lambda a, b, s: (a * (1 - s) + b * s)
    nodes3 = [tuple(p) for p in P]
    for a, b in Q.EDGES:
        nodes3.append(tuple(lerp(P[a], P[b], sp.Rational(1, 3))))   # nearer a
        nodes3.append(tuple(lerp(P[a], P[b], sp.Rational(2, 3))))   # nearer b
    nodes3.append(tuple((P[0] + P[1] + P[2]) / 3))
    nodes2 = [tuple(p) for p in P] + [tuple((P[a] + P[b]) / 2) for a, b in Q.EDGES]
    phi = _lagrange_basis(sp, X, Y, nodes3, 3)
    psi = _lagrange_basis(sp, X, Y, nodes2, 2)
    J = sp.Matrix.hstack(P[1] - P[0], P[2] - P[0])
    sub = {X: P[0][0] + J[0, 0] * S + J[0, 1] * T, Y: P[0][1] + J[1, 0] * S + J[1, 1] * T}
    detJ = abs(J.det())

    def integ(expr):
        e = sp.expand(sp.expand(expr).subs(sub))
        e = sp.integrate(e, (T, 0, 1 - S))
        return float(sp.integrate(sp.expand(e), (S, 0, 1)) * detJ)

    wn = np.array([[0.3, -0.2], [1.0, 0.5], [-0.7, 0.1], [0.2, 0.2], [0.9, -1.1],
                   [0.4, 0.6], [-0.5, 0.3], [0.1, -0.9], [0.8, 0.05], [-0.25, 0.75]])
    xv = np.array([[float(c) for c in v] for v in verts])
    E = Q.element(xv, wn, mass_coef=0.0, nu=1.0)
    gx = [[sp.diff(f, X), sp.diff(f, Y)] for f in phi]
    for i in (0, 4, 9):
        for j in (0, 3, 7, 9):
            assert abs(E["M"][i, j] - integ(phi[i] * phi[j])) < 1e-13
            assert abs(E["K"][i, j] - integ(gx[i][0] * gx[j][0] + gx[i][1] * gx[j][1])) < 1e-12
    wh = [sum(sp.Rational(str(wn[k, a])) * phi[k] for k in range(10)) for a in range(2)]
    for i in (1, 5):
        for j in range(10):
            ref = integ(phi[i] * (wh[0] * gx[j][0] + wh[1] * gx[j][1]))
            assert abs(E["N"][i, j] - ref) < 1e-12
    for c in range(2):
        for q in (0, 3, 5):
            for j in (0, 4, 9):
                assert abs(E["B"][c, q, j] - integ(psi[q] * gx[j][c])) < 1e-13
    px = [[sp.diff(f, X), sp.diff(f, Y)] for f in psi]
    for q in range(6):
        for s_ in (0, 4):
            ref = integ(px[q][0] * px[s_][0] + px[q][1] * px[s_][1])
            assert abs(E["Kp"][q, s_] - ref) < 1e-12


def test_p3p2_element_invariants():
    E = Q.element(np.array([[0.0, 0.0], [1.0, 0.2], [0.3, 0.8]]),
                  np.ones((10, 2)) * (0.4, -0.3), 2.0, 0.5)
    assert abs(E["M"].sum() - E["area"]) < 1e-14          # partition of unity
    assert np.abs(E["K"].sum(1)).max() < 1e-13             # gradients of 1
    assert np.abs(E["N"].sum(1)).max() < 1e-14             # (w . grad) 1 = 0
    assert np.abs(E["Kp"].sum(1)).max() < 1e-13
    assert np.allclose(E["K"], E["K"].T) and np.allclose(E["M"], E["M"].T)
    # summed over the P2 test functions (their sum is 1) and the P3 trial
    # functions (also 1): the integral of d_c 1 = 0
    assert np.abs(E["B"].sum((1, 2))).max() < 1e-14


def test_p3_dofmap_counts_and_node_positions():
    P = Q.Problem3(n=(4, 3), problem=W.JOHN, nu=1.0, dt=0.1, jitter=0.1, seed=3)
    ne = P.edges.shape[0]
    assert P.n3 == P.nv + 2 * ne + P.cells.shape[0] == 13 * 10
    assert P.np_ == P.nv + ne
    # every P3 node shared by neighbours sits at the same point from both
    # cells, and the Dirichlet nodes are exactly those on the boundary
    X = P.xyz3
    onb = (np.abs(X[:, 0]) < 1e-12) | (np.abs(X[:, 0] - 1) < 1e-12) | \
          (np.abs(X[:, 1]) < 1e-12) | (np.abs(X[:, 1] - 1) < 1e-12)
    assert np.array_equal(onb, P.mask.astype(bool))
    lam = Q._node_bary()
    for c in range(P.cells.shape[0]):
        assert np.allclose(X[P.c2d3[c]], lam @ P.coords[P.cells[c]], atol=1e-15)


@pytest.mark.parametrize("step", ["coupled", "ipcs"])
def test_p3p2_keeps_exact_discrete_steady_state(step):
    """u = (x^3, -3x^2 y) (div-free, P3), p = x^2 - y^2 (P2), constant w:
    the steady discrete equations hold for the interpolants, so both the
    coupled step and IPCS keep them, on a jittered mesh."""
    P = Q.Problem3(n=(4, 3), problem=W.POLY3, nu=0.7, dt=0.05, jitter=0.1, seed=9,
                   wconst=(1.0, 0.5))
    X = P.xyz3
    u = np.concatenate([X[:, 0] ** 3, -3 * X[:, 0] ** 2 * X[:, 1]])
    p2 = O.p2_coords(2, P.coords, P.edges)
    p = p2[:, 0] ** 2 - p2[:, 1] ** 2
    assert np.abs(P.u - u).max() < 1e-15 and np.abs(P.p - p).max() < 1e-15
    for _ in range(2):
        (P.coupled_step if step == "coupled" else P.ipcs_step)()
    assert np.abs(P.u - u).max() < 1e-12
    assert np.abs(P.p - p).max() < 1e-11


def test_p3p2_ipcs_converges_in_time_to_the_coupled_solution():
    def run(nt, ipcs):
        P = Q.Problem3(n=(3, 3), problem=W.JOHN, nu=1.0, dt=0.2 / nt, jitter=0.1, seed=2)
        for _ in range(nt):
            P.ipcs_step() if ipcs else P.coupled_step()
        return P.u.copy(), P.p.copy()
    ur, pr = run(512, False)
    d = [run(nt, True) for nt in (16, 32, 64)]
    du = [np.linalg.norm(u - ur) for u, _ in d]
    dp = [np.linalg.norm(p - pr) for _, p in d]
    assert du[0] / du[1] >= 1.8 and du[1] / du[2] >= 1.8, du
    assert dp[0] / dp[1] >= 1.5 and dp[1] / dp[2] >= 1.5, dp


def test_p3p2_ipcs_rates_match_the_paper_table():
    """Sec. 4.1 solution, nu = 1, IPCS with T = 0.02 and dt = 1e-4 (time
    error far below the spatial one): velocity rate -> 4 and pressure rate
    -> 3 on 1/h = 4, 8, 16, as in the paper's P3-P2 table (4.05, 4.00 and
    2.91, 3.06).  Absolute values are not compared (dt and T not stated)."""
    g = json.load(open(GOLDEN))
    eu, ep = [], []
    for n in (4, 8, 16):
        P = Q.Problem3(n=(n, n), problem=W.JOHN, nu=1.0, dt=1e-4)
        for _ in range(200):
            P.ipcs_step()
        a, b = P.errors()
        eu.append(a)
        ep.append(b)
    ru = [math.log2(eu[k - 1] / eu[k]) for k in (1, 2)]
    rp = [math.log2(ep[k - 1] / ep[k]) for k in (1, 2)]
    assert abs(ru[-1] - g["u_rate"][2]) < 0.1, ru
    assert abs(rp[-1] - g["p_rate"][2]) < 0.15, rp
    assert 3.7 < ru[0] < 4.3 and 2.7 < rp[0] < 3.4, (ru, rp)
