"""Helpers shared by the GPU parity tests: build the CUDA path and the oracle
problem from one workload description."""
import numpy as np

import fs_workloads as W
from oracle import oracle as O


def oracle_problem(wl):
    return O.Problem(dim=wl.dim, n=wl.n, lo=wl.lo, hi=wl.hi, problem=wl.problem, nu=wl.nu,
                     dt=wl.dt, jitter=wl.jitter, seed=wl.seed, side_mask=wl.side_mask,
                     pin_p0=wl.pin_p0, init=wl.init, wconst=wl.wconst)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def poly_oseen(dim, n, jitter=0.1, seed=9):
    return W.Workload(name=f"poly_oseen_{dim}d", dim=dim, n=n, lo=(0.0,) * dim,
                      hi=(1.0,) * dim, problem=W.POLY_OSEEN, nu=0.7, dt=0.05, steps=2,
                      jitter=jitter, seed=seed, side_mask=0x3F if dim == 3 else 0x0F,
                      pin_p0=True, wconst=(1.0, 0.5, 0.25)[:dim])


def poly_oseen_t(dim, n, jitter=0.1, seed=9, steps=3):
    """The time-affine polynomial Oseen problem: (1 + t) times the fields of
    poly_oseen, reproduced exactly by backward Euler at every step."""
    return poly_oseen(dim, n, jitter, seed).with_(name=f"poly_oseen_t_{dim}d",
                                                  problem=W.POLY_OSEEN_T, steps=steps)
