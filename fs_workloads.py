"""Seeded synthetic workloads: the shapes, sizes, coefficients and seeds of the
runs, and nothing of the method's arithmetic.

This is the one module both the oracle and the CUDA path's tests/bench read.
It holds mesh descriptions (grid sizes, domains, jitter fractions, seeds),
the physical coefficients (nu, dt, steps) and the seeded draws of the batched
and serving workloads (log-uniform sizes and Reynolds numbers, Poisson
arrival gaps).  The random numbers come from SplitMix64 (Steele, Lea and
Flood 2014) used as a counter-based hash, written out here from its
published definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

# problem ids shared by both sides of every comparison
JOHN, STEADY_POLY, CHANNEL, CUBE, POLY_OSEEN, POLY_OSEEN_T, POLY3 = 0, 1, 2, 3, 4, 5, 6

# Dirichlet side masks: bit s set = side s Dirichlet;
# sides 0: x=lo, 1: x=hi, 2: y=lo, 3: y=hi, 4: z=lo, 5: z=hi
ALL_SIDES_2D = 0x0F
ALL_SIDES_3D = 0x3F
CHANNEL_SIDES = 0x0D      # inflow x=lo and walls y=lo, y=hi; outflow x=hi free

_MASK64 = (1 << 64) - 1


def splitmix64(state: int) -> int:
    z = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def uniform(seed: int, key: int) -> float:
    """U in [0,1) from the 53 high bits of SplitMix64(seed XOR key)."""
    return (splitmix64((seed ^ key) & _MASK64) >> 11) * 2.0 ** -53


@dataclass(frozen=True)
class Workload:
    """One time-stepping problem on a structured simplicial mesh."""
    name: str
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    problem: int
    nu: float
    dt: float
    steps: int
    jitter: float = 0.0
    seed: int = 0
    side_mask: int = ALL_SIDES_2D
    pin_p0: bool = True
    init: str = "exact"            # "exact" = I_h u(0); "zero_interior"
    wconst: tuple | None = None    # constant convecting field (Oseen test)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    # counts (Taylor-Hood P2/P1 on the structured mesh)
    @property
    def ncell(self) -> int:
        return 2 * self.n[0] * self.n[1] if self.dim == 2 else \
            6 * self.n[0] * self.n[1] * self.n[2]

    @property
    def nvert(self) -> int:
        return math.prod(k + 1 for k in self.n)

    @property
    def n2(self) -> int:
        return math.prod(2 * k + 1 for k in self.n)

    @property
    def ndof(self) -> int:
        return self.dim * self.n2 + self.nvert


def unit_square(n=8, **kw) -> Workload:
    """2D unit square n x n, jitter 0.1h, the unsteady benchmark solution,
    nu = 1, dt = 0.01, 10 steps, FP64."""
    base = dict(name=f"unit_square_{n}x{n}", dim=2, n=(n, n), lo=(0.0, 0.0),
                hi=(1.0, 1.0), problem=JOHN, nu=1.0, dt=0.01, steps=10,
                jitter=0.1, seed=0, side_mask=ALL_SIDES_2D, pin_p0=True)
    base.update(kw)
    return Workload(**base)


def channel(nx=512, ny=96, **kw) -> Workload:
    """2D channel [0,2.2]x[0,0.41], parabolic inflow U_max = 1.5, do-nothing
    outflow, nu = 1e-3, dt = 1e-3, 200 steps, no jitter."""
    base = dict(name=f"channel_{nx}x{ny}", dim=2, n=(nx, ny), lo=(0.0, 0.0),
                hi=(2.2, 0.41), problem=CHANNEL, nu=1e-3, dt=1e-3, steps=200,
                jitter=0.0, seed=0, side_mask=CHANNEL_SIDES, pin_p0=False,
                init="zero_interior")
    base.update(kw)
    return Workload(**base)


def cube(n=48, **kw) -> Workload:
    """3D unit cube n^3 x 6 Kuhn tetrahedra, jitter 0.05h, the 3D
    manufactured solution, nu = 1e-2, dt = 5e-3, 20 steps."""
    base = dict(name=f"cube_{n}", dim=3, n=(n, n, n), lo=(0.0, 0.0, 0.0),
                hi=(1.0, 1.0, 1.0), problem=CUBE, nu=1e-2, dt=5e-3, steps=20,
                jitter=0.05, seed=0, side_mask=ALL_SIDES_3D, pin_p0=True)
    base.update(kw)
    return Workload(**base)


# The five configurations of the benchmark suite.
C1 = unit_square(8)
C2 = channel(512, 96)
C3 = cube(48)


def batched_instances(count=96, seed=0, nmin=16, nmax=256, remin=1.0,
                      remax=2000.0, dt=1e-3, steps=50):
    """Batched workload: `count` 2D unit-square instances with N and Re drawn
    log-uniform from SplitMix64 streams (N rounded to an integer)."""
    out = []
    for i in range(count):
        u1 = uniform(seed, 2 * i)
        u2 = uniform(seed, 2 * i + 1)
        n = int(round(math.exp(math.log(nmin) + u1 * (math.log(nmax) - math.log(nmin)))))
        re = math.exp(math.log(remin) + u2 * (math.log(remax) - math.log(remin)))
        out.append(unit_square(n, name=f"batch{i}_n{n}", nu=1.0 / re, dt=dt,
                               steps=steps, jitter=0.0))
    return out


@dataclass(frozen=True)
class Request:
    rid: int
    arrival: float
    workload: Workload


def serving_requests(count=10000, rate=200.0, seed=0, n2d=(16, 512),
                     n3d=(8, 48), re=(1.0, 2000.0), steps=(10, 100), dt=1e-3):
    """Poisson arrival stream of 2D and 3D solves (Bernoulli(1/2) mix),
    sizes and Re log-uniform, steps uniform in [steps0, steps1]."""
    t = 0.0
    out = []
    for i in range(count):
        k = 8 * i + (1 << 40)
        gap = -math.log(1.0 - uniform(seed, k)) / rate
        t += gap
        is3d = uniform(seed, k + 1) < 0.5
        lo, hi = n3d if is3d else n2d
        n = int(round(math.exp(math.log(lo) + uniform(seed, k + 2) *
                               (math.log(hi) - math.log(lo)))))
        r = math.exp(math.log(re[0]) + uniform(seed, k + 3) *
                     (math.log(re[1]) - math.log(re[0])))
        ns = steps[0] + int(uniform(seed, k + 4) * (steps[1] - steps[0] + 1))
        if is3d:
            w = cube(n, name=f"req{i}_3d_n{n}", nu=1.0 / r, dt=dt, steps=ns,
                     jitter=0.0)
        else:
            w = unit_square(n, name=f"req{i}_2d_n{n}", nu=1.0 / r, dt=dt,
                            steps=ns, jitter=0.0)
        out.append(Request(i, t, w))
    return out
