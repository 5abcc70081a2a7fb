"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds NO arithmetic of the method (no regulator, propagator,
quadrature, interpolation or stepping).  It only describes problems by their
parameters and draws seeded dressing-function profiles tabulated on the
logarithmic momentum grid that both sides interpret independently.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the state advances by the
golden-ratio increment and each output is the published 64-bit finaliser; a
uniform double takes the top 53 bits.

Workload shapes follow the paper's vertex-expansion setups (Sec. 3.3: 96-point
logarithmic momentum grid, 96x8x7 vertex grid, quadrature order 32x8^n in
Table 1) scaled to synthetic configurations: d=3 (64 ext x 64 x 32 nodes),
the d=4 vertex model (1281 ext x 128 x 64 x 16), finite T (64 |p| x 9 p0,
96 x 48 x (2N+1)), the full three-point vertex and the serving request mix.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

MASK64 = (1 << 64) - 1

# model identifiers (same numbering on both sides of the parity tests)
MODEL_D3 = 1          # d=3, T=0 scalar two-point flow
MODEL_D4_VERTEX = 2   # d=4, three coupled dressing tables (Z, lambda3, lambda4)
MODEL_FINITE_T = 3    # d=3 spatial + Matsubara sum (bosonic or fermionic loop)
MODEL_D4_FULL = 4     # d=4 with the three-point vertex on (S0, two shape variables)
MODEL_FINITE_T_4D = 5  # finite T with a 4D regulator on a k-scaled frequency domain

REG_EXP = 0
REG_LITIM = 1

STAT_BOSE = 0
STAT_FERMI = 1


class SplitMix64:
    """splitmix64 stream; ``uniform(lo, hi)`` uses the top 53 bits."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float, hi: float) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


@dataclasses.dataclass
class Problem:
    """Plain parameters of one right-hand-side evaluation (both sides read these)."""
    model: int
    n_rad: int
    n_ang1: int
    n_ext_p: int
    n_ang2: int = 1
    n_ext_ang: int = 1
    n_matsubara: int = 0
    include_p0: int = 0
    regulator: int = REG_EXP
    m2_over_k2: float = 0.5
    m2_shift: float = 0.0
    lam: float = 1.0
    T: float = 0.0
    p_min: float = 1e-3
    p_max: float = 10.0
    qmax_over_k: float = 4.0
    prefactor: float = 1.0
    # dressing tables: values[n_tables][n_stack][n_pts] on a log grid [x_min, x_max]
    n_tables: int = 1
    n_pts: int = 64
    n_stack: int = 1
    x_min: float = 1e-3
    x_max: float = 10.0
    # finite T: loop frequencies bosonic (STAT_BOSE) or fermionic (STAT_FERMI)
    statistics: int = 0
    # D4_FULL: three-point vertex nodes in its two shape variables (n_stack = n_va n_vb)
    n_va: int = 1
    n_vb: int = 1
    # FINITE_T_4D: Gauss-Legendre nodes of the frequency integral beyond the Matsubara cap
    n_x0: int = 0

    def n_ext(self) -> int:
        if self.model == MODEL_D3:
            return self.n_ext_p + (1 if self.include_p0 else 0)
        if self.model in (MODEL_D4_VERTEX, MODEL_D4_FULL):
            return 2 * self.n_ext_p + 1 + self.n_ext_p * self.n_ext_ang
        if self.model in (MODEL_FINITE_T, MODEL_FINITE_T_4D):
            return self.n_ext_p * self.n_ext_ang
        raise ValueError(self.model)

    def n_nodes(self) -> int:
        n = self.n_rad * self.n_ang1
        if self.model in (MODEL_D4_VERTEX, MODEL_D4_FULL):
            n *= self.n_ang2
        if self.model == MODEL_FINITE_T:
            n *= 2 * self.n_matsubara + 1 + (1 if self.statistics == STAT_FERMI else 0)
        if self.model == MODEL_FINITE_T_4D:   # at most: the Matsubara cap or the quadrature nodes
            n *= max(2 * self.n_matsubara + 1 + (1 if self.statistics == STAT_FERMI else 0), self.n_x0)
        return n

    def evals(self) -> int:
        """integrand evaluations of one RHS = external points x quadrature nodes."""
        return self.n_ext() * self.n_nodes()

    def table_size(self) -> int:
        return self.n_tables * self.n_stack * self.n_pts


@dataclasses.dataclass
class Workload:
    problem: Problem
    tables: np.ndarray              # float64 [n_tables, n_stack, n_pts]
    y0: Optional[np.ndarray] = None  # initial flow state (float64)
    Lambda: float = 10.0            # UV scale k at t_+ = 0
    k_end: float = 0.01
    feedback: int = 0
    seed: int = 0
    params: dict = dataclasses.field(default_factory=dict)


def log_grid(n: int, lo: float, hi: float) -> np.ndarray:
    """Abscissae of a logarithmic table grid: lo*(hi/lo)**(j/(n-1))."""
    if n == 1:
        return np.array([lo])
    j = np.arange(n, dtype=np.float64)
    return lo * (hi / lo) ** (j / (n - 1))


def _bump(p2, amp, width):
    return 1.0 + amp * np.exp(-p2 / width)


def make_d3(seed: int = 1, n_pts: int = 64, n_ext_p: int = 64, n_rad: int = 64, n_ang: int = 32,
            Lambda: float = 10.0, k_end: float = 0.01, feedback: int = 0, regulator: int = REG_EXP,
            m2_over_k2: float = 0.5, x_min: float = 1e-3, x_max: float = 10.0) -> Workload:
    """d=3 scalar two-point flow: Z(q) = 1 + a exp(-q^2/b), a in [0,0.2], b in [0.5,2]."""
    rng = SplitMix64(seed)
    a = rng.uniform(0.0, 0.2)
    b = rng.uniform(0.5, 2.0)
    pb = Problem(model=MODEL_D3, n_rad=n_rad, n_ang1=n_ang, n_ext_p=n_ext_p, regulator=regulator,
                 m2_over_k2=m2_over_k2, n_tables=1, n_pts=n_pts, n_stack=1,
                 include_p0=1 if feedback else 0, p_min=x_min, p_max=x_max, x_min=x_min, x_max=x_max)
    xs = log_grid(n_pts, pb.x_min, pb.x_max)
    tables = _bump(xs ** 2, a, b).reshape(1, 1, n_pts)
    m2_uv = m2_over_k2 * Lambda ** 2
    if feedback:
        if n_pts != n_ext_p:
            raise ValueError("feedback flow needs the external grid equal to the table grid")
        pb.m2_over_k2 = 0.0
        pb.m2_shift = m2_uv
        y0 = np.concatenate([[m2_uv], tables[0, 0]])
    else:
        ps = log_grid(n_ext_p, pb.p_min, pb.p_max)
        y0 = _bump(ps ** 2, a, b) * ps ** 2 + m2_uv
    return Workload(pb, tables, y0, Lambda, k_end, feedback, seed, dict(a=a, b=b))


def make_d4(seed: int = 2, n_pts: int = 128, n_ext_ang: int = 8, n_rad: int = 128, n_ang1: int = 64,
            n_ang2: int = 16, Lambda: float = 10.0, k_end: float = 0.01, M2: float = 1.0,
            regulator: int = REG_EXP) -> Workload:
    """d=4 vertex expansion with three tables Z, lambda3, lambda4 (external grid = table grid)."""
    rng = SplitMix64(seed)
    a = rng.uniform(0.0, 0.2)
    b = rng.uniform(0.5, 2.0)
    g3 = rng.uniform(0.5, 1.5)
    c3 = rng.uniform(-0.3, 0.3)
    b3 = rng.uniform(0.5, 2.0)
    g4 = rng.uniform(0.5, 1.5)
    c4 = rng.uniform(-0.3, 0.3)
    b4 = rng.uniform(0.5, 2.0)
    pb = Problem(model=MODEL_D4_VERTEX, n_rad=n_rad, n_ang1=n_ang1, n_ang2=n_ang2, n_ext_p=n_pts,
                 n_ext_ang=n_ext_ang, regulator=regulator, m2_over_k2=0.5, m2_shift=M2,
                 n_tables=3, n_pts=n_pts, n_stack=1)
    xs = log_grid(n_pts, pb.x_min, pb.x_max)
    x2 = xs ** 2
    tables = np.stack([_bump(x2, a, b), g3 * _bump(x2, c3, b3), g4 * _bump(x2, c4, b4)]).reshape(3, 1, n_pts)
    y0 = tables.reshape(-1).copy()
    return Workload(pb, tables, y0, Lambda, k_end, 1, seed,
                    dict(a=a, b=b, g3=g3, c3=c3, b3=b3, g4=g4, c4=c4, b4=b4))


def make_d4_full(seed: int = 7, n_pts: int = 96, n_va: int = 8, n_vb: int = 7, n_ext_ang: int = 8,
                 n_rad: int = 128, n_ang1: int = 64, n_ang2: int = 16, Lambda: float = 10.0, k_end: float = 0.01,
                 M2: float = 1.0, regulator: int = REG_EXP) -> Workload:
    """d=4 vertex expansion with the three-point vertex on (S0, a, b): a 96 x 8 x 7 grid by default
    (log S0 x uniform a, b in [-1, 1]); lambda3 = g3 (1 + c3 exp(-S^2/b3)) (1 + ea a + eb b + eab a b).
    Tables [3][n_va n_vb][n_pts]: Z and lambda4 in row 0 of tables 0 and 2 (other rows zero),
    lambda3 in row ia n_vb + ib of table 1.  Frozen-background flow state (ones)."""
    rng = SplitMix64(seed)
    a = rng.uniform(0.0, 0.2)
    b = rng.uniform(0.5, 2.0)
    g3 = rng.uniform(0.5, 1.5)
    c3 = rng.uniform(-0.3, 0.3)
    b3 = rng.uniform(0.5, 2.0)
    g4 = rng.uniform(0.5, 1.5)
    c4 = rng.uniform(-0.3, 0.3)
    b4 = rng.uniform(0.5, 2.0)
    ea, eb, eab = rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-0.1, 0.1)
    n_stack = n_va * n_vb
    pb = Problem(model=MODEL_D4_FULL, n_rad=n_rad, n_ang1=n_ang1, n_ang2=n_ang2, n_ext_p=n_pts,
                 n_ext_ang=n_ext_ang, regulator=regulator, m2_over_k2=0.5, m2_shift=M2,
                 n_tables=3, n_pts=n_pts, n_stack=n_stack, n_va=n_va, n_vb=n_vb)
    xs = log_grid(n_pts, pb.x_min, pb.x_max)
    x2 = xs ** 2
    av = np.linspace(-1.0, 1.0, n_va) if n_va > 1 else np.zeros(1)
    bv = np.linspace(-1.0, 1.0, n_vb) if n_vb > 1 else np.zeros(1)
    tables = np.zeros((3, n_stack, n_pts))
    tables[0, 0] = _bump(x2, a, b)
    tables[2, 0] = g4 * _bump(x2, c4, b4)
    for ia in range(n_va):
        for ib in range(n_vb):
            tables[1, ia * n_vb + ib] = g3 * _bump(x2, c3, b3) * (1 + ea * av[ia] + eb * bv[ib] + eab * av[ia] * bv[ib])
    y0 = np.ones(pb.n_ext())
    return Workload(pb, tables, y0, Lambda, k_end, 0, seed,
                    dict(a=a, b=b, g3=g3, c3=c3, b3=b3, g4=g4, c4=c4, b4=b4, ea=ea, eb=eb, eab=eab))


def make_finite_t(seed: int = 3, N: int = 16, T: float = 0.002, n_pts: int = 64, n_ext_p: int = 64,
                  n_ext_m: int = 9, n_rad: int = 96, n_ang: int = 48, Lambda: float = 10.0,
                  k_end: float = 0.01, regulator: int = REG_EXP, fermionic: bool = False) -> Workload:
    """Finite T: tables Z(j,|p|) and lam(j,|p|) stacked over the loop frequency index j <= N+8:
    bosonic omega_j = 2 pi T j, or (fermionic=True) nu_j = (2j+1) pi T."""
    rng = SplitMix64(seed)
    a = rng.uniform(0.0, 0.2)
    b = rng.uniform(0.5, 2.0)
    g = rng.uniform(0.5, 1.5)
    c = rng.uniform(-0.3, 0.3)
    bl = rng.uniform(0.5, 2.0)
    n_stack = N + n_ext_m
    pb = Problem(model=MODEL_FINITE_T, n_rad=n_rad, n_ang1=n_ang, n_ext_p=n_ext_p, n_ext_ang=n_ext_m,
                 n_matsubara=N, regulator=regulator, m2_over_k2=0.5, T=T,
                 n_tables=2, n_pts=n_pts, n_stack=n_stack, statistics=STAT_FERMI if fermionic else STAT_BOSE)
    xs = log_grid(n_pts, pb.x_min, pb.x_max)
    j = np.arange(n_stack, dtype=np.float64)
    om2 = (math.pi * T * (2.0 * j + 1.0) if fermionic else 2.0 * math.pi * T * j) ** 2
    e2 = xs[None, :] ** 2 + om2[:, None]
    tables = np.stack([_bump(e2, a, b), g * _bump(e2, c, bl)])
    ps = log_grid(n_ext_p, pb.p_min, pb.p_max)
    m2_uv = 0.5 * Lambda ** 2
    om2_ext = (2.0 * math.pi * T * np.arange(n_ext_m, dtype=np.float64)) ** 2
    y0 = (_bump(ps[:, None] ** 2 + om2_ext[None, :], a, b) * (ps[:, None] ** 2 + om2_ext[None, :])
          + m2_uv).reshape(-1)
    return Workload(pb, tables, y0, Lambda, k_end, 0, seed, dict(a=a, b=b, g=g, c=c, bl=bl))


def make_finite_t_4d(seed: int = 12, N: int = 16, T: float = 0.05, n_pts: int = 64, n_ext_p: int = 64,
                     n_ext_m: int = 9, n_rad: int = 96, n_ang: int = 48, n_x0: int = 64, Lambda: float = 10.0,
                     k_end: float = 0.01, regulator: int = REG_EXP, fermionic: bool = False) -> Workload:
    """Finite T with a 4D regulator on a k-scaled frequency domain: dressings Z(|Q|) and lam(|Q|) on one
    log grid in the 4-momentum magnitude; Matsubara cap N (sum while at most 2N+1 (+1) loop frequencies
    lie in |q0| <= qmax k, else n_x0 Gauss-Legendre nodes); fermionic: loop nu_n and the external
    fermion leg at p0f (n_ext_m must be 1)."""
    rng = SplitMix64(seed)
    a = rng.uniform(0.0, 0.2)
    b = rng.uniform(0.5, 2.0)
    g = rng.uniform(0.5, 1.5)
    c = rng.uniform(-0.3, 0.3)
    bl = rng.uniform(0.5, 2.0)
    if fermionic:
        n_ext_m = 1
    pb = Problem(model=MODEL_FINITE_T_4D, n_rad=n_rad, n_ang1=n_ang, n_ext_p=n_ext_p, n_ext_ang=n_ext_m,
                 n_matsubara=N, regulator=regulator, m2_over_k2=0.5, T=T, n_tables=2, n_pts=n_pts, n_stack=1,
                 statistics=STAT_FERMI if fermionic else STAT_BOSE, n_x0=n_x0)
    xs = log_grid(n_pts, pb.x_min, pb.x_max)
    x2 = xs ** 2
    tables = np.stack([_bump(x2, a, b), g * _bump(x2, c, bl)]).reshape(2, 1, n_pts)
    ps = log_grid(n_ext_p, pb.p_min, pb.p_max)
    om2_ext = (2.0 * math.pi * T * np.arange(n_ext_m, dtype=np.float64)) ** 2
    P2 = ps[:, None] ** 2 + om2_ext[None, :]
    y0 = (_bump(P2, a, b) * P2 + 0.5 * Lambda ** 2).reshape(-1)
    return Workload(pb, tables, y0, Lambda, k_end, 0, seed, dict(a=a, b=b, g=g, c=c, bl=bl))


def constant_tables(pb: Problem, values: List[float]) -> np.ndarray:
    """Tables that are constant in momentum (used by closed-form reductions)."""
    t = np.empty((pb.n_tables, pb.n_stack, pb.n_pts))
    for i, v in enumerate(values):
        t[i] = v
    return t


@dataclasses.dataclass
class Request:
    """One serving request: a flow with its own grid sizes and parameters."""
    rid: int
    arrival_s: float
    workload: Workload


def serving_stream(seed: int = 5, n_requests: int = 1024, rate_hz: float = 200.0,
                   ext_range=(32, 256), rad_range=(32, 128), ang_range=(16, 64),
                   pts_range=(64, 256), t_max: float = 1.0, n_cap: int = 64) -> List[Request]:
    """Poisson arrivals of flow requests scanning w = m^2/k^2 in [-0.2, 1] and T in [0, t_max].

    T < 0.01 selects the T = 0 family (d=3 two-point flow, frozen background);
    otherwise a finite-T flow with N = min(n_cap, ceil(Lambda / (2 pi T))).
    """
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += -math.log(1.0 - rng.uniform(0.0, 1.0)) / rate_hz
        w = rng.uniform(-0.2, 1.0)
        T = rng.uniform(0.0, t_max)
        n_ext = int(rng.uniform(ext_range[0], ext_range[1] + 1))
        n_rad = int(rng.uniform(rad_range[0], rad_range[1] + 1))
        n_ang = int(rng.uniform(ang_range[0], ang_range[1] + 1))
        n_pts = int(rng.uniform(pts_range[0], pts_range[1] + 1))
        sub_seed = rng.next_u64()
        if T < 0.01:
            wl = make_d3(seed=sub_seed, n_pts=n_pts, n_ext_p=n_ext, n_rad=n_rad, n_ang=n_ang,
                         m2_over_k2=w)
        else:
            N = min(n_cap, int(math.ceil(10.0 / (2.0 * math.pi * T))))
            n_ext_p = max(1, n_ext // 9)
            wl = make_finite_t(seed=sub_seed, N=N, T=T, n_pts=n_pts, n_ext_p=n_ext_p,
                               n_rad=n_rad, n_ang=n_ang)
            wl.problem.m2_over_k2 = w
            m2_uv = w * wl.Lambda ** 2
            wl.y0 = wl.y0 - 0.5 * wl.Lambda ** 2 + m2_uv
        out.append(Request(rid, t, wl))
    return out
