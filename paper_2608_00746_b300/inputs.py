"""Seeded synthetic initial conditions shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds geometry, random draws and initial-condition physics (stiffened-gas
Rankine-Hugoniot states) only: none of the finite-volume method's arithmetic.
Every generator returns PRIMITIVE fields
``V = [(alpha rho)_1..N, u_1..d, P, alpha_1..N]`` laid out ``[NV][nz][ny][nx]``
(x fastest) in FP64; each implementation converts them to conservative
variables with its own code.

Materials follow the stiffened-gas form of Eq. 26 (gamma, Pinf, D).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

AIR = dict(gamma=1.4, pinf=0.0, D=0.0, rho=1.0)
WATER = dict(gamma=4.4, pinf=6.0e8, D=0.0, rho=1000.0)
# third phase of the 3-D and learned workloads: gamma 6.1, Pinf 2e9; its
# density is not given, 1050 kg/m^3 is used
PHASE3 = dict(gamma=6.1, pinf=2.0e9, D=0.0, rho=1050.0)


@dataclass
class Case:
    name: str
    shape: tuple            # (nx,), (nx, ny) or (nx, ny, nz)
    dx: tuple
    gamma: list
    pinf: list
    D: list
    V: np.ndarray           # primitive state [NV][nz][ny][nx]
    bc: tuple               # 6 entries: lo/hi per axis
    flux: str = "hll"
    cfl: float = 0.2
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return len(self.gamma)

    @property
    def dim(self):
        return len(self.shape)


def _centres(shape, dx, lo=(0.0, 0.0, 0.0)):
    """Cell-centre coordinates, each broadcastable to [nz][ny][nx]."""
    d = len(shape)
    axes = []
    for a in range(d):
        x = lo[a] + (np.arange(shape[a]) + 0.5) * dx[a]
        sh = [1] * d
        sh[d - 1 - a] = shape[a]
        axes.append(x.reshape(sh))
    return axes


def _assemble(alpha, rho_p, u, P):
    """V from fractions alpha[N], phasic densities rho_p[N], velocity u[d], P."""
    N = len(alpha)
    d = len(u)
    shp = np.broadcast(*alpha, *rho_p, *u, P).shape
    V = np.empty((2 * N + d + 1,) + shp)
    for p in range(N):
        V[p] = np.broadcast_to(alpha[p] * rho_p[p], shp)
        V[N + d + 1 + p] = np.broadcast_to(alpha[p], shp)
    for j in range(d):
        V[N + j] = np.broadcast_to(u[j], shp)
    V[N + d] = np.broadcast_to(P, shp)
    return np.ascontiguousarray(V)


TAIL = 1e-15


def smooth_step(s, width):
    """0..1 indicator of s > 0 with a tanh edge of the given width.  Values
    within 1e-15 of 0 or 1 are set to exactly 0 or 1: the tails of the tanh
    carry no information at FP64 resolution of the fraction sum, and exact
    zeros keep a phase exactly absent away from its interfaces (the paper's
    own initial conditions are sharp, Eq. 31-33)."""
    v = 0.5 * (1.0 + np.tanh(s / width))
    return np.where(v < TAIL, 0.0, np.where(v > 1.0 - TAIL, 1.0, v))


def shock_state(gamma, pinf, rho1, p1, ratio):
    """Post-shock (rho2, u2) of a stiffened-gas shock of pressure ratio
    ``ratio`` running into fluid at rest (rho1, p1); the shocked fluid moves
    towards +x."""
    p2 = ratio * p1
    a, b = p2 + pinf, p1 + pinf
    r = ((gamma + 1.0) * a + (gamma - 1.0) * b) / ((gamma - 1.0) * a + (gamma + 1.0) * b)
    rho2 = rho1 * r
    w = np.sqrt((p2 - p1) / (rho1 * (1.0 - 1.0 / r)))
    u2 = w * (1.0 - 1.0 / r)
    return rho2, u2, p2


def _mat(phases):
    return ([m["gamma"] for m in phases], [m["pinf"] for m in phases],
            [m["D"] for m in phases], [m["rho"] for m in phases])


# ----------------------------------------------------------------------------
# Config 1: 1-D two-phase interface advection (air slab in water)
# ----------------------------------------------------------------------------
def interface_advection_1d(n=200, u0=1.0, p0=1.0e5, width_cells=2.0, absent_phase=False):
    """Air slab on [0.25, 0.75] inside water on the periodic [0, 1]; tanh edges
    of ``width_cells`` cells; uniform u and P.  ``absent_phase`` appends a
    third phase (the config-3 stiffened gas) with alpha = alpha*rho = 0."""
    dx = 1.0 / n
    (x,) = _centres((n,), (dx,))
    w = width_cells * dx
    a_air = 0.5 * (np.tanh((x - 0.25) / w) - np.tanh((x - 0.75) / w))
    a_air = np.where(a_air < TAIL, 0.0, np.where(a_air > 1.0 - TAIL, 1.0, a_air))
    phases = [AIR, WATER] + ([PHASE3] if absent_phase else [])
    g, pi, D, rho = _mat(phases)
    alpha = [a_air, 1.0 - a_air] + ([np.zeros_like(x)] if absent_phase else [])
    V = _assemble(alpha, rho, [np.full_like(x, u0)], np.full_like(x, p0))
    return Case("interface_advection_1d", (n,), (dx,), g, pi, D, V,
                ("periodic",) * 2 + ("periodic",) * 4, flux="hllc", cfl=0.5)


# ----------------------------------------------------------------------------
# Smooth two-phase advection (order of accuracy, Sec. 4.1.4)
# ----------------------------------------------------------------------------
def smooth_advection_1d(n):
    dx = 1.0 / n
    # cell averages of alpha_1 = 0.2 (3 + sin 2 pi x), exact integral
    xl = np.arange(n) * dx
    xr = xl + dx
    a1 = 0.6 + 0.2 * (np.cos(2 * np.pi * xl) - np.cos(2 * np.pi * xr)) / (2 * np.pi * dx)
    rho = [2.0, 1.0]
    V = _assemble([a1, 1.0 - a1], rho, [np.ones(n)], np.ones(n))
    return Case("smooth_advection_1d", (n,), (dx,), [1.5, 1.01], [0.0, 0.02], [0.0, 3.0], V,
                ("periodic",) * 6, flux="hllc", cfl=0.0,
                meta=dict(dt=dx ** (5.0 / 3.0)))


def smooth_alpha_average(n, t):
    """Exact cell averages of alpha_1 at time t for smooth_advection_1d (u = 1)."""
    dx = 1.0 / n
    xl = np.arange(n) * dx - t
    xr = xl + dx
    return 0.6 + 0.2 * (np.cos(2 * np.pi * xl) - np.cos(2 * np.pi * xr)) / (2 * np.pi * dx)


# ----------------------------------------------------------------------------
# 2-D advection of an air circle in water; five-phase Table 1 materials
# ----------------------------------------------------------------------------
TABLE1 = [  # rho, gamma, Pinf, D  (Table 1)
    (1.204e-3, 1.400, 0.000, 0.000),
    (1.000, 6.120, 0.163, 0.000),
    (0.800, 2.350, 0.476, -5.550e-4),
    (0.100e-3, 1.600, 0.000, 0.000),
    (1.000e-3, 3.000, 0.000, 0.000),
]


def multiphase_advection_2d(n=100, nphase=5, width_cells=1.0):
    """Doubly periodic [-0.5, 0.5]^2, u = (1, 1), P = 4.819e-5 (Sec. 4.1.2):
    phase 1 background, phase 2 circle (0, 0, 0.2), phase 3 circles
    (0, +-0.5, 0.15), phase 4 circles (+-0.5, 0, 0.15), phase 5 absent.
    ``nphase`` < 5 keeps the first phases (2: the air/water-like pair of
    Sec. 4.1.1 with the Table 1 values of phases 1 and 2)."""
    dx = 1.0 / n
    x, y = _centres((n, n), (dx, dx), lo=(-0.5, -0.5))
    w = width_cells * dx
    alpha = [np.ones((n, n))] + [np.zeros((n, n)) for _ in range(nphase - 1)]

    def put(q, cx, cy, r):
        if q >= nphase:
            return
        # periodic distance
        ddx = (x - cx + 0.5) % 1.0 - 0.5
        ddy = (y - cy + 0.5) % 1.0 - 0.5
        s = smooth_step(r - np.sqrt(ddx ** 2 + ddy ** 2), w)
        for k in range(nphase):
            alpha[k] = alpha[k] * (1.0 - s)
        alpha[q] = alpha[q] + s

    put(1, 0.0, 0.0, 0.2)
    put(2, 0.0, 0.5, 0.15)
    put(3, 0.5, 0.0, 0.15)
    mats = TABLE1[:nphase]
    V = _assemble(alpha, [m[0] for m in mats], [np.ones((n, n)), np.ones((n, n))],
                  np.full((n, n), 4.819e-5))
    return Case("multiphase_advection_2d", (n, n), (dx, dx), [m[1] for m in mats],
                [m[2] for m in mats], [m[3] for m in mats], V, ("periodic",) * 6,
                flux="hllc", cfl=0.0, meta=dict(dt=1e-3))


def two_phase_advection_2d(n=100, width_cells=1.0):
    """Sec. 4.1.1: doubly periodic [-0.5, 0.5]^2, an air circle (phase 1,
    rho 1.204e-3, gamma 1.4) of radius 0.2 at the origin in water (phase 2,
    rho 1, gamma 6.12, Pinf 0.1631), u = (1, 1), P = 4.819e-5, dt = 1e-3
    (one period = 1000 steps on the paper's 100^2 grid)."""
    dx = 1.0 / n
    x, y = _centres((n, n), (dx, dx), lo=(-0.5, -0.5))
    s = smooth_step(0.2 - np.sqrt(x ** 2 + y ** 2), width_cells * dx)
    rho = (1.204e-3, 1.0)
    V = _assemble([s, 1.0 - s], rho, [np.ones((n, n)), np.ones((n, n))],
                  np.full((n, n), 4.819e-5))
    return Case("two_phase_advection_2d", (n, n), (dx, dx), [1.4, 6.12], [0.0, 0.1631],
                [0.0, 0.0], V, ("periodic",) * 6, flux="hllc", cfl=0.0,
                meta=dict(dt=1e-3, rho=rho))


def miscible_advection_2d(n=100, width_cells=1.0):
    """Four-phase advection with a non-zero, non-unity constant fraction
    (Sec. 4.1.3): doubly periodic [-0.5, 0.5]^2, u = (1, 1), P = 4.819e-5,
    alpha_1 = 0.8 inside the circle (0, 0, 0.2) and alpha_2 = 0.8 outside
    (smoothed edge), alpha_3 = 0.2 everywhere, alpha_4 = 0 (absent); the
    first four phases of Table 1."""
    dx = 1.0 / n
    x, y = _centres((n, n), (dx, dx), lo=(-0.5, -0.5))
    s = smooth_step(0.2 - np.sqrt(x ** 2 + y ** 2), width_cells * dx)
    alpha = [0.8 * s, 0.8 * (1.0 - s), np.full((n, n), 0.2), np.zeros((n, n))]
    mats = TABLE1[:4]
    V = _assemble(alpha, [m[0] for m in mats], [np.ones((n, n)), np.ones((n, n))],
                  np.full((n, n), 4.819e-5))
    return Case("miscible_advection_2d", (n, n), (dx, dx), [m[1] for m in mats],
                [m[2] for m in mats], [m[3] for m in mats], V, ("periodic",) * 6,
                flux="hllc", cfl=0.0, meta=dict(dt=1e-3))


# ----------------------------------------------------------------------------
# Config 2: 2-D shock-bubble (N = 2, reflective walls)
# ----------------------------------------------------------------------------
def shock_bubble_2d(nx=1024, ny=512, seed=0, width_cells=2.0):
    rng = np.random.default_rng(seed)
    xc = rng.uniform(0.5, 1.5)
    yc = rng.uniform(0.3, 0.7)
    r = rng.uniform(0.1, 0.2)
    ratio = 10.0 ** rng.uniform(3.0, 4.0)
    lx, ly = 2.0, 1.0
    dx, dy = lx / nx, ly / ny
    x, y = _centres((nx, ny), (dx, dy))
    s = smooth_step(r - np.sqrt((x - xc) ** 2 + (y - yc) ** 2), width_cells * dx)
    p0 = 1.0e5
    rho2, u2, p2 = shock_state(WATER["gamma"], WATER["pinf"], WATER["rho"], p0, ratio)
    xs = xc - r - 0.05
    behind = (x < xs) & (y >= 0)
    rho_w = np.where(behind, rho2, WATER["rho"])
    u = np.where(behind, u2, 0.0) + 0.0 * y
    P = np.where(behind, p2, p0) + 0.0 * y
    V = _assemble([s + 0.0 * x, 1.0 - s], [AIR["rho"], rho_w], [u, np.zeros_like(u)], P)
    g, pi, D, _ = _mat([AIR, WATER])
    return Case("shock_bubble_2d", (nx, ny), (dx, dy), g, pi, D, V, ("reflective",) * 6,
                flux="hll", cfl=0.2, meta=dict(xc=xc, yc=yc, r=r, ratio=ratio, xs=xs))


# ----------------------------------------------------------------------------
# Config 3: 3-D N = 3 spheres + planar shock (outflow)
# ----------------------------------------------------------------------------
def spheres_shock_3d(n=256, seed=0, nsph=16, rmin_cells=8, rmax_cells=32, ratio=1.0e3,
                     width_cells=2.0, shape=None):
    shape = shape or (n, n, n)
    rng = np.random.default_rng(seed)
    dx = tuple(1.0 / s for s in shape)
    h = dx[0]
    x, y, z = _centres(shape, dx)
    full = (shape[2], shape[1], shape[0])
    alpha = [np.zeros(full), np.ones(full), np.zeros(full)]
    for k in range(nsph):
        r = rng.integers(rmin_cells, rmax_cells + 1) * h
        c = rng.uniform(0.0, 1.0, size=3)
        q = 0 if k % 2 == 0 else 2
        s = smooth_step(r - np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2),
                        width_cells * h)
        for p in range(3):
            alpha[p] = alpha[p] * (1.0 - s)
        alpha[q] = alpha[q] + s
    p0 = 1.0e5
    rho2, u2, p2 = shock_state(WATER["gamma"], WATER["pinf"], WATER["rho"], p0, ratio)
    behind = np.broadcast_to(x < 0.05, full)
    rho_w = np.where(behind, rho2, WATER["rho"])
    u = np.where(behind, u2, 0.0)
    P = np.where(behind, p2, p0)
    zero = np.zeros(full)
    V = _assemble(alpha, [AIR["rho"], rho_w, PHASE3["rho"]], [u, zero, zero], P)
    g, pi, D, _ = _mat([AIR, WATER, PHASE3])
    return Case("spheres_shock_3d", shape, dx, g, pi, D, V, ("outflow",) * 6, flux="hll",
                cfl=0.2)


# ----------------------------------------------------------------------------
# Config 5: 2-D N = 3 circles + shock (learned-weight workload)
# ----------------------------------------------------------------------------
def circles_shock_2d(n=2048, seed=0, ncirc=64, rmin_cells=10, rmax_cells=80, ratio=1.0e3,
                     width_cells=2.0, shape=None):
    shape = shape or (n, n)
    rng = np.random.default_rng(seed)
    dx = tuple(1.0 / s for s in shape)
    h = dx[0]
    x, y = _centres(shape, dx)
    full = (shape[1], shape[0])
    alpha = [np.zeros(full), np.ones(full), np.zeros(full)]
    for k in range(ncirc):
        r = rng.uniform(rmin_cells, rmax_cells) * h
        c = rng.uniform(0.0, 1.0, size=2)
        q = 0 if k % 2 == 0 else 2
        s = smooth_step(r - np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2), width_cells * h)
        for p in range(3):
            alpha[p] = alpha[p] * (1.0 - s)
        alpha[q] = alpha[q] + s
    p0 = 1.0e5
    rho2, u2, p2 = shock_state(WATER["gamma"], WATER["pinf"], WATER["rho"], p0, ratio)
    behind = np.broadcast_to(x < 0.05, full)
    rho_w = np.where(behind, rho2, WATER["rho"])
    u = np.where(behind, u2, 0.0)
    P = np.where(behind, p2, p0)
    V = _assemble(alpha, [AIR["rho"], rho_w, PHASE3["rho"]], [u, np.zeros(full)], P)
    g, pi, D, _ = _mat([AIR, WATER, PHASE3])
    return Case("circles_shock_2d", shape, dx, g, pi, D, V, ("outflow",) * 6, flux="hll",
                cfl=0.2)


# ----------------------------------------------------------------------------
# Config 4: batched AMR-like patches
# ----------------------------------------------------------------------------
PATCH_EDGES = (8, 12, 16, 24, 32)


def patch_batch(npatch=4096, seed=0, edges=PATCH_EDGES, width_cells=2.0):
    """Independent cube patches (edge uniform in ``edges``), N = 3 with the
    config-3 materials.  Each patch holds a plane interface with a random
    normal through a random interior point separating water from air or from
    the third phase (the other phase absent in that patch) and a plane
    pressure jump of ratio log-uniform in [10, 1e4].  Returns (edges, list of
    primitive patch states [NV][e][e][e], materials)."""
    rng = np.random.default_rng(seed)
    e_list = rng.choice(np.asarray(edges), size=npatch)
    g, pi, D, rho = _mat([AIR, WATER, PHASE3])
    states = []
    for e in e_list:
        e = int(e)
        h = 1.0 / e
        x, y, z = _centres((e, e, e), (h, h, h))
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        pt = rng.uniform(0.25, 0.75, size=3)
        s = smooth_step((x - pt[0]) * nrm[0] + (y - pt[1]) * nrm[1] + (z - pt[2]) * nrm[2],
                        width_cells * h)
        other = 0 if rng.uniform() < 0.5 else 2
        full = (e, e, e)
        alpha = [np.zeros(full), np.broadcast_to(1.0 - s, full).copy(), np.zeros(full)]
        alpha[other] = np.broadcast_to(s, full).copy()
        ratio = 10.0 ** rng.uniform(1.0, 4.0)
        n2 = rng.normal(size=3)
        n2 /= np.linalg.norm(n2)
        pt2 = rng.uniform(0.25, 0.75, size=3)
        side = ((x - pt2[0]) * n2[0] + (y - pt2[1]) * n2[1] + (z - pt2[2]) * n2[2]) < 0
        P = np.broadcast_to(np.where(side, 1.0e5 * ratio, 1.0e5), full)
        zero = np.zeros(full)
        states.append(_assemble(alpha, rho, [zero, zero, zero], P))
    return e_list, states, (g, pi, D)


def random_admissible_stencils(ncell, N, d, seed=0, near_vacuum=True):
    """Random admissible cell averages and raw face values for limiter tests:
    primitive V arrays [NV][ncell] for the cell average and for the two raw
    faces; faces may leave the admissible set (negative masses, fractions
    outside [0, 1], wrong sums) so that every limiter branch runs."""
    rng = np.random.default_rng(seed)
    nvar = 2 * N + d + 1

    def fractions(n):
        a = rng.dirichlet(np.full(N, 0.5), size=n).T
        if near_vacuum:
            m = rng.uniform(size=(N, n)) < 0.3
            a = np.where(m, a * 1e-12, a)
            a /= a.sum(0, keepdims=True)
        return a

    Vb = np.empty((nvar, ncell))
    ab = fractions(ncell)
    rho_p = 10.0 ** rng.uniform(-3, 3, size=(N, ncell))
    Vb[:N] = ab * rho_p
    Vb[N + d + 1:] = ab
    Vb[N:N + d] = rng.normal(size=(d, ncell)) * 10.0
    Vb[N + d] = 10.0 ** rng.uniform(3, 6, size=ncell)
    faces = []
    for _ in range(2):
        Vf = Vb.copy()
        scale = rng.uniform(0, 2.0, size=(1, ncell))
        Vf[:N] = Vb[:N] + scale * rng.normal(size=(N, ncell)) * Vb[:N]
        Vf[N + d + 1:] = Vb[N + d + 1:] + scale * rng.normal(size=(N, ncell)) * 0.5
        Vf[N:N + d] = Vb[N:N + d] + rng.normal(size=(d, ncell)) * 5.0
        Vf[N + d] = Vb[N + d] * (1.0 + rng.normal(size=ncell) * 0.5)
        faces.append(Vf)
    return Vb, faces[0], faces[1]
