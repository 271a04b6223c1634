"""Seeded synthetic workloads: lattice shapes, material constants and initial data.

This module is shared by the CUDA path's callers (tests, ``bench.py``) and by the
FP64 oracle's callers. It holds no peridynamic arithmetic: no micromodulus, no
stretch, no force, no time-step bound. It only states *what* is simulated
(lattice, constants, seeds) and draws the random initial data, so that both
sides receive bit-identical inputs.

Point order is the user order used at every public boundary: row-major lattice
order with x fastest, ``i = x + nx*(y + ny*z)``, and reference position
``X_i = origin + h*(x, y, z)``.

The workloads mirror the paper's synthetic lattices (EMU nodal discretization,
Sec. 3.1): 2D plates and 3D blocks on uniform grids. No dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Tuple

import numpy as np

PMB = 0   # bond-based prototype micro-elastic brittle model
LPS = 1   # state-based linear peridynamic solid
NP = 2    # bond-based nonlinear model of Algorithm 1 (potential psi, linearised bond strain)
LP = 3    # its linearisation (psi'(0) in place of psi')

BC_FREE = 0
BC_VELOCITY = 1      # prescribed velocity on this degree of freedom
BC_DISPLACEMENT = 2  # prescribed displacement (velocity held at zero)


@dataclasses.dataclass
class Grid:
    dim: int
    n: Tuple[int, int, int]
    h: float
    m: int                      # horizon factor, delta = m*h
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)

    @property
    def npoints(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def delta(self) -> float:
        return self.m * self.h

    def coords(self) -> np.ndarray:
        """Integer lattice coordinates (npoints, 3) in user order."""
        nx, ny, nz = self.n
        i = np.arange(self.npoints, dtype=np.int64)
        return np.stack([i % nx, (i // nx) % ny, i // (nx * ny)], axis=1)

    def positions(self) -> np.ndarray:
        """Reference positions (npoints, dim), FP64."""
        c = self.coords()[:, : self.dim].astype(np.float64)
        return np.asarray(self.origin[: self.dim], dtype=np.float64) + self.h * c


@dataclasses.dataclass
class Material:
    model: int = PMB
    E: float = 72e9          # Young's modulus, Pa
    rho: float = 2440.0      # mass density, kg/m^3
    K: float = 0.0           # bulk modulus (LPS), Pa
    mu: float = 0.0          # shear modulus (LPS), Pa
    s_c: float = 0.0         # critical stretch; 0 disables breaking
    thickness: float = 1.0   # plate thickness in 2D (m)
    vol_corr: int = 0        # partial-volume correction of boundary-of-horizon cells
    psi_c: float = 1.0       # NP / LP potential psi(r) = psi_c (1 - exp(-psi_beta r))
    psi_beta: float = 1.0


@dataclasses.dataclass
class Notch:
    """A planar rectangle; bonds whose segment crosses it start broken.

    All lengths are in lattice units (multiples of h from the origin). ``axis`` is
    the plane normal, ``pos`` its position (a half-integer keeps every lattice
    point off the plane), ``lo``/``hi`` the rectangle bounds on the other axes.
    """
    axis: int
    pos: float
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]


@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    mat: Material
    steps: int
    seed: int
    dt_factor: float = 0.5          # dt = dt_factor * (stable-step bound)
    dt: float = 0.0                 # > 0: a fixed time step instead
    notch: Optional[Notch] = None
    u0: Optional[np.ndarray] = None        # (n, dim) FP64
    v0: Optional[np.ndarray] = None        # (n, dim) FP64
    bc_kind: Optional[np.ndarray] = None   # (n, dim) uint8
    bc_val: Optional[np.ndarray] = None    # (n, dim) FP64


def collar_mask(grid: Grid, axis: int, side: int, width: Optional[int] = None) -> np.ndarray:
    """Points in the ``width`` outermost lattice layers (default m) on one side of an axis."""
    w = grid.m if width is None else width
    c = grid.coords()[:, axis]
    if side < 0:
        return c < w
    return c >= grid.n[axis] - w


def plate2d(nside: int = 50, seed: int = 1, steps: int = 200, m: int = 3) -> Workload:
    """2D square plate 1 m x 1 m, nside^2 lattice, PMB without breaking.

    Initial displacement N(0, (1e-4 h)^2) per component; the m outermost columns on
    the left/right x-edges move with prescribed v_x = -0.1 / +0.1 m/s, y free.
    """
    h = 1.0 / nside
    g = Grid(dim=2, n=(nside, nside, 1), h=h, m=m)
    mat = Material(model=PMB, E=72e9, rho=2440.0, s_c=0.0, thickness=1.0)
    rng = np.random.default_rng(seed)
    u0 = rng.normal(0.0, 1e-4 * h, size=(g.npoints, 2))
    v0 = np.zeros((g.npoints, 2))
    kind = np.zeros((g.npoints, 2), dtype=np.uint8)
    val = np.zeros((g.npoints, 2))
    left, right = collar_mask(g, 0, -1), collar_mask(g, 0, +1)
    kind[left, 0] = BC_VELOCITY
    kind[right, 0] = BC_VELOCITY
    val[left, 0] = -0.1
    val[right, 0] = 0.1
    v0[:, 0] = val[:, 0]
    return Workload("plate2d_%d_pmb" % nside, g, mat, steps, seed,
                    u0=u0, v0=v0, bc_kind=kind, bc_val=val)


def block3d_pulse(nside: int = 64, seed: int = 2, steps: int = 1000, m: int = 3,
                  s_c: float = 1e-3) -> Workload:
    """3D block nside^3 (h = 1/nside m), PMB with breaking at s_c.

    Gaussian velocity pulse v0 = 1 m/s * exp(-|X - Xc|^2 / w^2) e_x with w = 8h at the
    block centre, plus a pre-notch: the plane z = (nside/2 - 1/2) h, from the face
    x = 0 to depth 0.1 L, spanning all y. Nothing here is random; the seed is kept
    only to name the workload.
    """
    h = 1.0 / nside
    g = Grid(dim=3, n=(nside, nside, nside), h=h, m=m)
    mat = Material(model=PMB, E=72e9, rho=2440.0, s_c=s_c)
    X = g.positions()
    xc = 0.5 * h * (nside - 1)
    w = 8.0 * h
    r2 = ((X - xc) ** 2).sum(axis=1)
    v0 = np.zeros((g.npoints, 3))
    v0[:, 0] = 1.0 * np.exp(-r2 / (w * w))
    u0 = np.zeros((g.npoints, 3))
    depth = 0.1 * nside   # lattice units
    notch = Notch(axis=2, pos=nside / 2 - 0.5, lo=(-0.5, -0.5, 0.0), hi=(depth, nside - 0.5, 0.0))
    kind = np.zeros((g.npoints, 3), dtype=np.uint8)
    val = np.zeros((g.npoints, 3))
    return Workload("block3d_%d_pmb_break" % nside, g, mat, steps, seed, notch=notch,
                    u0=u0, v0=v0, bc_kind=kind, bc_val=val)


def block3d_lps(nside: int = 128, seed: int = 3, steps: int = 500, m: int = 3) -> Workload:
    """3D block nside^3 (h = 1/nside m), state-based LPS, K = 40 GPa, mu = 30 GPa.

    Initial displacement (1e-4/3) X (volumetric strain 1e-4) plus N(0, (1e-5 h)^2).
    """
    h = 1.0 / nside
    g = Grid(dim=3, n=(nside, nside, nside), h=h, m=m)
    mat = Material(model=LPS, E=72e9, rho=2440.0, K=40e9, mu=30e9, s_c=0.0)
    rng = np.random.default_rng(seed)
    X = g.positions()
    u0 = (1e-4 / 3.0) * X + rng.normal(0.0, 1e-5 * h, size=(g.npoints, 3))
    v0 = np.zeros((g.npoints, 3))
    kind = np.zeros((g.npoints, 3), dtype=np.uint8)
    val = np.zeros((g.npoints, 3))
    return Workload("block3d_%d_lps" % nside, g, mat, steps, seed,
                    u0=u0, v0=v0, bc_kind=kind, bc_val=val)


def np_square(k: int = 2, model: int = NP, ic: int = 1, steps: int = 200000, delta: float = 0.1,
              pad: int = 0) -> Workload:
    """The 2D explicit convergence study of Sec. 5.2.2: material domain
    [0, 1]^2, horizon delta = 0.1, h = delta / k (m = k), a lattice over
    [-delta, 1 + delta]^2 whose points outside [0, 1]^2 form the collar held at
    u = 0; rho = 1, psi(r) = 1 - exp(-r) (C = beta = 1), dt = 1e-5, time [0, 2]
    (200000 steps). Initial displacement a exp(-|X - x_c|^2 / beta), v0 = 0:
    IC 1: a = (0.001, 0), x_c = (0.5, 0.5), beta = 0.003;
    IC 2: a = (0.0002, 0.0007), x_c = (0.25, 0.25), beta = 0.01.
    ``pad`` adds that many lattice layers outside the collar on every side."""
    h = delta / k
    n = int(round((1.0 + 2.0 * delta) / h)) + 1 + 2 * pad
    g = Grid(dim=2, n=(n, n, 1), h=h, m=k, origin=(-delta - pad * h, -delta - pad * h, 0.0))
    mat = Material(model=model, E=0.0, rho=1.0, psi_c=1.0, psi_beta=1.0, thickness=1.0)
    a, xc, beta = ((0.001, 0.0), (0.5, 0.5), 0.003) if ic == 1 else ((0.0002, 0.0007), (0.25, 0.25), 0.01)
    u0 = gaussian_ic(g, a, xc, beta)
    X = g.positions()
    tol = 1e-9 * h
    collar = (X[:, 0] < -tol) | (X[:, 0] > 1.0 + tol) | (X[:, 1] < -tol) | (X[:, 1] > 1.0 + tol)
    u0[collar] = 0.0
    kind = np.zeros((g.npoints, 2), dtype=np.uint8)
    kind[collar, :] = BC_DISPLACEMENT
    val = np.zeros((g.npoints, 2))
    name = "np_square_k%d_%s_ic%d" % (k, "np" if model == NP else "lp", ic)
    return Workload(name, g, mat, steps, ic, dt=1e-5, u0=u0, v0=np.zeros_like(u0), bc_kind=kind, bc_val=val)


def np_benchmark(steps: int = 100, model: int = NP) -> Workload:
    """The explicit benchmark of Sec. 6.2: the setup of the 2D study (Sec. 5.2.2,
    IC 1) with horizon delta = 0.05 m and m = 20 (h = 0.0025 m), 196,249 nodes
    (443^2: the lattice over [-delta, 1 + delta]^2 plus one layer on each side)."""
    wl = np_square(k=20, model=model, ic=1, steps=steps, delta=0.05, pad=1)
    wl.name = "np_benchmark_443_m20_%s" % ("np" if model == NP else "lp")
    return wl


@dataclasses.dataclass
class StaticLoad:
    """A quasi-static load path: the prescribed displacements bc_val (full load)
    are applied in load_steps equal increments, s / load_steps for s = 1..load_steps."""
    name: str
    grid: Grid
    mat: Material
    bc_kind: np.ndarray          # (n, dim) uint8: BC_DISPLACEMENT or BC_FREE
    bc_val: np.ndarray           # (n, dim) FP64 at full load
    load_steps: int
    strain: float
    pin: Optional[int] = None    # point whose u_y is held at 0 (roller variant)


def plate_static(nx: int = 200, ny: Optional[int] = None, load_steps: int = 10, strain: float = 1e-4,
                 m: int = 3, variant: str = "clamped") -> StaticLoad:
    """2D plate, h = 1/nx m, PMB without breaking, loaded by its x collars
    (the m outermost columns on each side).

    clamped: left collar u = 0 (both components); right collar u_x = strain * W
             with W = (nx - 1) h, u_y free.
    roller:  both collars carry the uniaxial-stress field u_x = strain * X, u_y
             free, and the left-most point of row ny // 2 has u_y = 0; the
             continuum solution is then u_x = strain X, u_y = -nu strain (Y - Y0)
             with nu = 1/3 and Y0 the pinned point's Y.
    """
    ny = nx if ny is None else ny
    h = 1.0 / nx
    g = Grid(dim=2, n=(nx, ny, 1), h=h, m=m)
    mat = Material(model=PMB, E=72e9, rho=2440.0, s_c=0.0, thickness=1.0)
    kind = np.zeros((g.npoints, 2), dtype=np.uint8)
    val = np.zeros((g.npoints, 2))
    left, right = collar_mask(g, 0, -1), collar_mask(g, 0, +1)
    X = g.positions()
    pin = None
    if variant == "clamped":
        kind[left, :] = BC_DISPLACEMENT
        kind[right, 0] = BC_DISPLACEMENT
        val[right, 0] = strain * (nx - 1) * h
    elif variant == "roller":
        both = left | right
        kind[both, 0] = BC_DISPLACEMENT
        val[both, 0] = strain * X[both, 0]
        pin = (ny // 2) * nx
        kind[pin, 1] = BC_DISPLACEMENT
    else:
        raise ValueError("variant must be 'clamped' or 'roller'")
    return StaticLoad("plate_static_%dx%d_%s" % (nx, ny, variant), g, mat, kind, val, load_steps, strain, pin)


@dataclasses.dataclass
class Request:
    """One independent simulation of a serving mix."""
    grid: Grid
    mat: Material
    steps: int
    arrival: float               # seconds after the first arrival of the mix
    u0: np.ndarray               # (n, dim) FP64
    seed: int


def serving_mix(count: int = 512, seed: int = 5, rate: float = 1.0, side_median: float = 40.0,
                side_sigma: float = 0.5, side_lo: int = 20, side_hi: int = 96, steps_lo: int = 100,
                steps_hi: int = 2000, m_choices: Tuple[int, ...] = (2, 3, 4)) -> list:
    """Independent simulations for the request server, arriving as a Poisson
    process of the given rate (requests/s).

    Per request: model PMB or LPS with probability 1/2; dimension 2 or 3 with
    probability 1/2, LPS always 3D (its coefficients are 3D); side per axis
    round(exp(N(ln side_median, side_sigma^2))) clipped to [side_lo, side_hi];
    h = 1/side_x m; m uniform in m_choices; steps uniform in [steps_lo, steps_hi];
    u0 ~ N(0, (1e-4 h)^2) per component from the request's own seed, v0 = 0, no
    collar, no breaking. E = 72 GPa, rho = 2440 kg/m^3; LPS K = 40 GPa, mu = 30 GPa.
    """
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for k in range(count):
        lps = rng.random() < 0.5
        dim = 3 if (lps or rng.random() < 0.5) else 2
        sides = [int(np.clip(round(float(np.exp(rng.normal(np.log(side_median), side_sigma)))), side_lo, side_hi))
                 for _ in range(dim)]
        n = (sides[0], sides[1], sides[2] if dim == 3 else 1)
        m = int(rng.choice(m_choices))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        g = Grid(dim=dim, n=n, h=1.0 / n[0], m=m)
        mat = Material(model=LPS, E=72e9, rho=2440.0, K=40e9, mu=30e9) if lps else \
            Material(model=PMB, E=72e9, rho=2440.0)
        rs = int(rng.integers(0, 2 ** 31 - 1))
        u0 = np.random.default_rng(rs).normal(0.0, 1e-4 * g.h, size=(g.npoints, dim))
        if k > 0:
            t += float(rng.exponential(1.0 / rate))
        out.append(Request(grid=g, mat=mat, steps=steps, arrival=t, u0=u0, seed=rs))
    return out


def gaussian_ic(grid: Grid, a: Tuple[float, ...], xc: Tuple[float, ...], beta: float) -> np.ndarray:
    """Gaussian displacement u0 = a * exp(-|X - xc|^2 / beta), the initial-condition
    shape of the paper's explicit convergence study (Sec. 5.2.2)."""
    X = grid.positions()
    r2 = ((X - np.asarray(xc[: grid.dim])) ** 2).sum(axis=1)
    return np.exp(-r2 / beta)[:, None] * np.asarray(a[: grid.dim])[None, :]


def random_field(grid: Grid, scale: float, seed: int) -> np.ndarray:
    """N(0, scale^2) per component, (n, dim) FP64."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=(grid.npoints, grid.dim))


def small_grid(dim: int, n: Tuple[int, int, int], m: int, h: float = 0.01) -> Grid:
    return Grid(dim=dim, n=n, h=h, m=m)


WORKLOADS: Dict[str, object] = {
    "plate2d_50_pmb": plate2d,
    "block3d_64_pmb_break": block3d_pulse,
    "block3d_128_lps": block3d_lps,
    "plate_static_200_clamped": plate_static,
    "serving_mix_512": serving_mix,
}
