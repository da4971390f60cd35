"""Seeded synthetic problem definitions shared by the solver, its tests and the
benchmark.

This module only builds inputs: grids, velocity nodes and trapezoid weights,
solid masks, boundary settings and seeded random fields.  It holds none of the
solver's arithmetic (no equilibrium, sweep, moment or wall-density formula),
so that the CUDA solver and the CPU oracle can both take their inputs from it
without sharing any of the method.

Units (a reading; the paper is silent): length in the cavity side (cube side
for the cube case), velocity in sqrt(2 R T0), temperature in T0, density in
rho0.  Face order everywhere: -x, +x, -y, +y, -z, +z.

Workloads (paper Section 4; sizes as used by the tests and the benchmark):
  * ``cavity``: lid-driven cubic cavity (Section 4.1), all walls diffuse at
    T = 1, lid on the +y face moving along +x.
  * ``cube``: supersonic flow past a cube (Section 4.2), free-stream faces on
    all six sides, a solid cube of side 1 whose centre sits at one third of
    the box length.
  * ``batch_cavities``: uneven cavity instances drawn with splitmix64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

FACE_WALL = 0
FACE_INFLOW = 1
WALL_DISCRETE = 0
WALL_ANALYTIC = 1


@dataclasses.dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    xi_x: np.ndarray
    xi_y: np.ndarray
    xi_z: np.ndarray
    w_x: np.ndarray
    w_y: np.ndarray
    w_z: np.ndarray
    solid: Optional[np.ndarray] = None      # uint8 [nz, ny, nx], 1 = solid
    Kn: float = 1.0
    Pr: float = 2.0 / 3.0
    omega: float = 0.81
    face_type: List[int] = dataclasses.field(default_factory=lambda: [FACE_WALL] * 6)
    T_w: List[float] = dataclasses.field(default_factory=lambda: [1.0] * 6)
    U_w: List[List[float]] = dataclasses.field(default_factory=lambda: [[0.0, 0.0, 0.0] for _ in range(6)])
    rho_in: float = 1.0
    U_in: List[float] = dataclasses.field(default_factory=lambda: [0.0, 0.0, 0.0])
    T_in: float = 1.0
    T_solid: float = 1.0
    wall_mode: int = WALL_DISCRETE
    mass_rescale: int = 1
    q_lagged: int = 0                       # 1: heat flux about the lagged U^n (Algorithm 3's moments)
    order: int = 1                          # upwind order of the sweep: 1 (Eq. (7)) or 2 (three-point)
    name: str = ""

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nvel(self) -> int:
        return len(self.xi_x) * len(self.xi_y) * len(self.xi_z)

    @property
    def n_fluid(self) -> int:
        if self.solid is None:
            return self.ncell
        return int(self.ncell - np.count_nonzero(self.solid))

    def phase_points(self) -> int:
        return self.n_fluid * self.nvel


# --------------------------------------------------------------------------
# velocity axes (nodes and trapezoid weights)

def uniform_axis(n: int, L: float):
    """n equally spaced nodes on [-L, L] including both ends, with trapezoid
    weights h * (1/2, 1, ..., 1, 1/2).  Reading of Section 4: "the trapezoidal
    rule is used" is taken to place nodes at the end points."""
    if n == 1:
        return np.zeros(1), np.ones(1)
    x = np.linspace(-L, L, n)
    h = 2.0 * L / (n - 1)
    w = np.full(n, h)
    w[0] = w[-1] = 0.5 * h
    return x, w


def stretched_axis(n: int, L: float, beta: float = 3.0):
    """Nodes xi(s) = L sinh(beta s)/sinh(beta), s uniform on [-1, 1]
    (clustered near the origin), with non-uniform trapezoid weights
    (xi_{m+1} - xi_{m-1})/2 and half intervals at the ends."""
    s = np.linspace(-1.0, 1.0, n)
    x = L * np.sinh(beta * s) / math.sinh(beta)
    x = 0.5 * (x - x[::-1])  # exact antisymmetry
    w = np.empty(n)
    w[1:-1] = 0.5 * (x[2:] - x[:-2])
    w[0] = 0.5 * (x[1] - x[0])
    w[-1] = 0.5 * (x[-1] - x[-2])
    return x, w


# --------------------------------------------------------------------------
# workloads

def cavity(n_cells, n_vel, Kn: float = 1.0, lid: float = 0.16, L_v: float = 4.0,
           Pr: float = 2.0 / 3.0, omega: float = 0.81, wall_mode: int = WALL_DISCRETE,
           mass_rescale: int = 1, T_w: float = 1.0) -> Problem:
    """Lid-driven cubic cavity on [0,1]^3 (Section 4.1): uniform cells, all
    walls diffuse at T_w, the +y wall (the lid) moving along +x at ``lid``."""
    nx, ny, nz = (n_cells, n_cells, n_cells) if np.isscalar(n_cells) else n_cells
    nvx, nvy, nvz = (n_vel, n_vel, n_vel) if np.isscalar(n_vel) else n_vel
    xx, wx = uniform_axis(nvx, L_v)
    xy, wy = uniform_axis(nvy, L_v)
    xz, wz = uniform_axis(nvz, L_v)
    U_w = [[0.0, 0.0, 0.0] for _ in range(6)]
    U_w[3] = [lid, 0.0, 0.0]
    return Problem(nx=nx, ny=ny, nz=nz,
                   dx=np.full(nx, 1.0 / nx), dy=np.full(ny, 1.0 / ny), dz=np.full(nz, 1.0 / nz),
                   xi_x=xx, xi_y=xy, xi_z=xz, w_x=wx, w_y=wy, w_z=wz,
                   Kn=Kn, Pr=Pr, omega=omega, T_w=[T_w] * 6, U_w=U_w,
                   wall_mode=wall_mode, mass_rescale=mass_rescale,
                   name="cavity %dx%dx%d x %dx%dx%d Kn=%g lid=%g" % (nx, ny, nz, nvx, nvy, nvz, Kn, lid))


def cube(nx: int = 96, ny: int = 64, nz: int = 64, n_vel: int = 48, L_v: float = 8.0,
         beta: float = 3.0, Kn: float = 0.1, mach: float = 2.0, gamma: float = 5.0 / 3.0,
         cube_lo=(1.5, 1.5, 1.5), side: float = 1.0, h: float = 1.0 / 16.0,
         stretched: bool = True) -> Problem:
    """Supersonic flow past a cube (Section 4.2, with the benchmark's box):
    uniform cells of width h, a solid cube of side ``side`` with its low corner
    at ``cube_lo``, free stream rho = 1, T = 1, U = (Ma sqrt(gamma/2), 0, 0) in
    velocity units sqrt(2 R T_inf) on all six sides, cube surface at T = 1."""
    if stretched:
        ax, aw = stretched_axis(n_vel, L_v, beta)
    else:
        ax, aw = uniform_axis(n_vel, L_v)
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    lo = [int(round(c / h)) for c in cube_lo]
    ns = int(round(side / h))
    solid[lo[2]:lo[2] + ns, lo[1]:lo[1] + ns, lo[0]:lo[0] + ns] = 1
    u_inf = mach * math.sqrt(gamma / 2.0)
    return Problem(nx=nx, ny=ny, nz=nz,
                   dx=np.full(nx, h), dy=np.full(ny, h), dz=np.full(nz, h),
                   xi_x=ax.copy(), xi_y=ax.copy(), xi_z=ax.copy(),
                   w_x=aw.copy(), w_y=aw.copy(), w_z=aw.copy(),
                   solid=solid, Kn=Kn, face_type=[FACE_INFLOW] * 6,
                   rho_in=1.0, U_in=[u_inf, 0.0, 0.0], T_in=1.0, T_solid=1.0,
                   mass_rescale=0,
                   name="cube %dx%dx%d x %d^3 Ma=%g Kn=%g" % (nx, ny, nz, n_vel, mach, Kn))


def geometric_widths(n_inner: int, n_out_lo: int, r_lo: float, n_out_hi: int, r_hi: float, side: float = 1.0):
    """Cell widths along one axis of a body of length `side`: n_inner equal
    cells across the body, then n_out_lo cells towards the low end and
    n_out_hi towards the high end whose widths grow cell by cell by the ratios
    r_lo and r_hi, starting from the body's cell width.  Returns the widths
    (low end first) and the index of the first body cell."""
    h0 = side / n_inner
    lo = [h0 * r_lo ** k for k in range(n_out_lo, 0, -1)]
    hi = [h0 * r_hi ** k for k in range(1, n_out_hi + 1)]
    return np.array(lo + [h0] * n_inner + hi), n_out_lo


def cube_paper_mesh(n_inner: int = 31, n_lat: int = 75, n_front: int = 75, n_rear: int = 85, n_vel: int = 48,
                    L_v: float = 4.0, Kn: float = 1.0, mach: float = 2.0, gamma: float = 5.0 / 3.0) -> Problem:
    """Supersonic flow past a cube on the stretched mesh of Section 4.2:
    181 x 181 x 191 cells (with the defaults) whose widths grow cell by cell
    by 1.02 in front of and beside the unit cube and by 1.03 behind it, flow
    along x; 48^3 uniform velocities on [-4, 4]^3; Kn 1, Ma 2, free stream on
    every side, cube surface at the free-stream temperature.  Reading: the
    paper gives the cell counts and ratios but its domain figure is missing;
    n_inner cells span the cube, and the extents follow from the counts."""
    wx, ix0 = geometric_widths(n_inner, n_front, 1.02, n_rear, 1.03)
    wy, iy0 = geometric_widths(n_inner, n_lat, 1.02, n_lat, 1.02)
    wz, iz0 = geometric_widths(n_inner, n_lat, 1.02, n_lat, 1.02)
    nx, ny, nz = len(wx), len(wy), len(wz)
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[iz0:iz0 + n_inner, iy0:iy0 + n_inner, ix0:ix0 + n_inner] = 1
    ax, aw = uniform_axis(n_vel, L_v)
    u_inf = mach * math.sqrt(gamma / 2.0)
    return Problem(nx=nx, ny=ny, nz=nz, dx=wx, dy=wy, dz=wz,
                   xi_x=ax.copy(), xi_y=ax.copy(), xi_z=ax.copy(), w_x=aw.copy(), w_y=aw.copy(), w_z=aw.copy(),
                   solid=solid, Kn=Kn, face_type=[FACE_INFLOW] * 6,
                   rho_in=1.0, U_in=[u_inf, 0.0, 0.0], T_in=1.0, T_solid=1.0, mass_rescale=0,
                   name="cube (stretched mesh) %dx%dx%d x %d^3 Ma=%g Kn=%g" % (nx, ny, nz, n_vel, mach, Kn))


# --------------------------------------------------------------------------
# seeded randomness

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 (Steele, Lea & Flood 2014): state += 0x9E3779B97F4A7C15,
    then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """uniform integer in [lo, hi]"""
        return lo + int(self.uniform() * (hi - lo + 1))


def batch_cavities(n: int = 64, seed: int = 0, cells=(16, 48), vels=(16, 32)) -> List[Problem]:
    """Uneven cavity instances: Kn log-uniform on [0.05, 10], lid speed
    uniform on [0.05, 0.3], cells per side uniform on ``cells``, velocities
    per side uniform on ``vels`` (all drawn from splitmix64(seed))."""
    g = SplitMix64(seed)
    out = []
    for _ in range(n):
        kn = 0.05 * 200.0 ** g.uniform()
        lid = 0.05 + 0.25 * g.uniform()
        nc = g.randint(cells[0], cells[1])
        nv = g.randint(vels[0], vels[1])
        out.append(cavity(nc, nv, Kn=kn, lid=lid))
    return out


def random_macros(prob: Problem, seed: int, amp: float = 0.1) -> np.ndarray:
    """Smooth-ish seeded random macroscopic fields [8, nz, ny, nx]
    (rho, Ux, Uy, Uz, T, qx, qy, qz) around rho = 1, U = 0, T = 1, q = 0."""
    rng = np.random.default_rng(seed)
    shape = (prob.nz, prob.ny, prob.nx)
    m = np.zeros((8,) + shape)
    base = [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    scale = [amp, amp, amp, amp, amp, 0.2 * amp, 0.2 * amp, 0.2 * amp]
    for q in range(8):
        m[q] = base[q] + scale[q] * rng.uniform(-1.0, 1.0, size=shape)
    if prob.solid is not None:
        m[:, prob.solid.astype(bool)] = 0.0
    return m


def random_rho_w(prob: Problem, seed: int, amp: float = 0.1) -> np.ndarray:
    """Seeded wall densities around 1 for every cell face [6, nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    return 1.0 + amp * rng.uniform(-1.0, 1.0, size=(6, prob.nz, prob.ny, prob.nx))
