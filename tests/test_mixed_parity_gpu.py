"""Mixed-precision path (FP32 equilibrium and sweep, compensated FP32 moment
sums, FP64 closure) against the FP64 oracle at 1e-5, on the cases where FP32
rounding is hardest:

* the 64^3-cell cavity with an 8^3 velocity grid (the benchmark's oracle
  sample): octant x-lines of 4 nodes take the general moment loop, few
  velocities per cell average little of the rounding away, and the sweep runs
  64 cells deep at Kn = 1, where each update is mostly upwind transport;
* the supersonic flow past a cube (Section 4.2) reduced to 24 x 16 x 16 cells,
  with solid cells, free stream on every side, the 48-node stretched velocity
  grid on [-8, 8] (octant lines of 24 nodes) and |U| = 1.83 folded into the
  FP32 exponent;
* non-uniform cell widths (per-cell upwind coefficients).

The oracle sweeps contiguous velocity ranges on all host cores.  The FP64
path is checked on the same cases at 1e-10.  Besides the field-normalised
errors, each component of U and q is compared against its own largest
value (the spanwise components are about 1% of the streamwise ones).
"""
import os

import numpy as np
import pytest

from oracle import Oracle, parallel_build
from paper_1810_00348_gb300 import inputs
from tests.parity import assert_components_close, assert_fields_close, assert_rho_w_close

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5
FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def oracle_threads():
    cores = os.cpu_count() or 1
    return cores if parallel_build() else 1


def run_gpu(kgs, p, n_iter, precision, macros=None):
    ctx = kgs.kgs_setup(p, precision=precision)
    if macros is not None:
        kgs.kgs_set_initial(ctx, macros)
    rc, done, _ = kgs.kgs_iterate(ctx, n_iter)
    assert rc == kgs.KGS_OK and done == n_iter
    return kgs.kgs_moments(ctx), kgs.kgs_rho_w(ctx)


@pytest.fixture(scope="module")
def cavity8_from_rest():
    p = inputs.cavity(64, 8, Kn=1.0, lid=0.16)
    o = Oracle(p, threads=oracle_threads())
    o.iterate(1)
    return p, o.macros(), o.rho_w()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cavity64_8_velocities_from_rest(kgs, cavity8_from_rest, precision):
    p, ref, ref_rw = cavity8_from_rest
    prec = kgs.KGS_MIXED if precision == "mixed" else kgs.KGS_FP64
    tol = MIXED_TOL if precision == "mixed" else FP64_TOL
    m, rw = run_gpu(kgs, p, 1, prec)
    assert_fields_close(m, ref, tol, what="64^3 x 8^3 from rest, %s" % precision)
    assert_components_close(m, ref, tol, what="64^3 x 8^3 from rest, %s" % precision)
    assert_rho_w_close(rw, ref_rw, tol)


def test_cavity64_8_velocities_random_state_mixed(kgs):
    p = inputs.cavity(64, 8, Kn=1.0, lid=0.16)
    mac = inputs.random_macros(p, 811)
    o = Oracle(p, mac, threads=oracle_threads())
    o.iterate(2)
    m, rw = run_gpu(kgs, p, 2, kgs.KGS_MIXED, macros=mac)
    assert_fields_close(m, o.macros(), MIXED_TOL, what="64^3 x 8^3 random state, mixed")
    assert_components_close(m, o.macros(), MIXED_TOL, what="64^3 x 8^3 random state, mixed")
    assert_rho_w_close(rw, o.rho_w(), MIXED_TOL)


def reduced_cube():
    """Mach 2 flow past a cube of 6^3 cells in a 24 x 16 x 16 box of cells
    1/16 wide, Kn 0.1, 48^3 stretched velocities on [-8, 8]^3."""
    return inputs.cube(nx=24, ny=16, nz=16, n_vel=48, L_v=8.0, Kn=0.1, cube_lo=(0.375, 0.3125, 0.3125),
                       side=0.375, h=1.0 / 16.0)


@pytest.fixture(scope="module")
def cube_ref():
    p = reduced_cube()
    assert p.solid.sum() == 6 ** 3
    o = Oracle(p, threads=oracle_threads())
    o.iterate(2)
    return p, o.macros(), o.rho_w()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cube_stretched_48_against_oracle(kgs, cube_ref, precision):
    p, ref, ref_rw = cube_ref
    prec = kgs.KGS_MIXED if precision == "mixed" else kgs.KGS_FP64
    tol = MIXED_TOL if precision == "mixed" else FP64_TOL
    m, rw = run_gpu(kgs, p, 2, prec)
    assert_fields_close(m, ref, tol, solid=p.solid, what="cube 24x16x16 x 48^3 stretched, %s" % precision)
    assert_components_close(m, ref, tol, solid=p.solid, what="cube 24x16x16 x 48^3 stretched, %s" % precision)
    assert_rho_w_close(rw, ref_rw, tol)


def test_mixed_nonuniform_cells(kgs):
    p = inputs.cavity([20, 18, 22], 12, L_v=4.0, lid=0.2, Kn=0.5)
    rng = np.random.default_rng(17)
    p.dx = rng.uniform(0.5, 1.5, p.nx) / p.nx
    p.dy = rng.uniform(0.5, 1.5, p.ny) / p.ny
    p.dz = rng.uniform(0.5, 1.5, p.nz) / p.nz
    mac = inputs.random_macros(p, 19)
    o = Oracle(p, mac, threads=oracle_threads())
    o.iterate(2)
    m, rw = run_gpu(kgs, p, 2, kgs.KGS_MIXED, macros=mac)
    assert_fields_close(m, o.macros(), MIXED_TOL, what="non-uniform cells, mixed")
    assert_rho_w_close(rw, o.rho_w(), MIXED_TOL)
