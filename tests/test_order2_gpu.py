"""The second-order upwind sweep (kgs_opts.order = 2, the three-point
backward difference that Section 6 names as the next step) through the C ABI
against the FP64 oracle's order-2 sweep, on identical seeded inputs: 1e-10
for the FP64 path, 1e-5 for the mixed path.

The grids put a block boundary next to every kind of cell the stencil sees:
ragged last blocks one cell wide along x, y and z (the second upwind value of
the next block is then the halo of the one-cell block), block depths of 1, 3
and 32 along z (so slice k-2 comes from the face plane, from slice2, or from
the block's own march), odd velocity counts with a node at xi = 0 (no
transport along that axis), and a ragged last velocity group.
"""
import os

import numpy as np
import pytest

from oracle import Oracle, parallel_build
from paper_1810_00348_gb300 import inputs
from tests.parity import assert_components_close, assert_fields_close, assert_rho_w_close

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def order2(p):
    p.order = 2
    return p


def oracle_threads():
    return (os.cpu_count() or 1) if parallel_build() else 1


def run_pair(kgs, p, n_iter, precision, macros=None, rho_w=None, block_z=0):
    ctx = kgs.kgs_setup(p, precision=precision, block_z=block_z)
    o = Oracle(p, macros, threads=oracle_threads())
    if macros is not None:
        kgs.kgs_set_initial(ctx, macros)
    if rho_w is not None:
        kgs.kgs_set_rho_w(ctx, rho_w)
        o.set_rho_w(rho_w)
    for _ in range(n_iter):
        rc, done, res_g = kgs.kgs_iterate(ctx, 1)
        assert rc == kgs.KGS_OK and done == 1
        res_o = o.iterate()
    return ctx, o, res_g, res_o


@pytest.mark.parametrize("block_z", [1, 3, 32])
def test_fp64_order2_ragged_blocks(kgs, block_z):
    # 17 = 2 * 8 + 1 and 9 = 8 + 1: one-cell blocks along x and y; nz = 10
    p = order2(inputs.cavity([17, 9, 10], [7, 8, 9], L_v=3.5, lid=0.2, Kn=0.4))
    mac = inputs.random_macros(p, 201)
    rw = inputs.random_rho_w(p, 202)
    ctx, o, rg, ro = run_pair(kgs, p, 2, kgs.KGS_FP64, macros=mac, rho_w=rw, block_z=block_z)
    what = "order 2 fp64, block_z %d" % block_z
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, what=what)
    assert_components_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, what=what)
    assert_rho_w_close(kgs.kgs_rho_w(ctx), o.rho_w(), FP64_TOL)
    assert abs(rg - ro) <= 1e-8 * abs(ro)


@pytest.mark.parametrize("block_z", [3, 32])
def test_mixed_order2_ragged_blocks(kgs, block_z):
    p = order2(inputs.cavity([17, 9, 10], [7, 8, 9], L_v=3.5, lid=0.2, Kn=0.4))
    mac = inputs.random_macros(p, 203)
    ctx, o, _, _ = run_pair(kgs, p, 2, kgs.KGS_MIXED, macros=mac, block_z=block_z)
    what = "order 2 mixed, block_z %d" % block_z
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), MIXED_TOL, what=what)
    assert_components_close(kgs.kgs_moments(ctx), o.macros(), MIXED_TOL, what=what)
    assert_rho_w_close(kgs.kgs_rho_w(ctx), o.rho_w(), MIXED_TOL)


@pytest.fixture(scope="module")
def cavity24_ref():
    """24^3 cells (three full blocks per axis) x 32^3 velocities (octant
    x-lines of 16 nodes: the specialised moment loop), Kn 0.1, one iteration
    from rest."""
    p = order2(inputs.cavity(24, 32, Kn=0.1, lid=0.16))
    o = Oracle(p, threads=oracle_threads())
    o.iterate(1)
    return p, o.macros(), o.rho_w()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_order2_24cells_32velocities(kgs, cavity24_ref, precision):
    p, ref, ref_rw = cavity24_ref
    prec = kgs.KGS_FP64 if precision == "fp64" else kgs.KGS_MIXED
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    ctx = kgs.kgs_setup(p, precision=prec)
    rc, done, _ = kgs.kgs_iterate(ctx, 1)
    assert rc == kgs.KGS_OK and done == 1
    what = "order 2 24^3 x 32^3 " + precision
    assert_fields_close(kgs.kgs_moments(ctx), ref, tol, what=what)
    assert_components_close(kgs.kgs_moments(ctx), ref, tol, what=what)
    assert_rho_w_close(kgs.kgs_rho_w(ctx), ref_rw, tol)


def test_order2_is_not_order1_and_converges(kgs):
    p1 = inputs.cavity(16, 12, Kn=0.2, lid=0.16)
    p2 = order2(inputs.cavity(16, 12, Kn=0.2, lid=0.16))
    c1 = kgs.kgs_setup(p1, precision=kgs.KGS_FP64)
    c2 = kgs.kgs_setup(p2, precision=kgs.KGS_FP64)
    res = []
    for _ in range(40):
        _, _, r1 = kgs.kgs_iterate(c1, 1)
        _, _, r2 = kgs.kgs_iterate(c2, 1)
        res.append(r2)
    m1, m2 = kgs.kgs_moments(c1), kgs.kgs_moments(c2)
    # the two discretisations differ by more than the iteration error
    assert np.abs(m1[1] - m2[1]).max() > 1e-4
    # and the second-order source iteration still contracts
    assert res[-1] < 0.1 * res[5]
    assert np.all(np.isfinite(m2))


def test_order2_rejections(kgs):
    p = order2(inputs.cavity(12, 8, Kn=0.5))
    p.dx = np.linspace(0.5, 1.5, p.nx) / p.nx
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(p, precision=kgs.KGS_FP64)
    assert e.value.code == kgs.KGS_EINVAL
    q = order2(inputs.cube(nx=24, ny=16, nz=16, n_vel=8, cube_lo=(0.5, 0.375, 0.375), side=0.25, h=1.0 / 16.0))
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(q, precision=kgs.KGS_FP64)
    assert e.value.code == kgs.KGS_EINVAL
    f = order2(inputs.cavity(12, 8, Kn=0.5))
    f.face_type = [inputs.FACE_INFLOW] * 6
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(f, precision=kgs.KGS_MIXED)
    assert e.value.code == kgs.KGS_EINVAL
    r = order2(inputs.cavity(12, 8, Kn=0.5))
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(r, precision=kgs.KGS_MIXED, v_per_cta=256)
    assert e.value.code == kgs.KGS_EINVAL
    r.order = 3
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(r, precision=kgs.KGS_FP64)
    assert e.value.code == kgs.KGS_EINVAL
