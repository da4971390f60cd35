"""CUDA path (through the C ABI) against the FP64 oracle on identical seeded
inputs.  The FP64 path must agree to 1e-10 relative on rho, U, T, q (and on
the wall densities); the mixed FP32-sweep / FP64-moment path to 1e-5.

Sizes span several sweep blocks (8 x 8 x block_z cells) with ragged tails,
velocity grids with odd node counts (a node at xi = 0, uneven octants and a
ragged last velocity group), solid cells, free-stream faces, stretched
velocity grids, both wall normalisations, and the free-molecular limit.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_1810_00348_gb300 import inputs
from tests.parity import assert_fields_close, assert_rho_w_close, field_errors

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def run_pair(kgs, prob, n_iter, precision, macros=None, rho_w=None, **opts):
    ctx = kgs.kgs_setup(prob, precision=precision, **opts)
    o = Oracle(prob, macros)
    if macros is not None:
        kgs.kgs_set_initial(ctx, macros)
    # the initial wall densities are computed independently on both sides
    assert_rho_w_close(kgs.kgs_rho_w(ctx), o.rho_w(), 1e-12 if precision == kgs.KGS_FP64 else 1e-12)
    if rho_w is not None:
        kgs.kgs_set_rho_w(ctx, rho_w)
        o.set_rho_w(rho_w)
    for _ in range(n_iter):
        rc, done, res_g = kgs.kgs_iterate(ctx, 1)
        assert rc == kgs.KGS_OK and done == 1
        res_o = o.iterate()
    return ctx, o, res_g, res_o


def ragged_cavity(**kw):
    p = inputs.cavity([19, 17, 35], [9, 8, 7], L_v=3.5, lid=0.2, Kn=0.4, **kw)
    return p


@pytest.mark.parametrize("n_iter", [1, 2])
def test_fp64_ragged_random_state(kgs, n_iter):
    p = ragged_cavity()
    mac = inputs.random_macros(p, 101)
    rw = inputs.random_rho_w(p, 102)
    ctx, o, rg, ro = run_pair(kgs, p, n_iter, kgs.KGS_FP64, macros=mac, rho_w=rw)
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, what="fp64 ragged")
    assert_rho_w_close(kgs.kgs_rho_w(ctx), o.rho_w(), FP64_TOL)
    assert abs(rg - ro) <= 1e-8 * ro


@pytest.mark.parametrize("block_z", [1, 5, 16])
def test_fp64_block_shapes_agree(kgs, block_z):
    p = inputs.cavity([12, 9, 13], 6, L_v=3.0, lid=0.3, Kn=0.2)
    ctx, o, _, _ = run_pair(kgs, p, 2, kgs.KGS_FP64, block_z=block_z)
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, what="block_z=%d" % block_z)


def test_fp64_nonuniform_cells_analytic_walls_no_rescale(kgs):
    p = inputs.cavity([10, 11, 9], [8, 7, 6], L_v=3.5, lid=0.25, Kn=0.6, wall_mode=inputs.WALL_ANALYTIC,
                      mass_rescale=0)
    rng = np.random.default_rng(7)
    p.dx = rng.uniform(0.5, 1.5, p.nx) / p.nx
    p.dy = rng.uniform(0.5, 1.5, p.ny) / p.ny
    p.dz = rng.uniform(0.5, 1.5, p.nz) / p.nz
    p.T_w = [1.0, 1.1, 0.9, 1.05, 0.95, 1.2]
    ctx, o, _, _ = run_pair(kgs, p, 2, kgs.KGS_FP64)
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, what="nonuniform/analytic")
    assert_rho_w_close(kgs.kgs_rho_w(ctx), o.rho_w(), FP64_TOL)


def test_fp64_solid_and_free_stream(kgs):
    p = inputs.cube(nx=20, ny=12, nz=18, n_vel=8, L_v=5.0, Kn=0.3, cube_lo=(0.5, 0.25, 0.375), side=0.375,
                    h=1.0 / 16.0)
    assert p.solid.sum() == 6 ** 3
    ctx, o, _, _ = run_pair(kgs, p, 2, kgs.KGS_FP64)
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, solid=p.solid, what="cube")
    assert_rho_w_close(kgs.kgs_rho_w(ctx), o.rho_w(), FP64_TOL)


def test_fp64_free_molecular(kgs):
    p = inputs.cavity([9, 10, 11], 6, L_v=3.0, lid=0.3, Kn=math.inf)
    ctx, o, _, _ = run_pair(kgs, p, 2, kgs.KGS_FP64)
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, what="Kn=inf")


def test_fp64_bgk(kgs):
    p = inputs.cavity([9, 8, 10], 7, L_v=3.5, lid=0.2, Kn=0.3, Pr=1.0)
    ctx, o, _, _ = run_pair(kgs, p, 2, kgs.KGS_FP64)
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), FP64_TOL, what="BGK")


@pytest.fixture(scope="module")
def small_cavity_converged():
    """The 10^3-cell x 12^3-velocity cavity (Kn = 1, lid 0.16) run by the
    oracle to residual 1e-8."""
    p = inputs.cavity(10, 12, Kn=1.0, lid=0.16)
    o = Oracle(p)
    n = 0
    for n in range(1, 200):
        if o.iterate() < 1e-8:
            break
    return p, o.macros(), o.rho_w(), n


def test_fp64_small_cavity_to_convergence(kgs, small_cavity_converged):
    p, ref, ref_rw, n_oracle = small_cavity_converged
    ctx = kgs.kgs_setup(p, precision=kgs.KGS_FP64, tol=1e-8, max_iters=200)
    rc, done, res = kgs.kgs_iterate(ctx, 0)
    assert rc == kgs.KGS_OK and res < 1e-8
    assert done == n_oracle
    assert_fields_close(kgs.kgs_moments(ctx), ref, FP64_TOL, what="small cavity converged")
    assert_rho_w_close(kgs.kgs_rho_w(ctx), ref_rw, FP64_TOL)


def test_mixed_small_cavity_to_convergence(kgs, small_cavity_converged):
    p, ref, _, _ = small_cavity_converged
    for vpc in (128, 256):
        ctx = kgs.kgs_setup(p, precision=kgs.KGS_MIXED, tol=1e-8, max_iters=200, v_per_cta=vpc)
        rc, done, res = kgs.kgs_iterate(ctx, 0)
        err = field_errors(kgs.kgs_moments(ctx), ref)
        assert max(err.values()) <= MIXED_TOL, err


def test_mixed_one_iteration(kgs):
    p = ragged_cavity()
    mac = inputs.random_macros(p, 201)
    ctx, o, _, _ = run_pair(kgs, p, 1, kgs.KGS_MIXED, macros=mac)
    assert_fields_close(kgs.kgs_moments(ctx), o.macros(), MIXED_TOL, what="mixed")


@pytest.fixture(scope="module")
def line16_case():
    """32 velocity nodes per axis (octant x-lines of 16 nodes: the moment loop
    specialised to 16-node lines, as in the benchmark) on a ragged 9 x 7 x 10
    grid from a random state; two oracle iterations (about 1.3e7 phase points
    each)."""
    p = inputs.cavity([9, 7, 10], 32, L_v=4.0, lid=0.2, Kn=0.5)
    mac = inputs.random_macros(p, 301)
    o = Oracle(p, mac)
    o.iterate()
    o.iterate()
    return p, mac, o.macros(), o.rho_w()


@pytest.mark.parametrize("precision,vpc", [("fp64", 0), ("mixed", 128), ("mixed", 256)])
def test_line16_against_oracle(kgs, line16_case, precision, vpc):
    p, mac, ref, ref_rw = line16_case
    prec = kgs.KGS_FP64 if precision == "fp64" else kgs.KGS_MIXED
    ctx = kgs.kgs_setup(p, precision=prec, v_per_cta=vpc)
    kgs.kgs_set_initial(ctx, mac)
    rc, done, _ = kgs.kgs_iterate(ctx, 2)
    assert rc == kgs.KGS_OK and done == 2
    tol = FP64_TOL if precision == "fp64" else MIXED_TOL
    assert_fields_close(kgs.kgs_moments(ctx), ref, tol, what="32-node lines, %s" % precision)
    if precision == "fp64":
        assert_rho_w_close(kgs.kgs_rho_w(ctx), ref_rw, FP64_TOL)


def test_deterministic_and_resumable(kgs):
    p = inputs.cavity([12, 10, 14], 8, L_v=3.5, lid=0.2, Kn=0.5)
    a = kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
    kgs.kgs_iterate(a, 3)
    ck = kgs.kgs_save(a)
    kgs.kgs_iterate(a, 2)
    m_a = kgs.kgs_moments(a).copy()
    b = kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
    kgs.kgs_iterate(b, 5)
    assert np.array_equal(m_a, kgs.kgs_moments(b))  # same run twice: bit for bit
    c = kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
    assert kgs.kgs_load(c, ck) == kgs.KGS_OK
    assert kgs.kgs_info(c)["iteration"] == 3
    kgs.kgs_iterate(c, 2)
    assert np.array_equal(m_a, kgs.kgs_moments(c))  # resume: bit for bit


def test_abi_errors(kgs):
    p = inputs.cavity(4, 4)
    p.dx = np.array([0.25, 0.25, -0.25, 0.25])
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(p)
    assert e.value.code == kgs.KGS_EINVAL
    p = inputs.cavity(4, 5, Kn=math.inf)  # odd grid: xi = 0 on every axis
    with pytest.raises(kgs.KgsError):
        kgs.kgs_setup(p)
    q = inputs.cavity(4, 4)
    ctx = kgs.kgs_setup(q)
    other = kgs.kgs_setup(inputs.cavity(5, 4))
    assert kgs.kgs_load(ctx, kgs.kgs_save(other)) == kgs.KGS_EFORMAT
    assert kgs.kgs_load(ctx, b"xx") == kgs.KGS_EFORMAT
    bad = inputs.random_macros(q, 3)
    bad[0, 0, 0, 0] = -1.0
    with pytest.raises(kgs.KgsError):
        kgs.kgs_set_initial(ctx, bad)
