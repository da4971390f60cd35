"""Checks at the benchmark's full sizes, in the launch configuration the
benchmark times, where the oracle cannot follow (one outer iteration of the
64^3 x 32^3 cavity is about 8.6e9 phase points): properties that hold at any
size, the two precisions against each other, and batch instances against
single contexts.
"""
import numpy as np
import pytest

from paper_1810_00348_gb300 import inputs
from tests.parity import field_errors

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def mirror_errors(m, axis):
    """Largest deviation from the mirror symmetry of the fields about the mid
    plane normal to `axis` (0 = x, 1 = y, 2 = z of the [8, nz, ny, nx]
    array): the velocity and heat-flux components along `axis` are odd, all
    other fields even.  Normalised like the parity errors."""
    ax = {0: 3, 1: 2, 2: 1}[axis]
    f = np.flip(m, axis=ax)
    sign = np.ones(8)
    sign[1 + axis] = sign[5 + axis] = -1.0
    d = m - sign[:, None, None, None] * f
    scale = [1.0, *(3 * [np.abs(m[1:4]).max()]), 1.0, *(3 * [np.abs(m[5:8]).max()])]
    return max(np.abs(d[q]).max() / scale[q] for q in range(8))


@pytest.fixture(scope="module")
def cavity64(kgs):
    p = inputs.cavity(64, 32, Kn=1.0, lid=0.16)
    out = {}
    for prec in (kgs.KGS_FP64, kgs.KGS_MIXED):
        ctx = kgs.kgs_setup(p, precision=prec)  # autotuned shape, as the benchmark
        rc, n, res = kgs.kgs_iterate(ctx, 2)
        assert rc == kgs.KGS_OK
        out[prec] = (kgs.kgs_moments(ctx), res, ctx)
    return p, out


def test_cavity64_mixed_matches_fp64(kgs, cavity64):
    _, out = cavity64
    err = field_errors(out[kgs.KGS_MIXED][0], out[kgs.KGS_FP64][0])
    assert max(err.values()) <= 1e-5, err


def test_cavity64_kn01_mixed_matches_fp64(kgs):
    # the second Knudsen number of the 64^3 x 32^3 workload family: collisions
    # dominate, the equilibrium term is ten times stiffer
    p = inputs.cavity(64, 32, Kn=0.1, lid=0.16)
    m = {}
    for prec in (kgs.KGS_FP64, kgs.KGS_MIXED):
        ctx = kgs.kgs_setup(p, precision=prec)
        rc, n, res = kgs.kgs_iterate(ctx, 2)
        assert rc == kgs.KGS_OK
        m[prec] = kgs.kgs_moments(ctx)
    err = field_errors(m[kgs.KGS_MIXED], m[kgs.KGS_FP64])
    assert max(err.values()) <= 1e-5, err
    assert mirror_errors(m[kgs.KGS_FP64], 2) < 1e-12


def test_cavity64_z_mirror_symmetry_and_mass(kgs, cavity64):
    p, out = cavity64
    m64 = out[kgs.KGS_FP64][0]
    assert mirror_errors(m64, 2) < 1e-12
    assert mirror_errors(out[kgs.KGS_MIXED][0], 2) < 1e-5
    # closed cavity with the mass rescale: the total mass stays the initial one
    vol = 1.0 / p.ncell
    assert abs(m64[0].sum() * vol - 1.0) < 1e-12


def test_cavity64_rest_state(kgs):
    # lid at rest and walls at the gas temperature: the uniform state is the
    # fixed point (discrete wall normalisation), to rounding; 24 nodes on
    # [-6, 6] make the trapezoid moments of the Maxwellian exact to ~1e-14
    p = inputs.cavity(64, 24, Kn=1.0, lid=0.0, L_v=6.0)
    ctx = kgs.kgs_setup(p, precision=kgs.KGS_FP64)
    kgs.kgs_iterate(ctx, 2)
    m = kgs.kgs_moments(ctx)
    assert np.abs(m[0] - 1.0).max() < 1e-12 and np.abs(m[4] - 1.0).max() < 1e-12
    assert np.abs(m[1:4]).max() < 1e-12 and np.abs(m[5:8]).max() < 1e-12


def test_cube_mirror_symmetry_and_positivity(kgs):
    # Mach 2 past a cube centred in y and z: the y and z mirrors map the
    # solution to itself every iteration
    p = inputs.cube()
    ctx = kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
    rc, n, res = kgs.kgs_iterate(ctx, 2)
    assert rc == kgs.KGS_OK
    m = kgs.kgs_moments(ctx)
    solid = p.solid.astype(bool)
    assert np.all(m[:, solid] == 0.0)
    assert mirror_errors(m, 1) < 1e-5 and mirror_errors(m, 2) < 1e-5
    fluid = ~solid
    assert np.all(m[0][fluid] > 0) and np.all(m[4][fluid] > 0)


def test_batch64_instances_equal_single_contexts(kgs):
    probs = inputs.batch_cavities(n=64, seed=0)
    b = kgs.kgs_batch_setup(probs, precision=kgs.KGS_MIXED)
    rc, done, res = kgs.kgs_batch_iterate(b, 2)
    assert rc == kgs.KGS_OK and done == [2] * 64
    info = kgs.kgs_batch_info(b, 0)
    for i in (0, 17, 63):  # sampled instances
        c = kgs.kgs_setup(probs[i], precision=kgs.KGS_MIXED, v_per_cta=info["v_per_cta"],
                          block_z=info["block_z"])
        kgs.kgs_iterate(c, 2)
        # a lone instance may take the moment loop specialised to 16-node
        # lines, which the mixed-size batch cannot: same sums, FP32 rounding
        err = field_errors(kgs.kgs_batch_moments(b, i), kgs.kgs_moments(c))
        assert max(err.values()) <= 1e-6, (i, err)
