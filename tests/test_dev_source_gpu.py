"""The deviation-form FP32 source of the first-order sweep (kgs_opts.dev_source
= 1: rtau (f^S - M_ref) from the small differences of the exponents of f^S and
of the reference Maxwellian) against the FP64 oracle at 1e-5, per field and
per component, on the cases the mixed tests use; and its purpose: a lower
residual floor of the mixed iteration than the default form's.
"""
import os

import numpy as np
import pytest

from oracle import Oracle, parallel_build
from paper_1810_00348_gb300 import inputs
from tests.parity import assert_components_close, assert_fields_close, assert_rho_w_close

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def oracle_threads():
    return (os.cpu_count() or 1) if parallel_build() else 1


def run_dev(kgs, p, n_iter, macros=None, **kw):
    ctx = kgs.kgs_setup(p, precision=kgs.KGS_MIXED, dev_source=1, **kw)
    if macros is not None:
        kgs.kgs_set_initial(ctx, macros)
    rc, done, _ = kgs.kgs_iterate(ctx, n_iter)
    assert rc == kgs.KGS_OK and done == n_iter
    return kgs.kgs_moments(ctx), kgs.kgs_rho_w(ctx)


def test_dev_source_cavity64_8_from_rest(kgs):
    p = inputs.cavity(64, 8, Kn=1.0, lid=0.16)
    o = Oracle(p, threads=oracle_threads())
    o.iterate(1)
    m, rw = run_dev(kgs, p, 1)
    assert_fields_close(m, o.macros(), MIXED_TOL, what="dev source 64^3 x 8^3")
    assert_components_close(m, o.macros(), MIXED_TOL, what="dev source 64^3 x 8^3")
    assert_rho_w_close(rw, o.rho_w(), MIXED_TOL)


@pytest.mark.parametrize("v_per_cta", [128, 256])
def test_dev_source_ragged_random_state(kgs, v_per_cta):
    p = inputs.cavity([19, 17, 35], [9, 8, 7], L_v=3.5, lid=0.2, Kn=0.4)
    mac = inputs.random_macros(p, 301)
    o = Oracle(p, mac, threads=oracle_threads())
    o.iterate(2)
    m, rw = run_dev(kgs, p, 2, macros=mac, v_per_cta=v_per_cta)
    what = "dev source ragged, %d velocities per CTA" % v_per_cta
    assert_fields_close(m, o.macros(), MIXED_TOL, what=what)
    assert_components_close(m, o.macros(), MIXED_TOL, what=what)
    assert_rho_w_close(rw, o.rho_w(), MIXED_TOL)


def test_dev_source_24cells_32velocities(kgs):
    """The 16-node-line moment loop with the unrolled diagonals, Kn 0.1."""
    p = inputs.cavity(24, 32, Kn=0.1, lid=0.16)
    o = Oracle(p, threads=oracle_threads())
    o.iterate(1)
    m, rw = run_dev(kgs, p, 1)
    assert_fields_close(m, o.macros(), MIXED_TOL, what="dev source 24^3 x 32^3")
    assert_components_close(m, o.macros(), MIXED_TOL, what="dev source 24^3 x 32^3")
    assert_rho_w_close(rw, o.rho_w(), MIXED_TOL)


def test_dev_source_lowers_the_residual_floor(kgs):
    p = inputs.cavity(16, 16, Kn=0.2, lid=0.16)
    floors = []
    for dev in (0, 1):
        ctx = kgs.kgs_setup(p, precision=kgs.KGS_MIXED, dev_source=dev)
        res = [kgs.kgs_iterate(ctx, 1)[2] for _ in range(300)]
        floors.append(min(res[150:]))
    assert floors[1] < 0.5 * floors[0], floors


def test_dev_source_rejections(kgs):
    p = inputs.cavity(12, 8, Kn=0.5)
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(p, precision=kgs.KGS_FP64, dev_source=1)
    assert e.value.code == kgs.KGS_EINVAL
    q = inputs.cavity(12, 8, Kn=0.5)
    q.dx = np.linspace(0.5, 1.5, q.nx) / q.nx
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(q, precision=kgs.KGS_MIXED, dev_source=1)
    assert e.value.code == kgs.KGS_EINVAL
    f = inputs.cavity(12, 8, Kn=0.5)
    f.face_type = [inputs.FACE_INFLOW] * 6
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(f, precision=kgs.KGS_MIXED, dev_source=1)
    assert e.value.code == kgs.KGS_EINVAL
