"""Argument checks of the C ABI, on the host only: every malformed problem
or option set is rejected with KGS_EINVAL by kgs_setup (and the entry points
that take a problem directly) before any CUDA call is made, so these run
without a GPU.  Each case breaks one rule stated in include/kgs.h and starts
from a valid cavity, so that the rejection is due to that rule alone."""
import math

import numpy as np
import pytest

from paper_1810_00348_gb300 import inputs


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


def cavity():
    return inputs.cavity(4, 4)


def with_(p, **kw):
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def bad_width():
    p = cavity()
    p.dy = np.array([0.25, 0.0, 0.25, 0.5])
    return p


def bad_weight():
    p = cavity()
    p.w_z = p.w_z.copy()
    p.w_z[1] = 0.0
    return p


def bad_node():
    p = cavity()
    p.xi_x = p.xi_x.copy()
    p.xi_x[0] = math.nan
    return p


def inflow(p=None, rho_in=1.0, T_in=1.0):
    p = p or cavity()
    p.face_type = list(p.face_type)
    p.face_type[0] = inputs.FACE_INFLOW
    p.rho_in, p.T_in = rho_in, T_in
    return p


def solid(p=None, T_solid=1.0):
    p = p or cavity()
    s = np.zeros((p.nz, p.ny, p.nx), np.uint8)
    s[1, 1, 1] = 1
    p.solid, p.T_solid = s, T_solid
    return p


def stretched_cells():
    p = cavity()
    p.dx = np.array([0.2, 0.25, 0.25, 0.3])
    return p


PROBLEMS = {
    "zero cell width": bad_width,
    "zero quadrature weight": bad_weight,
    "non-finite velocity node": bad_node,
    "Kn = 0": lambda: with_(cavity(), Kn=0.0),
    "negative Kn": lambda: with_(cavity(), Kn=-1.0),
    "Pr = 0": lambda: with_(cavity(), Pr=0.0),
    "omega above 1.5": lambda: with_(cavity(), omega=2.0),
    "negative omega": lambda: with_(cavity(), omega=-0.1),
    "wall at T = 0": lambda: with_(cavity(), T_w=[1.0, 1.0, 0.0, 1.0, 1.0, 1.0]),
    "unknown face type": lambda: with_(cavity(), face_type=[inputs.FACE_WALL] * 5 + [7]),
    "inflow with rho = 0": lambda: inflow(rho_in=0.0),
    "inflow with T = 0": lambda: inflow(T_in=0.0),
    "solid at T = 0": lambda: solid(T_solid=0.0),
    "unknown wall normalisation": lambda: with_(cavity(), wall_mode=5),
    # Kn = infinity with a zero node on every axis: a velocity with no equation
    "free-molecular with xi = 0": lambda: inputs.cavity(4, 5, Kn=math.inf),
    "order 3": lambda: with_(cavity(), order=3),
    "order 2 with a solid cell": lambda: with_(solid(), order=2),
    "order 2 with a free-stream side": lambda: with_(inflow(), order=2),
    "order 2 on unequal cell widths": lambda: with_(stretched_cells(), order=2),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_malformed_problem_is_rejected(kgs, name):
    p = PROBLEMS[name]()
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(p, precision=kgs.KGS_MIXED)
    assert e.value.code == kgs.KGS_EINVAL, kgs.kgs_strerror(e.value.code)


OPTIONS = {
    "unknown precision": dict(precision=7),
    "v_per_cta 64": dict(v_per_cta=64),
    "FP64 with 256 velocities per block": dict(precision="fp64", v_per_cta=256),
    "negative block depth": dict(block_z=-1),
    "velocity planes out of range": dict(vz=(2, 5)),
    "empty velocity plane range": dict(vz=(2, 2)),
    "deviation source in FP64": dict(precision="fp64", dev_source=1),
    "deviation source flag 2": dict(dev_source=2),
}


@pytest.mark.parametrize("name", sorted(OPTIONS))
def test_malformed_options_are_rejected(kgs, name):
    kw = dict(OPTIONS[name])
    kw["precision"] = {"fp64": kgs.KGS_FP64, None: kgs.KGS_MIXED}.get(kw.get("precision"), kw.get("precision"))
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(cavity(), **kw)
    assert e.value.code == kgs.KGS_EINVAL


def test_deviation_source_needs_walls_on_every_side(kgs):
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_setup(inflow(), precision=kgs.KGS_MIXED, dev_source=1)
    assert e.value.code == kgs.KGS_EINVAL


def test_solve_arguments(kgs):
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_solve(cavity(), tol=0.0)
    assert e.value.code == kgs.KGS_EINVAL
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_solve(cavity(), tol=1e-6, max_iters=0)
    assert e.value.code == kgs.KGS_EINVAL


def test_noalloc_rejects_before_touching_the_device(kgs):
    # aliased state buffers, then a problem too large for the fixed scratch
    # array (face planes of 64^2 cells x 32^3 velocities alone exceed it);
    # the pointers are never dereferenced
    a, b = 1 << 20, 2 << 20
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_iterate_noalloc(cavity(), a, b, a, b + 64)
    assert e.value.code == kgs.KGS_EINVAL
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_iterate_noalloc(inputs.cavity(64, 32), a, b, a + 4096, b + 4096, precision=kgs.KGS_MIXED)
    assert e.value.code == kgs.KGS_EINVAL
    with pytest.raises(kgs.KgsError) as e:
        kgs.kgs_iterate_noalloc(bad_width(), a, b, a + 4096, b + 4096)
    assert e.value.code == kgs.KGS_EINVAL


def test_error_messages(kgs):
    for code in (kgs.KGS_EINVAL, kgs.KGS_ENOMEM, kgs.KGS_ECUDA, kgs.KGS_EDIVERGED, kgs.KGS_ETIMEOUT,
                 kgs.KGS_EFORMAT, kgs.KGS_NOTCONVERGED):
        msg = kgs.kgs_strerror(code)
        assert msg and msg != kgs.kgs_strerror(12345)
