"""Failure detection without a GPU fault: a NaN planted on the host in one
wall density makes the next iteration produce non-finite moments, which the
closure reports as KGS_EDIVERGED after that iteration; the context stays
usable and iterates normally once a clean state is loaded."""
import numpy as np
import pytest

from paper_1810_00348_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_wall_density_is_reported_as_divergence(kgs, precision):
    p = inputs.cavity(8, 8, Kn=0.5, lid=0.2)
    prec = kgs.KGS_FP64 if precision == "fp64" else kgs.KGS_MIXED
    ctx = kgs.kgs_setup(p, precision=prec)
    clean = kgs.kgs_save(ctx)
    rw = np.array(kgs.kgs_rho_w(ctx))
    flat = rw.reshape(-1)
    flat[np.flatnonzero(flat)[0]] = np.nan  # one wall face of one cell
    kgs.kgs_set_rho_w(ctx, rw)
    rc, done, _ = kgs.kgs_iterate(ctx, 3)
    assert rc == kgs.KGS_EDIVERGED and done == 1
    assert kgs.kgs_load(ctx, clean) == kgs.KGS_OK
    rc, done, res = kgs.kgs_iterate(ctx, 2)
    assert rc == kgs.KGS_OK and done == 2 and np.isfinite(res)
    m = kgs.kgs_moments(ctx)
    assert np.all(np.isfinite(m))
