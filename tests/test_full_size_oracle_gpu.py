"""The benchmark's workload family at full size (64^3 cells x 32^3
velocities, the launch configuration the benchmark times) against the FP64
oracle after two outer iterations from the uniform start.  The oracle sweeps
contiguous velocity ranges on all host cores (about 1.7e10 cell updates per
iteration, close to three minutes on 16 cores); the test is skipped on hosts
with fewer than 8 cores or without a threaded oracle build.  Both Knudsen
numbers of the workload family run: Kn = 1 (the benchmark's case) and
Kn = 0.1.
"""
import os

import pytest

from oracle import Oracle, parallel_build
from paper_1810_00348_gb300 import inputs
from tests.parity import assert_fields_close, assert_rho_w_close

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


KNUDSEN = [1.0, 0.1]


@pytest.mark.parametrize("kn", KNUDSEN)
def test_cavity64_two_iterations_against_oracle(kgs, kn):
    cores = os.cpu_count() or 1
    if cores < 8 or not parallel_build():
        pytest.skip("the full-size oracle needs a threaded build and at least 8 host cores")
    p = inputs.cavity(64, 32, Kn=kn, lid=0.16)
    o = Oracle(p, threads=cores)
    o.iterate(2)
    ref, ref_rw = o.macros(), o.rho_w()
    for prec, tol in ((kgs.KGS_FP64, 1e-10), (kgs.KGS_MIXED, 1e-5)):
        ctx = kgs.kgs_setup(p, precision=prec)  # autotuned shape, as the benchmark
        rc, done, _ = kgs.kgs_iterate(ctx, 2)
        assert rc == kgs.KGS_OK and done == 2
        assert_fields_close(kgs.kgs_moments(ctx), ref, tol, what="64^3 x 32^3, Kn=%g, precision %d" % (kn, prec))
        if prec == kgs.KGS_FP64:
            assert_rho_w_close(kgs.kgs_rho_w(ctx), ref_rw, 1e-10)
