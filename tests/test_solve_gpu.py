"""kgs_solve: mixed-precision iterations while they make progress, then FP64
to the tolerance.  The result must be the FP64 fixed point (the same field
as a plain FP64 solve, within what the tolerance leaves), reached with fewer
FP64 iterations than a plain FP64 solve from the same start."""
import numpy as np
import pytest

from paper_1810_00348_gb300 import inputs
from tests.parity import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kgs():
    from paper_1810_00348_gb300 import kgs as k
    k.load()
    return k


@pytest.mark.parametrize("kn", [0.2, 0.05])
def test_solve_reaches_the_fp64_fixed_point(kgs, kn):
    p = inputs.cavity(16, 16, Kn=kn, lid=0.2)
    rc, m, n_mixed, n_fp64, res = kgs.kgs_solve(p, tol=1e-8, max_iters=3000)
    assert rc == kgs.KGS_OK and res < 1e-8
    assert n_mixed > 0
    c = kgs.kgs_setup(p, precision=kgs.KGS_FP64, tol=1e-8, max_iters=3000)
    rc2, n_plain, res2 = kgs.kgs_iterate(c, 0)
    assert rc2 == kgs.KGS_OK
    assert n_fp64 < n_plain
    err = field_errors(m, kgs.kgs_moments(c))
    # both stop within the tolerance of the same fixed point; the remaining
    # distance is of the order of tol / (1 - contraction rate)
    assert max(err.values()) < 1e-5, err


def test_solve_from_a_guess_and_budget(kgs):
    p = inputs.cavity(12, 12, Kn=0.5, lid=0.1)
    rc, m, nm1, nd1, _ = kgs.kgs_solve(p, tol=1e-7)
    # from the converged field: the mixed phase only drifts into its noise
    # band and stalls, and the FP64 phase needs only a few iterations
    rc, m2, n_mixed, n_fp64, res = kgs.kgs_solve(p, initial=m, tol=1e-7)
    assert rc == kgs.KGS_OK and n_fp64 <= 10 and n_mixed + n_fp64 < nm1 + nd1, (n_mixed, n_fp64, nm1, nd1)
    assert max(field_errors(m2, m).values()) < 1e-5
    # a budget too small to converge is reported, not raised
    rc, _, n_mixed, n_fp64, res = kgs.kgs_solve(p, tol=1e-12, max_iters=6)
    assert rc == kgs.KGS_NOTCONVERGED and res > 1e-12 and n_mixed + n_fp64 == 6
