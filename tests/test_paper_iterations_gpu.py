"""Loose pin against the one iteration count the paper prints (Section 4.1):
the lid-driven cavity at Kn = 1, lid 0.1, reaches a relative change of 1e-9
in 36 iterations.  The paper's wall condition is the analytic normalisation
of Eq. (9) with the global mass rescale of Section 3.4.  The velocity grid
is halved here (32^3 instead of 64^3 nodes on the same interval) to keep the
FP64 run near a minute; at Kn = 1 the count is set by the gas-wall exchange,
not by the velocity resolution.  The residual reading and the precision of
the paper's run are not stated, so the count must fall within a factor of
1.5 of the printed one."""
import os

import pytest

from paper_1810_00348_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cavity_iterations.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_iterations_to_1e9_match_the_printed_count():
    from paper_1810_00348_gb300 import kgs
    kgs.load()
    g = golden()
    p = inputs.cavity(int(g["cells"]), int(g["velocities"]) // 2, Kn=g["kn"], lid=g["lid"],
                      wall_mode=inputs.WALL_ANALYTIC)
    ctx = kgs.kgs_setup(p, precision=kgs.KGS_FP64, tol=g["tol"], max_iters=200)
    rc, n, res = kgs.kgs_iterate(ctx, 0)
    assert rc == kgs.KGS_OK and res < g["tol"]
    assert g["iterations"] / 1.5 <= n <= g["iterations"] * 1.5, n
