"""The oracle's pins catch plausible mistakes: each case plants one
single-line bug in a copy of the oracle source (a dropped constant, a wrong
side, a missing term, a scaled coefficient) and requires the pin suite to
fail on it.  Test infrastructure only; everything runs on the CPU in a
temporary copy, the committed oracle is not touched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("gas constant dropped from the Maxwellian exponent",
     "exp(-c2 / (2.0 * R_GAS * T))", "exp(-c2 / (2.0 * T))"),
    ("upwind neighbour taken on the downwind side",
     "int face = 2 * d + (xi[d] > 0.0 ? 0 : 1); /* upwind side */",
     "int face = 2 * d + (xi[d] > 0.0 ? 1 : 0); /* upwind side */"),
    ("wall velocity dropped from the wall Maxwellian",
     "U[0] = s->p.U_w[kind][0];", "U[0] = 0.0;"),
    ("Shakhov term without its (1 - Pr) factor",
     "(1.0 - s->p.Pr) * cq / (5.0 * p * R_GAS * T)", "cq / (5.0 * p * R_GAS * T)"),
    ("heat flux taken about zero instead of the new U",
     "cc[d] = xi[d] - U[(size_t)d * nc + c];", "cc[d] = xi[d];"),
    ("relaxation rate scaled",
     "    return p / mu;", "    return 2.0 * p / mu;"),
    ("viscosity law with T^(omega - 1) in place of T^omega",
     "double mu = s->mu_ref * pow(T, s->p.omega);", "double mu = s->mu_ref * pow(T, s->p.omega - 1.0);"),
    ("pressure in the relaxation time without the gas constant",
     "double p = rho * R_GAS * T;\n    return p / mu;", "double p = rho * T;\n    return p / mu;"),
    ("lagged heat flux taken about the new velocity",
     "        Uq = Ulag;", "        Uq = U;"),
    ("incoming wall flux without the quadrature weight",
     "return xn < 0.0 ? w * (-xn) * f : 0.0;", "return xn < 0.0 ? (-xn) * f : 0.0;"),
    ("second-order stencil with the first-order diagonal",
     "den += 1.5 * coef;", "den += coef;"),
    ("second upwind neighbour with the wrong weight",
     "num += coef * (2.0 * f[n] - 0.5 * f[n2]);", "num += coef * (2.0 * f[n] - 1.0 * f[n2]);"),
    ("second-order stencil reusing the first upwind neighbour",
     "int n2 = n >= 0 ? neighbour(s, n, face) : -1;", "int n2 = n;"),
    ("temperature without the kinetic energy subtracted",
     "double T = (rhoE[c] - 0.5 * rho[c] * (u0 * u0 + u1 * u1 + u2 * u2)) / (1.5 * rho[c] * R_GAS);",
     "double T = rhoE[c] / (1.5 * rho[c] * R_GAS);"),
]


@pytest.mark.slow
@pytest.mark.parametrize("label,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_fail_on_a_planted_bug(tmp_path, label, old, new):
    src = open(os.path.join(ROOT, "oracle", "kgs_oracle.c")).read()
    assert src.count(old) == 1, "the line to mutate is not unique: " + label
    for d in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    pkg = tmp_path / "paper_1810_00348_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, "paper_1810_00348_gb300", f), pkg / f)
    (tmp_path / "oracle" / "kgs_oracle.c").write_text(src.replace(old, new))
    # the mutant must build: the pins, not the compiler, have to reject it
    b = subprocess.run([sys.executable, "-c", "from oracle import build; build.build_oracle(force=True)"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=300)
    assert b.returncode == 0, b.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, "no pin caught: %s\n%s" % (label, r.stdout[-2000:])
    # a pin's assertion rejected the mutant, not an exception raised by it
    for exc in ("IndexError", "ValueError", "TypeError", "NameError", "AttributeError", "OSError"):
        assert exc not in r.stdout, r.stdout[-2000:]
    assert "assert" in r.stdout, r.stdout[-2000:]
