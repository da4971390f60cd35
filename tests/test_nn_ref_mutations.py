"""The network reference's pins catch plausible mistakes: each case plants
one single-line bug in a copy of `oracle/nn_ref.py` (a mirrored tap, a scaled
or misplaced gradient, a missing ReLU mask, a wrong loss derivative, the
wrong rounding tie) and requires the pin suite to fail on it.  CPU only; the
committed reference is not touched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("forward tap mirrored",
     'y += np.einsum("zyxi,oi->zyxo", xp[kz:kz + D, ky:ky + H, kx:kx + Wd], W[t])',
     'y += np.einsum("zyxi,oi->zyxo", xp[kz:kz + D, ky:ky + H, kx:kx + Wd], W[26 - t])'),
    ("weight gradient scaled",
     'dW[t] = np.einsum("zyxo,zyxi->oi", dy, xp[kz:kz + D, ky:ky + H, kx:kx + Wd])',
     'dW[t] = 0.5 * np.einsum("zyxo,zyxi->oi", dy, xp[kz:kz + D, ky:ky + H, kx:kx + Wd])'),
    ("data gradient through the mirrored tap",
     'dxp[kz:kz + D, ky:ky + H, kx:kx + Wd] += np.einsum("zyxo,oi->zyxi", dy, W[t])',
     'dxp[kz:kz + D, ky:ky + H, kx:kx + Wd] += np.einsum("zyxo,oi->zyxi", dy, W[26 - t])'),
    ("bias gradient averaged instead of summed",
     "db = dy.sum(axis=(0, 1, 2))", "db = dy.mean(axis=(0, 1, 2))"),
    ("ReLU mask dropped in the backward pass",
     "g = dx * (acts[l] > 0.0)  # ReLU of layer l-1", "g = dx  # ReLU of layer l-1"),
    ("loss derivative without the factor 2",
     "return float((d * d).sum() / cnt), 2.0 * d / cnt", "return float((d * d).sum() / cnt), d / cnt"),
    ("bf16 ties rounded up instead of to even",
     "u = (u + 0x7FFF + lsb) & 0xFFFF0000", "u = (u + 0x8000) & 0xFFFF0000"),
]


@pytest.mark.slow
@pytest.mark.parametrize("label,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_nn_pins_fail_on_a_planted_bug(tmp_path, label, old, new):
    src = open(os.path.join(ROOT, "oracle", "nn_ref.py")).read()
    assert src.count(old) == 1, "the line to mutate is not unique: " + label
    for d in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    pkg = tmp_path / "paper_1810_00348_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, "paper_1810_00348_gb300", f), pkg / f)
    (tmp_path / "oracle" / "nn_ref.py").write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_nn_ref_pins.py", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, "no pin caught: %s\n%s" % (label, r.stdout[-2000:])
    # a pin's assertion rejected the mutant, not an exception raised by it
    for exc in ("IndexError", "ValueError", "TypeError", "NameError", "AttributeError", "SyntaxError"):
        assert exc not in r.stdout, r.stdout[-2000:]
    assert "assert" in r.stdout, r.stdout[-2000:]
