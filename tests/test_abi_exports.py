"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/kgs.h declares (no compute call is made here)."""
import ctypes
import os
import re

from paper_1810_00348_gb300 import build as kbuild
from paper_1810_00348_gb300 import kgs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(kgs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    path = kbuild.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    assert set(declared_functions()) <= set(kgs.SIGNATURES)
    kgs.load()  # declares argtypes for every symbol; no device call


def test_strerror_without_gpu():
    lib = kgs.load()
    assert lib.kgs_strerror(kgs.KGS_EINVAL) == b"invalid argument"
    assert lib.kgs_strerror(12345) == b"unknown error code"
