"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/swedg.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_1804_02221_gb300 import build as B
from paper_1804_02221_gb300 import swedg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "swedg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(swe_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("swe_create", "swe_rhs", "swe_limit", "swe_max_dt", "swe_step", "swe_mass",
              "swe_entropy", "swe_destroy", "swe_last_error"):
        assert s in syms


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} declared in swedg.h but not exported"
    # the Python binding names the same entry points
    assert set(swedg.SYMBOLS) == set(declared_symbols())


def test_last_error_callable_without_gpu():
    lib = swedg.lib()
    assert isinstance(lib.swe_last_error(), bytes)
