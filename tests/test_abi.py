"""The C ABI library builds for sm_103a, loads, and exports every entry point declared in include/vie.h."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vie.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(vie_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib_path():
    import paper_1902_02196_gb300 as vie

    return vie.build()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("vie_setup", "vie_matvec", "vie_solve", "vie_destroy", "vie_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vie_[a-z_0-9]+)", out))
    missing = declared() - exported
    assert not missing, missing


def test_library_loads_and_binding_matches(lib_path):
    import paper_1902_02196_gb300 as vie

    lib = ctypes.CDLL(lib_path)
    for n in declared():
        assert hasattr(lib, n)
    assert set(vie.EXPORTS) == declared()
    assert vie.vie_strerror(vie.VIE_EINVAL) == "invalid argument"
    assert vie.vie_strerror(vie.VIE_NOT_CONVERGED).startswith("solver")
