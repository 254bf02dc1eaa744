"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/rad.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(rad_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import paper_2302_04283_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2302_04283_gb300 import build
        build.build()
    return pkg.LIB_PATH


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for s in ("rad_init_angles", "rad_set_metric", "rad_step", "rad_moments", "rad_step_adjoint"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_the_c_abi(libpath):
    import paper_2302_04283_gb300 as pkg
    for s in declared_symbols():
        assert hasattr(pkg, s), s
