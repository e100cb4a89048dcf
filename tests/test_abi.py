"""The C-ABI library loads and exports every entry point include/mpcg.h declares
(no compute: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("mpcg_", "mg_"))))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_12833_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("mg_hierarchy_setup", "mpcg_solve", "mg_hierarchy_destroy", "mpcg_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2402_12833_gb300 import mpcg
    assert set(_declared()) <= set(mpcg._SIGS)


def test_options_struct_matches_header_defaults(lib):
    from paper_2402_12833_gb300 import mpcg
    mpcg._lib = None
    o = mpcg.mpcg_default_options()
    assert o.m == 5 and o.nu == 2 and abs(o.omega - 2 / 3) < 1e-15
    assert o.precision == mpcg.MPCG_FP64
