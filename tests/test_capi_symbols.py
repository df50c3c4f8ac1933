"""The C-ABI library loads and exports every function include/*.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2603_18527_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ["cbs_apply", "cbs_solve", "npbs_solve", "fgmres_solve", "npbs_create", "npbs_build_potential"]:
        assert fn in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2603_18527_gb300 import capi
    missing = [n for n in _declared() if n not in capi.exported_symbols()]
    assert not missing, missing


def test_version_string_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.npbs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.npbs_version()
