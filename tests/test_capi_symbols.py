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


def test_header_is_plain_c(tmp_path):
    """include/npbs.h is a C header: a C99 translation unit that includes it
    compiles warning-free (no C++-only constructs in the ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use_header.c"
    src.write_text('#include "npbs.h"\nint main(void) { npbs_ctx* c = 0; (void)c; return (int)NPBS_OK; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
                        "-c", str(src), "-o", str(tmp_path / "use_header.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
