"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/ks.h declares (no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest


def test_library_exports_header_symbols():
    from paper_2311_01598_gb300 import build, ks
    build.build()
    L = ctypes.CDLL(ks.lib_path())
    names = ks.exported_symbols()
    assert "ks_switch" in names and "ks_switch_batch" in names and "ks_params_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_argument_errors_before_any_launch():
    """Argument errors are reported on the host with a message (no device)."""
    from paper_2311_01598_gb300 import ks
    L = ks.lib()
    h = ctypes.c_void_p()
    assert L.ks_params_create(9, 3, 1, 3, None, None, 50, ctypes.byref(h)) == ks.KS_EUNSUPPORTED
    assert b"logN" in L.ks_last_error()
    assert L.ks_params_create(12, 3, 1, 4, None, None, 50, ctypes.byref(h)) == ks.KS_EINVAL
    assert L.ks_params_create(12, 3, 1, 3, None, None, 57, ctypes.byref(h)) == ks.KS_EUNSUPPORTED
    assert L.ks_switch(None, None, 1, None, None, None, 0, None) == ks.KS_EINVAL
    assert L.ks_switch_batch(None, 0, None, 0, None) == ks.KS_EINVAL
    assert L.ks_ntt(None, 0, 1, None, 0, None) == ks.KS_EINVAL


def test_header_declares_the_boundary():
    from paper_2311_01598_gb300 import ks
    names = set(ks.exported_symbols())
    for n in ("ks_params_create", "ks_params_destroy", "ks_keygen_upload", "ks_key_upload_raw",
              "ks_key_destroy", "ks_switch", "ks_switch_batch", "ks_last_error"):
        assert n in names, n


def test_product_path_does_not_import_oracle():
    """The product package never references the oracle."""
    pkg = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2311_01598_gb300")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(root, f)) as fh:
                    text = fh.read()
                assert not re.search(r"\boracle\b.*import|import\s+oracle|from\s+oracle|ks_oracle", text), f


def test_header_is_plain_c():
    """include/ks.h compiles as strict C99 (a C caller needs no C++ and no
    torch types), every entry point referenced once."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    inc = os.path.join(root, "include")
    text = open(os.path.join(inc, "ks.h")).read()
    names = sorted(set(re.findall(r"^\w[\w\s\*]*?\b(ks_\w+)\s*\(", text, re.M)))
    assert "ks_switch" in names and "ks_switch_batch" in names
    body = "\n".join(f"    (void)&{n};" for n in names)
    src = f'#include "ks.h"\nint main(void)\n{{\n{body}\n    return 0;\n}}\n'
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "t.c")
        open(c, "w").write(src)
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + inc, "-fsyntax-only", c],
                           capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
