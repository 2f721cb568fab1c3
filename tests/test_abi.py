"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads, and
exports every function include/*.h declares, with a binding for each."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ig_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ig_create", "ig_mesh_upload", "ig_assemble", "ig_solve", "ig_adjoint", "ig_mesh_free",
                     "ig_destroy", "ig_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2602_12105_gb300 import _native, build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    unbound = [n for n in sorted(_declared()) if n not in _native.SIGNATURES]
    assert not unbound, unbound


def test_status_strings_without_gpu():
    from paper_2602_12105_gb300 import _native
    lib = _native.load()
    assert lib.ig_status_str(0) == b"ok"
    assert b"converge" in lib.ig_status_str(4)


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2602_12105_gb300 import _native, api
    with pytest.raises(_native.NativeLibraryError):
        api.Context()


def test_oracle_is_not_reachable_from_the_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2602_12105_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(path).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), path
            assert "oracle.c" not in txt, path
