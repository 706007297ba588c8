"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point (no GPU)."""
import ctypes
import os
import re

from paper_2207_07488_gb300 import build as B
from paper_2207_07488_gb300 import spnet

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "spnet.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+([a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("build_network_operator", "setup_preconditioner", "pcg_solve", "spnet_assemble"):
        assert must in names
    assert set(names) == set(spnet.EXPORTED)


def test_library_loads_and_exports_every_symbol():
    B.build()
    lib = ctypes.CDLL(B.LIB)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_reports_errors_without_a_gpu():
    lib = spnet.load()
    # a null operator is rejected by argument checks before any device call
    rc = lib.setup_preconditioner(None, 0.5, None, None, ctypes.byref(ctypes.c_void_p()))
    assert rc == -1
    assert "null operator" in spnet.last_error()


def test_every_entry_point_has_argument_types():
    # without argtypes ctypes passes Python ints as C int: a 64-bit pointer would be cut to 32 bits
    lib = spnet.load()
    for name in spnet.EXPORTED:
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert fn.restype is ctypes.c_int, name


def test_argument_types_match_the_header():
    # each declaration's parameter count in the header equals the binding's argtypes
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    lib = spnet.load()
    for name, params in re.findall(r"^\s*int\s+([a-z_0-9]+)\s*\(([^)]*)\)\s*;", src, flags=re.M):
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, name
