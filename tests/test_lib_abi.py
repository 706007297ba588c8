"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

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


def test_static_restrict_argument_checks_on_host():
    # the binding's checks of spnet_pc_restrict_static's tensors run before any launch;
    # exercised here with stand-ins that report CUDA placement without a GPU
    import torch

    from paper_2207_07488_gb300.spnet import check_static_restrict_args

    class T:
        def __init__(self, n, dtype=torch.float64, contiguous=True, device="cuda:0"):
            self.n, self.dtype, self._c, self.device = n, dtype, contiguous, device
            self.is_cuda = device.startswith("cuda")

        def is_contiguous(self):
            return self._c

        def numel(self):
            return self.n

    T.__module__ = "torch.stand_in"
    check_static_restrict_args(T(10), T(4), 10, 4)
    check_static_restrict_args(T(10), T(5), 10, 4)   # a longer rc is fine
    bad = [(T(10, dtype=torch.float32), T(4)), (T(10), T(4, dtype=torch.float32)),
           (T(10, contiguous=False), T(4)), (T(10), T(4, contiguous=False)),
           (T(9), T(4)), (T(11), T(4)), (T(10), T(3)), (T(10, device="cpu"), T(4)),
           (T(10), T(4, device="cuda:1")), (np.zeros(10), T(4))]
    for a, b in bad:
        with pytest.raises(ValueError):
            check_static_restrict_args(a, b, 10, 4)


def test_record_iterates_argument_checks_on_host():
    # the binding's checks of spnet_pc_record_iterates' buffer, with stand-ins that
    # report CUDA placement without a GPU
    import torch

    from paper_2207_07488_gb300.spnet import check_record_args

    class T:
        def __init__(self, shape, dtype=torch.float64, contiguous=True, device="cuda:0"):
            self.shape, self.dtype, self._c, self.device = shape, dtype, contiguous, device
            self.is_cuda = device.startswith("cuda")

        def is_contiguous(self):
            return self._c

        def dim(self):
            return len(self.shape)

    T.__module__ = "torch.stand_in"
    check_record_args(T((5, 10)), 10)
    check_record_args(T((1, 10)), 10)
    for bad in (T((5, 9)), T((0, 10)), T((50,)), T((5, 10), dtype=torch.float32), T((5, 10), contiguous=False),
                T((5, 10), device="cpu"), np.zeros((5, 10))):
        with pytest.raises(ValueError):
            check_record_args(bad, 10)
