"""The C-ABI library builds, loads and exports every symbol its header declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2202_08612_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mlcc3_\w+)\s*\(", text))
    return names


def test_exports_match_header(lib):
    names = declared_symbols()
    assert "mlcc3_jacobian_left" in names and len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.EXPORTS) == names


def test_argument_errors_without_gpu(lib):
    """Invalid dimensions are rejected before any CUDA call."""
    binding.load()
    L = binding._lib
    h = ctypes.c_void_p()
    bad = binding._Dims(4, 10, 5, 3, 8, None)      # n_o > N_O
    assert L.mlcc3_create(ctypes.byref(h), ctypes.byref(bad), 0, None) == -1
    assert b"dimensions" in L.mlcc3_last_error()
    ok = binding._Dims(4, 10, 2, 3, 8, None)
    assert L.mlcc3_create(ctypes.byref(h), ctypes.byref(ok), 7, None) == -1
    assert L.mlcc3_create(None, ctypes.byref(ok), 0, None) == -1
    assert L.mlcc3_triples_omega(None, None, None) == -1
    assert L.mlcc3_debug_nbatches(None) == -1
    assert L.mlcc3_set_param(None, b"tc_kcap", 8) == -1
    # the FP64-accurate GEMM: null operands, bad sizes, leading dimensions below
    # the row length and slice counts outside 2..6 fail before any CUDA call
    a = np.zeros((4, 8))
    P = a.ctypes.data
    for args in ((None, 8, P, 8, P, 4, 4, 4, 8, 5), (P, 8, P, 8, P, 4, 0, 4, 8, 5),
                 (P, 7, P, 8, P, 4, 4, 4, 8, 5), (P, 8, P, 8, P, 3, 4, 4, 8, 5),
                 (P, 8, P, 8, P, 4, 4, 4, 8, 1), (P, 8, P, 8, P, 4, 4, 4, 8, 7)):
        assert L.mlcc3_fp64emu_gemm(*args, None) == -1, args
        assert b"fp64emu" in L.mlcc3_last_error()


def test_ptr_marshalling():
    a = np.zeros((3, 4))
    assert binding._ptr(a) == a.ctypes.data
    with pytest.raises(ValueError):
        binding._ptr(np.zeros(3, dtype=np.float32))
