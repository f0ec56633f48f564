"""The C-ABI library: it loads, exports every entry point include/gaborbank.h declares, and
validates arguments synchronously (no GPU needed for these checks)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gaborbank.h")


def _lib():
    from paper_1704_05231_gb300 import bank, build
    if not os.path.exists(bank.LIB_PATH):
        build.build()
    return bank.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:gb_status|int64_t|const char\s*\*)\s*(\w+)\s*\(", text, flags=re.M)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gabor_bank_create", "gabor_bank_filter", "gabor_bank_sdft", "gabor_bank_destroy",
              "gabor_bank_filter_batch", "gabor_bank_filter_host", "gabor_bank_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _lib()
    for n in declared_functions():
        assert hasattr(lib, n), f"{n} not exported"


def test_binding_signatures_cover_the_header():
    from paper_1704_05231_gb300 import bank
    missing = [n for n in declared_functions() if n not in bank.SIGNATURES]
    assert not missing


def _dbl(v):
    return (ctypes.c_double * max(1, len(v)))(*v)


def test_create_validates_before_touching_the_gpu():
    lib = _lib()
    h = ctypes.c_void_p()
    th, om = _dbl([0.0, 1.0]), _dbl([0.5])
    assert lib.gabor_bank_create(None, th, 2, om, _dbl([2.0]), 1, 3.0, 0, 0, 0) == -1
    assert lib.gabor_bank_create(ctypes.byref(h), th, 2, om, _dbl([0.0]), 1, 3.0, 0, 0, 0) == -1
    assert "sigma" in lib.gabor_bank_last_error().decode()
    assert lib.gabor_bank_create(ctypes.byref(h), th, 2, om, _dbl([-1.0]), 1, 3.0, 0, 0, 0) == -1
    assert lib.gabor_bank_create(ctypes.byref(h), th, 2, _dbl([math.nan]), _dbl([2.0]), 1, 3.0, 0, 0, 0) == -1
    assert lib.gabor_bank_create(ctypes.byref(h), th, 2, om, _dbl([2.0]), 1, 3.0, 7, 0, 0) == -1
    assert lib.gabor_bank_create(ctypes.byref(h), th, 0, om, _dbl([2.0]), 1, 3.0, 0, 0, 0) == -1
    # radius 3 * 60 = 180 px is above the library's limit
    assert lib.gabor_bank_create(ctypes.byref(h), th, 2, om, _dbl([60.0]), 1, 3.0, 0, 0, 0) == -4
    assert h.value is None


def test_calls_on_null_handle_fail_cleanly():
    lib = _lib()
    buf = (ctypes.c_float * 16)()
    assert lib.gabor_bank_filter(None, buf, 4, 4, 4, buf, None) == -1
    assert lib.gabor_bank_sdft(None, buf, 4, 4, 4, 1.0, 4, 4, 0, buf, None) == -1
    assert lib.gabor_bank_set_option(None, 1, 0) == -1
    assert lib.gabor_bank_destroy(None) == 0
    assert lib.gabor_bank_output_elems(None, 4, 4) == 0
    assert b"sm_103a" in lib.gabor_bank_version()


def test_create_without_gpu_reports_cuda_error():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    lib = _lib()
    h = ctypes.c_void_p()
    rc = lib.gabor_bank_create(ctypes.byref(h), _dbl([0.0]), 1, _dbl([0.5]), _dbl([2.0]), 1, 3.0, 0, 0, 0)
    assert rc == -3
    assert h.value is None
    assert lib.gabor_bank_last_error().decode()
