"""The allocation-free SDFT entry point (gabor_sdft_noalloc) against gabor_bank_sdft.

Callers such as custom allocators or fixed-budget applications cannot call cudaMalloc; for
them the library offers gabor_sdft_noalloc, which keeps its tables in a fixed device array.
This file runs last so that a failure here does not hide the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    from paper_1704_05231_gb300 import bank
    lib = bank.load_library()
    fn = lib.gabor_sdft_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return lib, fn


def test_noalloc_matches_handle_path_two_calls():
    import torch
    from paper_1704_05231_gb300 import GaborBank
    lib, fn = _noalloc_fn()
    stream = torch.cuda.current_stream()
    # Two calls in a row with different windows: the shared table must be rebuilt each time.
    for (H, W, sigma, M) in ((70, 150, 4.0, 16), (41, 97, 1.5, 8)):
        img = torch.from_numpy(synth.pink_noise([21, H, W], H, W)).cuda()
        out = torch.empty((M, M, H, W), dtype=torch.complex64, device="cuda")
        rc = fn(ctypes.c_void_p(img.data_ptr()), H, W, W, sigma, M, M, 0, ctypes.c_void_p(out.data_ptr()),
                ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.gabor_bank_last_error().decode()
        with GaborBank(precision="fp32") as gbk:
            ref = gbk.sdft(img, sigma, M)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) <= FP32_TOL


def test_noalloc_rejects_oversized_window():
    import torch
    lib, fn = _noalloc_fn()
    img = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    out = torch.empty((2, 2, 8, 8), dtype=torch.complex64, device="cuda")
    rc = fn(ctypes.c_void_p(img.data_ptr()), 8, 8, 8, 4.0, 66, 66, 0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -4
    assert "64" in lib.gabor_bank_last_error().decode()
