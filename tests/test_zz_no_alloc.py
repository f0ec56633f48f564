"""The allocation-free SDFT entry point (gabor_sdft_noalloc), called through the C ABI.

Some callers cannot call cudaMalloc: code that runs inside a custom allocator or a memory pool
(which must not re-enter the allocator), or an application whose device-memory budget is fixed
before it starts.  For them the library offers gabor_sdft_noalloc, which keeps its tables in a
fixed device array instead of in memory a handle allocates.  Each case here is compared with
the handle-based gabor_bank_sdft and with the FP64 oracle, and the cases run one after another
so that every call must rewrite the shared table left by the previous one: square and
non-square windows (both orientations), a pitched view (pitch > W) and the half spectrum.
This file is collected last so that a failure here does not hide the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu

# (H, W, sigma, My, Mx, half_spectrum, column offset of a pitched view or None)
CASES = [
    (70, 150, 4.0, 16, 16, 0, None),
    (41, 97, 1.5, 8, 8, 0, None),
    (53, 120, 2.5, 8, 32, 0, None),
    (90, 61, 2.5, 32, 8, 0, None),
    (64, 77, 2.0, 12, 6, 0, 9),       # strided view: pitch 77 + 2 * 9 > W
    (48, 100, 4.0, 16, 16, 1, None),  # v = 0 .. My/2 only
    (37, 45, 1.5, 6, 16, 1, 5),
]


def _noalloc_fn():
    from paper_1704_05231_gb300 import bank
    lib = bank.load_library()
    fn = lib.gabor_sdft_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return lib, fn


def _image(torch, H, W, off, seed):
    """The FP32 image as a device tensor (a strided view of a wider one when off is set)."""
    if off is None:
        host = synth.pink_noise([21, seed, H, W], H, W)
        return host, torch.from_numpy(host).cuda()
    wide = synth.pink_noise([22, seed, H, W], H, W + 2 * off)
    return np.ascontiguousarray(wide[:, off:off + W]), torch.from_numpy(wide).cuda()[:, off:off + W]


def test_noalloc_matches_handle_path_and_oracle_calls_in_a_row():
    import torch
    from paper_1704_05231_gb300 import GaborBank
    lib, fn = _noalloc_fn()
    stream = torch.cuda.current_stream()
    for i, (H, W, sigma, My, Mx, half, off) in enumerate(CASES):
        host, img = _image(torch, H, W, off, i)
        pitch = img.stride(0)
        assert (pitch > W) == (off is not None)
        nv = My // 2 + 1 if half else My
        out = torch.full((nv, Mx, H, W), float("nan"), dtype=torch.complex64, device="cuda")
        rc = fn(ctypes.c_void_p(img.data_ptr()), H, W, pitch, sigma, My, Mx, half,
                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.gabor_bank_last_error().decode()
        with GaborBank(precision="fp32") as gbk:
            ref = gbk.sdft(img, sigma, (My, Mx), half_spectrum=bool(half))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref.cpu().numpy()) <= FP32_TOL, (H, W, My, Mx, half, off)
        exact = oracle.sdft(host, sigma, My, Mx)[:nv]
        e = rel_err(got, exact)
        print("noalloc", (H, W, My, Mx, half, off), "rel err vs oracle", e)
        assert e <= FP32_TOL, (H, W, My, Mx, half, off)


def test_noalloc_rejects_oversized_window():
    import torch
    lib, fn = _noalloc_fn()
    img = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    out = torch.empty((2, 2, 8, 8), dtype=torch.complex64, device="cuda")
    rc = fn(ctypes.c_void_p(img.data_ptr()), 8, 8, 8, 4.0, 66, 66, 0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -4
    assert "64" in lib.gabor_bank_last_error().decode()
    rc = fn(ctypes.c_void_p(img.data_ptr()), 8, 8, 8, 4.0, 16, 80, 0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -4
