"""Thin ctypes binding of libgaborbank.so (the C ABI in include/gaborbank.h).

Argument marshalling only: every step of the filter bank and the SDFT runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current CUDA stream.  There is no CPU
fallback: if the library is missing or fails to load, every call raises ``GBError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgaborbank.so")

GB_OK = 0
STATUS = {0: "GB_OK", -1: "GB_ERR_INVALID_ARG", -2: "GB_ERR_OUT_OF_MEMORY", -3: "GB_ERR_CUDA",
          -4: "GB_ERR_UNSUPPORTED", -5: "GB_ERR_BUDGET", -6: "GB_ERR_TIMEOUT"}
STATUS_CODE = {v: k for k, v in STATUS.items()}
PRECISION = {"fp32": 0, "fp16_tc": 1, "bf16_tc": 2}
OPTION = {"reuse": 1, "tile_rows": 2, "segments": 3, "boundary": 4, "layout": 5, "smoother": 6, "sdft_order": 7, "pipeline": 8, "row_pass": 9, "bank_ctas": 10, "sdft_form": 11, "sdft_reuse": 12, "tc_tiles": 13}
SMOOTHER = {"fir": 0, "iir": 1}
BOUNDARY = {"zero": 0, "replicate": 1, "mirror": 2}
LAYOUT = {"planes": 0, "pixels": 1}

# Every entry point the header declares, with its ctypes signature.
_c_int, _c_dbl, _c_i64, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
SIGNATURES = {
    "gabor_bank_create": (_c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_c_dbl), _c_int,
                                   ctypes.POINTER(_c_dbl), ctypes.POINTER(_c_dbl), _c_int,
                                   _c_dbl, _c_int, _c_int, _c_int]),
    "gabor_bank_destroy": (_c_int, [_vp]),
    "gabor_bank_filter": (_c_int, [_vp, _vp, _c_int, _c_int, _c_i64, _vp, _vp]),
    "gabor_bank_filter_host": (_c_int, [_vp, _vp, _c_int, _c_int, _c_i64, _vp, _vp]),
    "gabor_bank_sdft": (_c_int, [_vp, _vp, _c_int, _c_int, _c_i64, _c_dbl, _c_int, _c_int,
                                 _c_int, _vp, _vp]),
    "gabor_bank_filter_batch": (_c_int, [_vp, _c_int, ctypes.POINTER(_vp), ctypes.POINTER(_c_int),
                                         ctypes.POINTER(_c_int), ctypes.POINTER(_c_i64),
                                         ctypes.POINTER(_vp), _vp]),
    "gabor_bank_set_option": (_c_int, [_vp, _c_int, _c_i64]),
    "gabor_bank_set_tiling": (_c_int, [_vp, _c_int, _c_int, _c_int]),
    "gabor_bank_device_status": (_c_int, [_vp, _vp]),
    "gabor_bank_output_elems": (_c_i64, [_vp, _c_int, _c_int]),
    "gabor_bank_last_error": (ctypes.c_char_p, []),
    "gabor_bank_version": (ctypes.c_char_p, []),
    "gabor_sdft_noalloc": (_c_int, [_vp, _c_int, _c_int, _c_i64, _c_dbl, _c_int, _c_int, _c_int, _vp, _vp]),
    "gabor_bank_selftest_wait": (_c_int, [_vp, _c_int, _c_dbl, _vp]),
    "gabor_fp32_fma_probe": (_c_int, [_vp, _c_int, _c_int, _c_int, _vp]),
    "gabor_store_probe": (_c_int, [_vp, ctypes.c_int64, _c_int, _c_int, _c_int, _vp]),
    "gabor_bank_workspace_bytes": (_c_i64, [_vp, _c_int, _c_int]),
    "gabor_bank_set_workspace": (_c_int, [_vp, _vp, _c_i64]),
    "gabor_arena_create": (_c_int, [ctypes.POINTER(_vp), _c_i64]),
    "gabor_arena_wrap": (_c_int, [ctypes.POINTER(_vp), _vp, _c_i64]),
    "gabor_arena_alloc": (_c_int, [_vp, _c_i64, ctypes.POINTER(_vp)]),
    "gabor_arena_free": (_c_int, [_vp, _vp]),
    "gabor_arena_stats": (_c_int, [_vp, ctypes.POINTER(_c_i64), ctypes.POINTER(_c_i64),
                                   ctypes.POINTER(_c_i64)]),
    "gabor_arena_destroy": (_c_int, [_vp]),
}

_lock = threading.Lock()
_lib = None


class GBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH):
    """Load libgaborbank.so and declare its signatures (raises GBError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise GBError(-3, f"{path} is not built (run __graft_entry__.build())")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc):
    if rc != GB_OK:
        raise GBError(rc, _lib.gabor_bank_last_error().decode())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dbl_array(vals):
    arr = (ctypes.c_double * max(1, len(vals)))(*[float(v) for v in vals])
    return arr


class GaborBank:
    """A filter-bank plan on the current CUDA device (Algorithm 1's Sigma, Omega, Theta).

    thetas: orientations (rad); omegas, sigmas: one (omega, sigma) per frequency.
    precision: 'fp32', 'fp16_tc' or 'bf16_tc'.  An empty bank (no thetas / omegas) makes an
    SDFT-only handle.  boundary: 'zero', 'replicate' or 'mirror' (image extension); layout:
    'planes' (out[s][k][y][x]) or 'pixels' (out[y][x][s][k]); smoother: 'fir' (truncated
    Gaussian, exact) or 'iir' (recursive Gaussian, FP32 only).
    """

    def __init__(self, thetas=(), omegas=(), sigmas=(), radius_factor=3.0, precision="fp32",
                 max_shape=(0, 0), boundary="zero", layout="planes", smoother="fir"):
        lib = load_library()
        if len(omegas) != len(sigmas):
            raise ValueError("omegas and sigmas must have the same length")
        self.thetas = [float(t) for t in thetas]
        self.omegas = [float(w) for w in omegas]
        self.sigmas = [float(s) for s in sigmas]
        self.precision = precision
        h = ctypes.c_void_p()
        _check(lib.gabor_bank_create(ctypes.byref(h), _dbl_array(self.thetas), len(self.thetas),
                                     _dbl_array(self.omegas), _dbl_array(self.sigmas),
                                     len(self.omegas), float(radius_factor),
                                     PRECISION[precision], int(max_shape[0]), int(max_shape[1])))
        self._h = h
        self._lib = lib
        self.layout = "planes"
        if boundary != "zero":
            self.set_option("boundary", BOUNDARY[boundary])
        if layout != "planes":
            self.set_option("layout", LAYOUT[layout])
            self.layout = layout
        if smoother != "fir":
            self.set_option("smoother", SMOOTHER[smoother])

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            self._lib.gabor_bank_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_option(self, key, value):
        if key == "boundary" and isinstance(value, str):
            value = BOUNDARY[value]
        if key == "layout" and isinstance(value, str):
            value = LAYOUT[value]
        if key == "smoother" and isinstance(value, str):
            value = SMOOTHER[value]
        _check(self._lib.gabor_bank_set_option(self._h, OPTION[key] if isinstance(key, str) else int(key),
                                               int(value)))
        if key in ("layout", OPTION["layout"]):
            self.layout = "pixels" if int(value) == 1 else "planes"

    def set_tiling(self, s, tile_rows, segments):
        """FP32 kernel tile geometry for frequency s (-1: all); 0 means automatic."""
        _check(self._lib.gabor_bank_set_tiling(self._h, int(s), int(tile_rows), int(segments)))

    def device_status(self, stream=None):
        _check(self._lib.gabor_bank_device_status(self._h, _stream_handle(stream)))

    def selftest_wait(self, signal, limit_ms=5.0, stream=None):
        """Run the bounded-wait self-test kernel (see gabor_bank_selftest_wait)."""
        _check(self._lib.gabor_bank_selftest_wait(self._h, int(signal), float(limit_ms), _stream_handle(stream)))

    def workspace_bytes(self, H, W):
        """Device bytes of tensor-core intermediate an H x W image needs (0 for FP32)."""
        return int(self._lib.gabor_bank_workspace_bytes(self._h, int(H), int(W)))

    def set_workspace(self, ptr, nbytes):
        """Use caller-owned device memory (raw pointer) as the intermediate; (0, 0) resets."""
        _check(self._lib.gabor_bank_set_workspace(self._h, ctypes.c_void_p(ptr or None), int(nbytes)))

    # -- shapes
    def out_shape(self, H, W):
        if self.layout == "pixels":
            return (H, W, len(self.omegas), len(self.thetas))
        return (len(self.omegas), len(self.thetas), H, W)

    # -- compute
    @staticmethod
    def _img_args(img):
        import torch
        if not isinstance(img, torch.Tensor) or not img.is_cuda or img.dtype != torch.float32:
            raise TypeError("image must be a float32 CUDA tensor")
        if img.dim() != 2 or img.stride(1) != 1:
            raise ValueError("image must be 2-D with unit column stride")
        H, W = img.shape
        return ctypes.c_void_p(img.data_ptr()), H, W, img.stride(0)

    def filter(self, img, out=None, stream=None):
        """complex64 [n_freq][n_theta][H][W] on img's device (Eq. 1 for every filter)."""
        import torch
        p, H, W, pitch = self._img_args(img)
        if out is None:
            out = torch.empty(self.out_shape(H, W), dtype=torch.complex64, device=img.device)
        elif out.dtype != torch.complex64 or not out.is_contiguous() or tuple(out.shape) != self.out_shape(H, W):
            raise ValueError("out must be a contiguous complex64 tensor of shape " + str(self.out_shape(H, W)))
        _check(self._lib.gabor_bank_filter(self._h, p, H, W, pitch, ctypes.c_void_p(out.data_ptr()),
                                           _stream_handle(stream)))
        return out

    def filter_host(self, img, out=None, stream=None):
        """The bank on host buffers (numpy float32 in, numpy complex64 out), synchronous."""
        img = np.ascontiguousarray(img, dtype=np.float32)
        H, W = img.shape
        if out is None:
            out = np.empty(self.out_shape(H, W), dtype=np.complex64)
        _check(self._lib.gabor_bank_filter_host(self._h, ctypes.c_void_p(img.ctypes.data), H, W, W,
                                                ctypes.c_void_p(out.ctypes.data), _stream_handle(stream)))
        return out

    def filter_host_ptr(self, img_ptr, H, W, pitch, out_ptr, stream=None):
        """gabor_bank_filter_host on raw host pointers (e.g. pinned torch tensors)."""
        _check(self._lib.gabor_bank_filter_host(self._h, ctypes.c_void_p(img_ptr), H, W, pitch,
                                                ctypes.c_void_p(out_ptr), _stream_handle(stream)))

    def filter_batch(self, imgs, outs=None, stream=None):
        """The bank for a list of images of any sizes; returns the list of outputs."""
        import torch
        n = len(imgs)
        args = [self._img_args(t) for t in imgs]
        if outs is None:
            outs = [torch.empty(self.out_shape(H, W), dtype=torch.complex64, device=t.device)
                    for t, (_, H, W, _) in zip(imgs, args)]
        ptrs = (ctypes.c_void_p * max(1, n))(*[a[0].value for a in args])
        Hs = (ctypes.c_int * max(1, n))(*[a[1] for a in args])
        Ws = (ctypes.c_int * max(1, n))(*[a[2] for a in args])
        Ps = (ctypes.c_int64 * max(1, n))(*[a[3] for a in args])
        Os = (ctypes.c_void_p * max(1, n))(*[o.data_ptr() for o in outs])
        _check(self._lib.gabor_bank_filter_batch(self._h, n, ptrs, Hs, Ws, Ps, Os, _stream_handle(stream)))
        return outs

    def sdft(self, img, sigma, M, half_spectrum=False, out=None, stream=None):
        """Localized SDFT (Eq. 17): complex64 [My or My/2+1][Mx][H][W].  M: int or (My, Mx)."""
        import torch
        My, Mx = (M, M) if isinstance(M, int) else (int(M[0]), int(M[1]))
        p, H, W, pitch = self._img_args(img)
        nv = My // 2 + 1 if half_spectrum else My
        shape = (nv, Mx, H, W)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device=img.device)
        elif out.dtype != torch.complex64 or not out.is_contiguous() or tuple(out.shape) != shape:
            raise ValueError("out must be a contiguous complex64 tensor of shape " + str(shape))
        _check(self._lib.gabor_bank_sdft(self._h, p, H, W, pitch, float(sigma), My, Mx,
                                         1 if half_spectrum else 0, ctypes.c_void_p(out.data_ptr()),
                                         _stream_handle(stream)))
        return out


class Arena:
    """Fixed-budget device memory (gabor_arena_*) over one torch-owned buffer.

    alloc(nbytes) returns a byte offset into `buffer` or None when no free range fits (the
    budget is exhausted); view(off, shape, dtype) is a tensor over that range.
    """

    def __init__(self, nbytes, device=None):
        import torch
        lib = load_library()
        self.buffer = torch.empty(int(nbytes), dtype=torch.uint8, device=device or "cuda")
        h = ctypes.c_void_p()
        _check(lib.gabor_arena_wrap(ctypes.byref(h), ctypes.c_void_p(self.buffer.data_ptr()), int(nbytes)))
        self._h = h
        self._lib = lib
        self.base = self.buffer.data_ptr()

    def alloc(self, nbytes):
        p = ctypes.c_void_p()
        rc = self._lib.gabor_arena_alloc(self._h, int(nbytes), ctypes.byref(p))
        if rc == STATUS_CODE["GB_ERR_BUDGET"]:
            return None
        _check(rc)
        return p.value - self.base

    def free(self, off):
        _check(self._lib.gabor_arena_free(self._h, ctypes.c_void_p(self.base + off)))

    def stats(self):
        c, u, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.gabor_arena_stats(self._h, ctypes.byref(c), ctypes.byref(u), ctypes.byref(f)))
        return {"capacity": c.value, "in_use": u.value, "largest_free": f.value}

    def ptr(self, off):
        return self.base + off

    def view(self, off, shape, dtype):
        import torch
        n = 1
        for d in shape:
            n *= int(d)
        nbytes = n * torch.empty((), dtype=dtype).element_size()
        return self.buffer[off:off + nbytes].view(dtype).view(*shape)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gabor_arena_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def store_probe(out, ctas=None, stream=None):
    """Enqueue the library's store-pattern probe on `out` (a contiguous complex64 CUDA tensor of
    shape (nplanes, H, W), W a multiple of 128): the tensor-core SDFT's output stream without
    its arithmetic, `ctas` CTAs of 16 warps (default: one per SM)."""
    import torch
    lib = load_library()
    nplanes, H, W = out.shape
    if ctas is None:
        ctas = torch.cuda.get_device_properties(out.device).multi_processor_count
    _check(lib.gabor_store_probe(ctypes.c_void_p(out.data_ptr()), nplanes, H, W, ctas, _stream_handle(stream)))


def fp32_fma_peak(iters=4096, waves=8, steps=5):
    """Measured FP32 CUDA-core throughput (TFLOP/s) of the library's FMA probe on the current
    device: {"scalar": ..., "packed": ..., "peak": max of the two}."""
    import torch
    lib = load_library()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * waves   # 8 CTAs of 256 threads fill an SM's 64 warps
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = _stream_handle(None)
    res = {}
    for name, packed in (("scalar", 0), ("packed", 1)):
        _check(lib.gabor_fp32_fma_probe(ctypes.c_void_p(out.data_ptr()), blocks, iters, packed, st))
        torch.cuda.synchronize()
        best = None
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _check(lib.gabor_fp32_fma_probe(ctypes.c_void_p(out.data_ptr()), blocks, iters, packed, st))
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        res[name] = blocks * 256 * 32.0 * iters / (best * 1e-3) / 1e12
    res["peak"] = max(res["scalar"], res["packed"])
    return res


def capture_graph(fn, warmup=1):
    """Capture `fn` (library calls on the current stream) into a CUDA graph.

    `fn` runs `warmup` times eagerly on a side stream first, so that the library builds its
    tables and work lists outside the capture; the returned torch.cuda.CUDAGraph replays the
    launches with `.replay()`.
    """
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fn()
    return graph


def version():
    return load_library().gabor_bank_version().decode()
