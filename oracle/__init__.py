"""Plain FP64 CPU oracle for the Gabor filter bank and the localized sliding DFT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.  The
product path (``paper_1704_05231_gb300``) never imports it, and this module imports nothing
from the product.

The arithmetic lives in ``gabor_oracle.c`` (direct sums of Eq. 1, Eq. 3, Eq. 4 and Eq. 17 of
arXiv 1704.05231, in double precision); this file only compiles it with gcc, loads it with
ctypes and marshals numpy arrays.  Inputs are converted to float64 exactly, so the oracle sees
the same FP32 image the GPU sees.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gabor_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile gabor_oracle.c into oracle/_oracle.so (gcc, OpenMP, no fp contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_gauss.restype = ctypes.c_double
            lib.oracle_gauss.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_radius.restype = ctypes.c_int
            lib.oracle_radius.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_gabor_direct.restype = ctypes.c_int
            lib.oracle_gabor_direct.argtypes = [
                _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                _ip, _ip, ctypes.c_long, _dp, ctypes.c_int]
            lib.oracle_gabor_rows.restype = ctypes.c_int
            lib.oracle_gabor_rows.argtypes = [
                _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int]
            lib.oracle_gabor_cols.restype = ctypes.c_int
            lib.oracle_gabor_cols.argtypes = [
                _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int]
            lib.oracle_sdft_direct.restype = ctypes.c_int
            lib.oracle_sdft_direct.argtypes = [
                _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                _ip, _ip, ctypes.c_long, _dp, ctypes.c_int]
            lib.oracle_iir_smooth.restype = ctypes.c_int
            lib.oracle_iir_smooth.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]
            lib.oracle_iir_gabor.restype = ctypes.c_int
            lib.oracle_iir_gabor.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int]
            lib.oracle_iir_coeffs.restype = None
            lib.oracle_iir_coeffs.argtypes = [ctypes.c_double, _dp]
            lib.oracle_iir_pad.restype = ctypes.c_int
            lib.oracle_iir_pad.argtypes = [ctypes.c_double]
            lib.oracle_gabor_direct_b.restype = ctypes.c_int
            lib.oracle_gabor_direct_b.argtypes = lib.oracle_gabor_direct.argtypes + [ctypes.c_int]
            lib.oracle_sdft_direct_b.restype = ctypes.c_int
            lib.oracle_sdft_direct_b.argtypes = lib.oracle_sdft_direct.argtypes + [ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def _split(img):
    img = np.asarray(img)
    if img.ndim != 2:
        raise ValueError("image must be 2-D (H, W)")
    if np.iscomplexobj(img):
        re = np.ascontiguousarray(img.real, dtype=np.float64)
        im = np.ascontiguousarray(img.imag, dtype=np.float64)
    else:
        re = np.ascontiguousarray(img, dtype=np.float64)
        im = None
    return re, im


def _points(points):
    if points is None:
        return None, None, 0
    xs, ys = points
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    if xs.shape != ys.shape or xs.ndim != 1:
        raise ValueError("points must be two equal 1-D arrays (xs, ys)")
    return xs, ys, xs.size


def gauss(d, sigma):
    """S_sigma(d) as the oracle evaluates it."""
    return _load().oracle_gauss(float(d), float(sigma))


def radius(sigma, radius_factor=3.0):
    """R = ceil(radius_factor * sigma) (Gaussian truncation radius)."""
    return _load().oracle_radius(float(sigma), float(radius_factor))


BOUNDARY = {"zero": 0, "replicate": 1, "mirror": 2}


def gabor_filter(img, omega, theta, sigma, radius_factor=3.0, support=None, points=None,
                 threads=0, boundary="zero"):
    """One 2-D complex Gabor output F_{omega,theta,sigma} by the direct sum of Eq. 1.

    support: optional ((dx_lo, dx_hi), (dy_lo, dy_hi)) for dx = x-k, dy = y-l; the default
    is the square |dx|, |dy| <= R.  points: optional (xs, ys) to evaluate a subset.
    boundary: how the image extends beyond its edges: 'zero', 'replicate' (edge pixel
    repeated) or 'mirror' (mirrored about the pixel edges, f(-1) = f(0)).
    Returns complex128 (H, W), or (npts,) with points.
    """
    lib = _load()
    re, im = _split(img)
    H, W = re.shape
    if support is None:
        R = radius(sigma, radius_factor)
        (xl, xh), (yl, yh) = (-R, R), (-R, R)
    else:
        (xl, xh), (yl, yh) = support
    xs, ys, n = _points(points)
    nout = n if xs is not None else H * W
    out = np.empty(2 * nout, dtype=np.float64)
    rc = lib.oracle_gabor_direct_b(_ptr(re), _ptr(im), H, W, float(omega), float(theta),
                                   float(sigma), int(xl), int(xh), int(yl), int(yh),
                                   _ptr(xs, _ip), _ptr(ys, _ip), n, _ptr(out), int(threads),
                                   BOUNDARY[boundary])
    if rc != 0:
        raise ValueError(f"oracle_gabor_direct failed ({rc})")
    out = out.view(np.complex128)
    return out if xs is not None else out.reshape(H, W)


def gabor_bank(img, thetas, omegas, sigmas, radius_factor=3.0, points=None, threads=0,
               boundary="zero"):
    """The bank of Algorithm 1's output: complex128 [n_freq][n_theta][H][W] (or [..][npts])."""
    res = []
    for om, sg in zip(omegas, sigmas):
        res.append([gabor_filter(img, om, th, sg, radius_factor, points=points, threads=threads,
                                 boundary=boundary)
                    for th in thetas])
    return np.array(res)


def gabor_rows(img, omega, theta, sigma, radius_factor=3.0, threads=0):
    """The horizontal 1-D pass J of Eq. 3 (complex128 (H, W))."""
    lib = _load()
    re, im = _split(img)
    H, W = re.shape
    out = np.empty(2 * H * W, dtype=np.float64)
    rc = lib.oracle_gabor_rows(_ptr(re), _ptr(im), H, W, float(omega), float(theta),
                               float(sigma), radius(sigma, radius_factor), _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_gabor_rows failed ({rc})")
    return out.view(np.complex128).reshape(H, W)


def gabor_cols(J, omega, theta, sigma, radius_factor=3.0, threads=0):
    """The vertical 1-D pass of Eq. 4 applied to a complex J (complex128 (H, W))."""
    lib = _load()
    J = np.ascontiguousarray(J, dtype=np.complex128)
    H, W = J.shape
    Jd = J.view(np.float64).reshape(-1)
    out = np.empty(2 * H * W, dtype=np.float64)
    rc = lib.oracle_gabor_cols(_ptr(Jd), H, W, float(omega), float(theta), float(sigma),
                               radius(sigma, radius_factor), _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_gabor_cols failed ({rc})")
    return out.view(np.complex128).reshape(H, W)


def sdft(img, sigma, My, Mx=None, support=None, points=None, threads=0, boundary="zero"):
    """The 2-D localized SDFT of Eq. 17 by direct summation.

    Returns complex128 [My][Mx][H][W] (or [My][Mx][npts]); bin [v][u] has u along x.
    support: optional ((a_lo, a_hi), (b_lo, b_hi)) window offsets from (xhat, yhat); the
    default is the M_x x M_y window [0, Mx) x [0, My).  boundary as in gabor_filter.
    """
    lib = _load()
    Mx = My if Mx is None else Mx
    re, im = _split(img)
    H, W = re.shape
    if support is None:
        (al, ah), (bl, bh) = (0, Mx - 1), (0, My - 1)
    else:
        (al, ah), (bl, bh) = support
    xs, ys, n = _points(points)
    nout = n if xs is not None else H * W
    out = np.empty(2 * nout * Mx * My, dtype=np.float64)
    rc = lib.oracle_sdft_direct_b(_ptr(re), _ptr(im), H, W, float(sigma), int(My), int(Mx),
                                  int(al), int(ah), int(bl), int(bh), _ptr(xs, _ip), _ptr(ys, _ip),
                                  n, _ptr(out), int(threads), BOUNDARY[boundary])
    if rc != 0:
        raise ValueError(f"oracle_sdft_direct failed ({rc})")
    out = out.view(np.complex128)
    return out.reshape(My, Mx, nout) if xs is not None else out.reshape(My, Mx, H, W)


def iir_smooth(x, sigma, boundary="zero"):
    """The Young-van Vliet recursive Gaussian (forward then backward) of a real 1-D signal."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    rc = lib.oracle_iir_smooth(_ptr(x), int(x.size), float(sigma), BOUNDARY[boundary], _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_iir_smooth failed ({rc})")
    return out


def iir_coeffs(sigma):
    """(B, b1/b0, b2/b0, b3/b0) of the recursion w[n] = B x[n] + sum_i (b_i / b0) w[n - i]."""
    out = np.empty(4, dtype=np.float64)
    _load().oracle_iir_coeffs(float(sigma), _ptr(out))
    return tuple(float(v) for v in out)


def iir_pad(sigma):
    """Samples the recursive passes extend each signal by on both sides."""
    return _load().oracle_iir_pad(float(sigma))


def iir_gabor_filter(img, omega, theta, sigma, boundary="zero", threads=0):
    """Algorithm 1 with the recursive Gaussian smoother (complex128 (H, W))."""
    lib = _load()
    f = np.ascontiguousarray(img, dtype=np.float64)
    H, W = f.shape
    out = np.empty(2 * H * W, dtype=np.float64)
    rc = lib.oracle_iir_gabor(_ptr(f), H, W, float(omega), float(theta), float(sigma), BOUNDARY[boundary],
                              _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_iir_gabor failed ({rc})")
    return out.view(np.complex128).reshape(H, W)


def iir_gabor_bank(img, thetas, omegas, sigmas, boundary="zero", threads=0):
    """complex128 [n_freq][n_theta][H][W] with the recursive smoother."""
    return np.array([[iir_gabor_filter(img, om, th, sg, boundary, threads) for th in thetas]
                     for om, sg in zip(omegas, sigmas)])


def ser_db(fast, exact):
    """Signal-to-error ratio of Sec. IV-C for the real and the imaginary parts (dB):
    10 log10(sum part(F)^2 / sum (part(F) - part(F_t))^2), F the fast result, F_t the FIR one."""
    fast = np.asarray(fast)
    exact = np.asarray(exact)
    res = []
    for part in (np.real, np.imag):
        num = float(np.sum(part(fast) ** 2))
        den = float(np.sum((part(fast) - part(exact)) ** 2))
        res.append(10.0 * np.log10(num / den) if den > 0 else float("inf"))
    return tuple(res)


__all__ = ["build", "gauss", "radius", "gabor_filter", "gabor_bank", "gabor_rows",
           "gabor_cols", "sdft", "iir_smooth", "iir_coeffs", "iir_pad", "iir_gabor_filter", "iir_gabor_bank",
           "ser_db"]
