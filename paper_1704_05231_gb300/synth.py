"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds input generation only: none of the filter-bank or SDFT arithmetic.  The
paper measured on USC-SIPI images and on unnamed 1024x1024 and 250x234 images; those are not
available, so 1/f-spectrum noise images (the usual statistical stand-in for natural images)
of the paper's sizes replace them.

All generators use numpy's ``default_rng`` in float64 and return C-contiguous float32 arrays.
"""
from __future__ import annotations

import math

import numpy as np


def uniform01(seed: int, H: int, W: int) -> np.ndarray:
    """Values uniform on [0, 1) from ``default_rng(seed)``, cast to float32."""
    return np.random.default_rng(seed).random((H, W)).astype(np.float32)


def _normalise01(a: np.ndarray) -> np.ndarray:
    lo, hi = float(a.min()), float(a.max())
    if hi <= lo:
        return np.zeros_like(a)
    return (a - lo) / (hi - lo)


def _pink(rng: np.random.Generator, H: int, W: int) -> np.ndarray:
    """Zero-mean Gaussian noise whose amplitude spectrum falls as 1/|f| (power 1/f^2)."""
    white = rng.standard_normal((H, W))
    spec = np.fft.fft2(white)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    spec *= 1.0 / np.maximum(f, 1.0 / max(H, W))
    spec[0, 0] = 0.0
    return np.real(np.fft.ifft2(spec))


def pink_noise(seed, H: int, W: int) -> np.ndarray:
    """1/f-amplitude (1/f^2-power) Gaussian noise normalised to [0, 1], float32.

    ``seed`` is anything ``default_rng`` accepts (an int or a list such as [1, i]).
    """
    return _normalise01(_pink(np.random.default_rng(seed), H, W)).astype(np.float32)


def paper_like(seed: int, H: int, W: int, n_sinusoids: int = 8) -> np.ndarray:
    """1/f^2 noise plus oriented sinusoids, normalised to [0, 1] (float32).

    Sinusoid j has frequency pi * 2**-U(1,5) rad/px, orientation U(0, pi), phase U(0, 2 pi)
    and amplitude U(0.5, 1) times the noise standard deviation.
    """
    rng = np.random.default_rng(seed)
    base = _pink(rng, H, W)
    sd = float(base.std())
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(n_sinusoids):
        w = math.pi * 2.0 ** (-rng.uniform(1.0, 5.0))
        th = rng.uniform(0.0, math.pi)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        amp = rng.uniform(0.5, 1.0) * sd
        base += amp * np.cos(w * (xx * math.cos(th) + yy * math.sin(th)) + ph)
    return _normalise01(base).astype(np.float32)


def impulse(H: int, W: int, x0: int, y0: int) -> np.ndarray:
    """A unit impulse at (x0, y0), float32."""
    a = np.zeros((H, W), dtype=np.float32)
    a[y0, x0] = 1.0
    return a


def batch_shapes(seed: int = 1, n: int = 64, lo: int = 128, hi: int = 2048):
    """(H, W) pairs drawn uniformly on [lo, hi] (the uneven-batch workload)."""
    rng = np.random.default_rng(seed)
    hw = rng.integers(lo, hi + 1, size=(n, 2))
    return [(int(h), int(w)) for h, w in hw]


def batch_images(seed: int = 1, n: int = 64, lo: int = 128, hi: int = 2048):
    """The uneven batch: image i is 1/f noise from default_rng([seed, i])."""
    return [pink_noise([seed, i], h, w) for i, (h, w) in enumerate(batch_shapes(seed, n, lo, hi))]


def octave_bank(n_theta: int, n_freq: int, sigma_times_omega: float = math.pi):
    """theta_k = k pi / N, omega_s = pi / 2**(s+1), sigma_s = sigma_times_omega / omega_s."""
    thetas = [k * math.pi / n_theta for k in range(n_theta)]
    omegas = [math.pi / 2 ** (s + 1) for s in range(n_freq)]
    sigmas = [sigma_times_omega / w for w in omegas]
    return thetas, omegas, sigmas


def request_stream(seed: int = 2, n: int = 2200, rate_hz: float = 100.0,
                   lo: int = 256, hi: int = 4096, p_sdft: float = 0.1):
    """A served-request stream: Poisson arrival times and per-request shapes and banks.

    Each request is a dict with ``t`` (arrival, s), ``H``, ``W`` (log-uniform on [lo, hi]),
    ``kind`` ('bank' or 'sdft'), and for banks ``thetas``, ``omegas``, ``sigmas``
    (N ~ U{4..8} orientations, S ~ U{2..5} octave frequencies, sigma = pi/omega); for SDFT
    requests ``M`` = 16 and ``sigma`` = 4.  ``seed`` seeds the image of the request.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    reqs = []
    for i in range(n):
        H = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        W = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        if rng.random() < p_sdft:
            reqs.append(dict(t=float(t[i]), H=H, W=W, kind="sdft", M=16, sigma=4.0,
                             seed=[seed, i]))
        else:
            N = int(rng.integers(4, 9))
            S = int(rng.integers(2, 6))
            th, om, sg = octave_bank(N, S)
            reqs.append(dict(t=float(t[i]), H=H, W=W, kind="bank", thetas=th, omegas=om,
                             sigmas=sg, seed=[seed, i]))
    return reqs


def pink_noise_device(seed: int, H: int, W: int, device="cuda"):
    """1/f-amplitude noise normalised to [0, 1] as a float32 CUDA tensor, made on the device.

    The same construction as ``pink_noise`` (white Gaussian noise, spectrum times
    1/max(|f|, 1/max(H, W)), DC removed, min-max normalised) with torch's seeded device
    generator, for inputs too large to synthesise on the host in time (the served stream's
    4096 x 4096 source images).  Values differ from ``pink_noise`` for the same seed.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    white = torch.randn((H, W), generator=g, device=device, dtype=torch.float32)
    spec = torch.fft.rfft2(white)
    fy = torch.fft.fftfreq(H, device=device)[:, None]
    fx = torch.fft.rfftfreq(W, device=device)[None, :]
    f = torch.sqrt(fx * fx + fy * fy)
    spec = spec / torch.clamp(f, min=1.0 / max(H, W))
    spec[0, 0] = 0
    a = torch.fft.irfft2(spec, s=(H, W))
    lo, hi = a.min(), a.max()
    return ((a - lo) / torch.clamp(hi - lo, min=1e-30)).contiguous()
