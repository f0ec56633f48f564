"""Shared test helpers: tolerance checks and bank configurations (no method arithmetic)."""
import math

import numpy as np

FP32_TOL = 1e-5   # max|err| <= 1e-5 * max|out| per result tensor (FP32 path)
TC_TOL = 2e-3     # max|err| <= 2e-3 * max|out| per result tensor (tensor-core path)


def rel_err(got, ref):
    """max|got - ref| / max|ref| over a whole result tensor, and the worst plane ratio."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    scale = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(got - ref)))
    return err / scale if scale > 0 else err


def plane_rel_errs(got, ref):
    got = np.asarray(got).reshape(-1, *np.asarray(got).shape[-2:]) if np.asarray(got).ndim > 2 else np.asarray(got)[None]
    ref = np.asarray(ref).reshape(got.shape)
    out = []
    for g, r in zip(got, ref):
        s = float(np.max(np.abs(r)))
        out.append(float(np.max(np.abs(g - r))) / s if s > 0 else 0.0)
    return out


def c1_bank():
    """256x256 uniform image, 4 orientations x 2 frequencies, sigma = 4."""
    thetas = [0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4]
    omegas = [math.pi / 4, math.pi / 8]
    sigmas = [4.0, 4.0]
    return thetas, omegas, sigmas


def c2_bank():
    """6 orientations k pi / 6 x 4 octave frequencies pi/2 .. pi/16, sigma = pi / omega."""
    thetas = [k * math.pi / 6 for k in range(6)]
    omegas = [math.pi / 2, math.pi / 4, math.pi / 8, math.pi / 16]
    sigmas = [math.pi / w for w in omegas]
    return thetas, omegas, sigmas


def sample_points(rng, H, W, n, border=8):
    """n pixels: all four corners, a band along every border, the rest uniform."""
    xs = [0, W - 1, 0, W - 1]
    ys = [0, 0, H - 1, H - 1]
    nb = min(n // 4, 4 * border * 8)
    for _ in range(nb):
        side = rng.integers(4)
        if side == 0:
            xs.append(int(rng.integers(W))); ys.append(int(rng.integers(min(border, H))))
        elif side == 1:
            xs.append(int(rng.integers(W))); ys.append(H - 1 - int(rng.integers(min(border, H))))
        elif side == 2:
            xs.append(int(rng.integers(min(border, W)))); ys.append(int(rng.integers(H)))
        else:
            xs.append(W - 1 - int(rng.integers(min(border, W)))); ys.append(int(rng.integers(H)))
    while len(xs) < n:
        xs.append(int(rng.integers(W)))
        ys.append(int(rng.integers(H)))
    return np.array(xs, dtype=np.int32), np.array(ys, dtype=np.int32)
