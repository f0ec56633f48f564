"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv 1704.05231 it follows.  The pins are chosen so that a
plausible slip anywhere in the oracle (a wrong phase sign, a transposed index, a dropped
normalisation, a mishandled border, a reversed window) fails at least one of them:

* impulse response (the kernel of Eq. 1-2 itself, at every offset),
* closed form for complex-exponential images (the truncated and the continuous Gaussian
  spectrum, Poisson summation),
* exact symmetries between orientations (conjugation, mirror, transpose; Eq. 13),
* brute force on 16x16 inputs: a dense operator matrix and numpy's FFT convolution,
* the constant image (border handling with zero padding),
* the separable form of Eq. 3-4 and the decomposition of Eq. 5-6,
* for the localized SDFT (Eq. 17): numpy's fft2 of the Gaussian-weighted patch, the box
  window limit, conjugate symmetry, and the link to the Gabor oracle.
"""
import math

import numpy as np
import pytest

import oracle


def S(d, sigma):
    d = np.asarray(d, dtype=np.float64)
    return np.exp(-d * d / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma)


def kernel2d(omega, theta, sigma, R):
    """K[dy+R, dx+R] = exp(i omega (dx cos + dy sin)) S(dx) S(dy) (Eq. 1-2)."""
    d = np.arange(-R, R + 1)
    dx = d[None, :]
    dy = d[:, None]
    return np.exp(1j * omega * (dx * math.cos(theta) + dy * math.sin(theta))) * S(dx, sigma) * S(dy, sigma)


RNG = np.random.default_rng(1234)


# ---------------------------------------------------------------- Gaussian (Sec. II)

def test_gauss_normalisation_and_radius():
    # S_sigma(0) = 1/(sqrt(2 pi) sigma): the continuous density, unnormalised after truncation.
    for sg in (0.7, 2.0, 4.0, 16.0):
        assert oracle.gauss(0, sg) == pytest.approx(1 / (math.sqrt(2 * math.pi) * sg), rel=1e-15)
        R = oracle.radius(sg)
        tot = sum(oracle.gauss(d, sg) for d in range(-R, R + 1))
        # midpoint rule of the density over [-R-1/2, R+1/2]
        assert tot == pytest.approx(math.erf((R + 0.5) / (sg * math.sqrt(2))), abs=2e-3 if sg < 1 else 5e-4)
    # "radius 3 sigma = 12" for sigma = 4; sigma = pi/omega gives 2, 4, 8, 16.
    assert oracle.radius(4.0) == 12
    assert [oracle.radius(math.pi / (math.pi / 2 ** s)) for s in (1, 2, 3, 4)] == [6, 12, 24, 48]
    assert oracle.radius(1.0 / 3.0) == 1


# ---------------------------------------------------------------- Eq. 1-2, impulse

@pytest.mark.parametrize("omega,theta,sigma", [(math.pi / 4, 0.0, 2.0), (math.pi / 8, 3 * math.pi / 4, 3.0),
                                               (1.1, 0.4, 1.5), (math.pi / 2, math.pi / 2, 2.0)])
def test_impulse_response_is_the_kernel(omega, theta, sigma):
    R = oracle.radius(sigma)
    H, W = 2 * R + 9, 2 * R + 12
    x0, y0 = R + 5, R + 3
    f = np.zeros((H, W))
    f[y0, x0] = 1.0
    F = oracle.gabor_filter(f, omega, theta, sigma)
    exp = np.zeros((H, W), complex)
    exp[y0 - R:y0 + R + 1, x0 - R:x0 + R + 1] = kernel2d(omega, theta, sigma, R)
    assert np.max(np.abs(F - exp)) < 1e-15


# ---------------------------------------------------------------- closed form

def ghat_trunc(nu, sigma, R):
    d = np.arange(1, R + 1)
    return S(0, sigma) + 2 * np.sum(S(d, sigma) * np.cos(nu * d))


@pytest.mark.parametrize("a,b,omega,theta,sigma", [
    (0.7, -0.3, 0.8, 0.2, 2.0), (math.pi / 4, 0.0, math.pi / 4, 0.0, 4.0),
    (0.1, 0.5, math.pi / 8, math.pi / 3, 3.0), (-1.2, 0.9, 1.5, 2.3, 1.2)])
def test_complex_exponential_closed_form(a, b, omega, theta, sigma):
    R = oracle.radius(sigma)
    H, W = 2 * R + 7, 2 * R + 10
    yy, xx = np.mgrid[0:H, 0:W]
    f = np.exp(1j * (a * xx + b * yy))
    F = oracle.gabor_filter(f, omega, theta, sigma)
    inner = (slice(R, H - R), slice(R, W - R))
    gx = ghat_trunc(a - omega * math.cos(theta), sigma, R)
    gy = ghat_trunc(b - omega * math.sin(theta), sigma, R)
    assert np.max(np.abs(F[inner] - f[inner] * gx * gy)) < 1e-13
    # Against the continuous Gaussian spectrum: truncation tail plus aliasing only.
    nux, nuy = a - omega * math.cos(theta), b - omega * math.sin(theta)
    cont = math.exp(-sigma ** 2 * nux ** 2 / 2) * math.exp(-sigma ** 2 * nuy ** 2 / 2)
    tail = math.erfc((R + 0.5) / (sigma * math.sqrt(2)))
    alias = 2 * math.exp(-sigma ** 2 * (2 * math.pi - abs(nux)) ** 2 / 2) + 2 * math.exp(-sigma ** 2 * (2 * math.pi - abs(nuy)) ** 2 / 2)
    assert np.max(np.abs(F[inner] / f[inner] - cont)) <= 2 * tail + alias + 1e-12


def test_real_cosine_image():
    a, b, omega, theta, sigma = 0.6, 0.25, 0.7, 0.35, 2.0
    R = oracle.radius(sigma)
    H, W = 2 * R + 6, 2 * R + 6
    yy, xx = np.mgrid[0:H, 0:W]
    f = np.cos(a * xx + b * yy)
    F = oracle.gabor_filter(f, omega, theta, sigma)
    e = np.exp(1j * (a * xx + b * yy))
    c, s = math.cos(theta), math.sin(theta)
    exp = 0.5 * (e * ghat_trunc(a - omega * c, sigma, R) * ghat_trunc(b - omega * s, sigma, R)
                 + np.conj(e) * ghat_trunc(-a - omega * c, sigma, R) * ghat_trunc(-b - omega * s, sigma, R))
    inner = (slice(R, H - R), slice(R, W - R))
    assert np.max(np.abs(F[inner] - exp[inner])) < 1e-13


# ---------------------------------------------------------------- symmetries

def test_orientation_symmetries():
    H, W = 19, 23
    f = RNG.random((H, W))
    omega, sigma = 0.9, 1.7
    for theta in (0.0, 0.3, 1.1, math.pi / 2):
        F = oracle.gabor_filter(f, omega, theta, sigma)
        scale = np.max(np.abs(F))
        # theta + pi gives the complex conjugate for a real image.
        assert np.max(np.abs(oracle.gabor_filter(f, omega, theta + math.pi, sigma) - np.conj(F))) < 1e-13 * scale
        # pi - theta equals theta on the image mirrored in x, read back mirrored.
        Fm = oracle.gabor_filter(f[:, ::-1], omega, theta, sigma)[:, ::-1]
        assert np.max(np.abs(oracle.gabor_filter(f, omega, math.pi - theta, sigma) - Fm)) < 1e-13 * scale
        # pi/2 - theta equals theta on the transposed image, read back transposed.
        Ft = oracle.gabor_filter(f.T, omega, theta, sigma).T
        assert np.max(np.abs(oracle.gabor_filter(f, omega, math.pi / 2 - theta, sigma) - Ft)) < 1e-13 * scale


def test_horizontal_pass_conjugate_pair_eq13():
    H, W = 12, 31
    f = RNG.random((H, W))
    omega, sigma = 1.3, 2.2
    for theta in (0.2, 0.9, 1.4):
        J = oracle.gabor_rows(f, omega, theta, sigma)
        Jm = oracle.gabor_rows(f, omega, math.pi - theta, sigma)
        assert np.max(np.abs(Jm - np.conj(J))) < 1e-14


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("H,W,sigma", [(16, 16, 1.5), (16, 16, 8.0), (12, 20, 2.5), (16, 9, 4.0)])
def test_bruteforce_dense_operator_and_fft(H, W, sigma):
    f = RNG.random((H, W))
    omega, theta = 1.0, 0.6
    R = oracle.radius(sigma)
    K = kernel2d(omega, theta, sigma, R)
    F = oracle.gabor_filter(f, omega, theta, sigma)
    # Dense operator: A[(y,x),(l,k)] = K(x-k, y-l) for |x-k|,|y-l| <= R.
    A = np.zeros((H * W, H * W), complex)
    for y in range(H):
        for x in range(W):
            for l in range(H):
                for k in range(W):
                    dx, dy = x - k, y - l
                    if abs(dx) <= R and abs(dy) <= R:
                        A[y * W + x, l * W + k] = K[dy + R, dx + R]
    assert np.max(np.abs((A @ f.reshape(-1)).reshape(H, W) - F)) < 1e-14
    # numpy FFT linear convolution with zero padding, cropped to 'same'.
    PH, PW = H + 2 * R, W + 2 * R
    full = np.fft.ifft2(np.fft.fft2(f, (PH, PW)) * np.fft.fft2(K, (PH, PW)))
    assert np.max(np.abs(full[R:R + H, R:R + W] - F)) < 1e-12


def test_constant_image_border_closed_form():
    H, W = 21, 34
    omega, theta, sigma = 0.75, 1.0, 3.0
    R = oracle.radius(sigma)
    F = oracle.gabor_filter(np.ones((H, W)), omega, theta, sigma)
    c, s = math.cos(theta), math.sin(theta)
    x = np.arange(W)
    y = np.arange(H)
    A = np.array([sum(np.exp(1j * omega * c * (xi - k)) * S(xi - k, sigma)
                      for k in range(W) if abs(xi - k) <= R) for xi in x])
    B = np.array([sum(np.exp(1j * omega * s * (yi - l)) * S(yi - l, sigma)
                      for l in range(H) if abs(yi - l) <= R) for yi in y])
    assert np.max(np.abs(F - B[:, None] * A[None, :])) < 1e-14


def test_linearity():
    H, W = 14, 17
    f, g = RNG.random((H, W)), RNG.random((H, W))
    args = (0.8, 0.5, 2.0)
    lhs = oracle.gabor_filter(2.5 * f - 0.75 * g, *args)
    rhs = 2.5 * oracle.gabor_filter(f, *args) - 0.75 * oracle.gabor_filter(g, *args)
    assert np.max(np.abs(lhs - rhs)) < 1e-13


# ---------------------------------------------------------------- Eq. 3-6

def test_separable_passes_equal_direct_sum():
    H, W = 18, 25
    f = RNG.random((H, W))
    omega, sigma = math.pi / 4, 2.0
    for theta in (0.0, math.pi / 4, math.pi / 2, 2.5):
        J = oracle.gabor_rows(f, omega, theta, sigma)
        F = oracle.gabor_cols(J, omega, theta, sigma)
        assert np.max(np.abs(F - oracle.gabor_filter(f, omega, theta, sigma))) < 1e-14


def test_row_pass_matches_demodulation_form_eq5_6():
    # Eq. 5-6 written out with numpy: demodulate, smooth with S, remodulate.
    H, W = 5, 40
    f = RNG.random((H, W))
    omega, theta, sigma = 0.9, 0.7, 2.5
    R = oracle.radius(sigma)
    wc = omega * math.cos(theta)
    k = np.arange(W)
    fc, fs = f * np.cos(wc * k), f * np.sin(wc * k)
    taps = S(np.arange(-R, R + 1), sigma)
    A = np.array([np.convolve(r, taps, mode="full")[R:R + W] for r in fc])
    B = np.array([np.convolve(r, taps, mode="full")[R:R + W] for r in fs])
    re = np.cos(wc * k) * A + np.sin(wc * k) * B
    im = -np.cos(wc * k) * B + np.sin(wc * k) * A
    J = oracle.gabor_rows(f, omega, theta, sigma)
    assert np.max(np.abs(J - (re + 1j * im))) < 1e-15


# ---------------------------------------------------------------- localized SDFT (Eq. 17-18)

def window_weights(sigma, My, Mx):
    a = np.arange(Mx)
    b = np.arange(My)
    return S(b - My // 2, sigma)[:, None] * S(a - Mx // 2, sigma)[None, :]


@pytest.mark.parametrize("H,W,My,Mx,sigma", [(13, 17, 8, 8, 1.3), (16, 16, 16, 16, 4.0),
                                             (11, 15, 4, 6, 1.0), (9, 20, 6, 4, 2.0)])
def test_sdft_equals_fft2_of_weighted_patch(H, W, My, Mx, sigma):
    f = RNG.random((H, W))
    F = oracle.sdft(f, sigma, My, Mx)
    pad = np.zeros((H + 2 * My, W + 2 * Mx))
    pad[My:My + H, Mx:Mx + W] = f
    w = window_weights(sigma, My, Mx)
    for y in range(H):
        for x in range(W):
            xh, yh = x - Mx // 2, y - My // 2
            patch = pad[My + yh:My + yh + My, Mx + xh:Mx + xh + Mx]
            ref = np.fft.fft2(patch * w)  # ref[v, u]
            assert np.max(np.abs(F[:, :, y, x] - ref)) < 1e-14


def test_sdft_symmetries_and_limits():
    H, W, M, sigma = 12, 14, 8, 1.5
    f = RNG.random((H, W))
    F = oracle.sdft(f, sigma, M)
    for v in range(M):
        for u in range(M):
            assert np.max(np.abs(F[(M - v) % M, (M - u) % M] - np.conj(F[v, u]))) < 1e-14
    # DC bin: the Gaussian-weighted local sum.
    w = window_weights(sigma, M, M)
    pad = np.pad(f, M)
    dc = np.array([[np.sum(pad[M + y - M // 2:M + y + M // 2, M + x - M // 2:M + x + M // 2] * w)
                    for x in range(W)] for y in range(H)])
    assert np.max(np.abs(F[0, 0] - dc)) < 1e-14
    # sigma -> infinity: the plain box-window DFT times S(0)^2.
    big = 1e6
    Fb = oracle.sdft(f, big, M)
    s0 = 1 / (2 * math.pi * big * big)
    for (y, x) in ((0, 0), (5, 7), (H - 1, W - 1)):
        patch = pad[M + y - M // 2:M + y + M // 2, M + x - M // 2:M + x + M // 2]
        assert np.max(np.abs(Fb[:, :, y, x] / s0 - np.fft.fft2(patch))) < 1e-9


def test_sdft_is_a_gabor_filter_on_the_window():
    # F_{u,v} = (-1)^{u+v} Gabor(omega0 (u, v)) over dx, dy in [-M/2+1, M/2].
    H, W, M, sigma = 10, 13, 8, 1.7
    f = RNG.random((H, W))
    F = oracle.sdft(f, sigma, M)
    w0 = 2 * math.pi / M
    sup = ((-M // 2 + 1, M // 2), (-M // 2 + 1, M // 2))
    for (u, v) in ((0, 0), (1, 0), (0, 3), (2, 5), (7, 1), (4, 4)):
        omega = w0 * math.hypot(u, v)
        theta = math.atan2(v, u)
        G = oracle.gabor_filter(f, omega, theta, sigma, support=sup)
        assert np.max(np.abs(F[v, u] - (-1) ** (u + v) * G)) < 1e-13


def test_points_subset_matches_full():
    H, W = 15, 18
    f = RNG.random((H, W))
    xs = np.array([0, 3, 17, 9])
    ys = np.array([0, 14, 7, 2])
    F = oracle.gabor_filter(f, 0.9, 0.3, 1.5)
    Fp = oracle.gabor_filter(f, 0.9, 0.3, 1.5, points=(xs, ys))
    assert np.array_equal(Fp, F[ys, xs])
    D = oracle.sdft(f, 1.5, 8)
    Dp = oracle.sdft(f, 1.5, 8, points=(xs, ys))
    assert np.array_equal(Dp, D[:, :, ys, xs])


# ---------------------------------------------------------------- boundary modes
# The boundary rule is the image extension; with it the filter is the zero-padded filter of
# the explicitly extended image (numpy.pad: 'edge' = replicate, 'symmetric' = mirror about the
# pixel edges), cropped.  Padding wider than the image (R > W) checks the periodic mirror.
_PAD = {"replicate": "edge", "mirror": "symmetric"}


@pytest.mark.parametrize("boundary", ["replicate", "mirror"])
@pytest.mark.parametrize("H,W,sigma", [(12, 17, 1.5), (5, 3, 2.5)])
def test_boundary_equals_zero_padded_extended_image(boundary, H, W, sigma):
    rng = np.random.default_rng(31)
    img = rng.random((H, W))
    R = oracle.radius(sigma)
    ext = np.pad(img, R, mode=_PAD[boundary])
    for theta, omega in [(0.3, 0.9), (2.0, 0.4)]:
        got = oracle.gabor_filter(img, omega, theta, sigma, boundary=boundary)
        ref = oracle.gabor_filter(ext, omega, theta, sigma)[R:R + H, R:R + W]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("boundary", ["replicate", "mirror"])
def test_boundary_constant_image_is_the_interior_closed_form(boundary):
    # An extended constant image is constant everywhere, so every pixel (border included)
    # sees the same sum: F = c * Ghat_R(-w cos t) Ghat_R(-w sin t).
    c, omega, theta, sigma = 0.7, 0.8, 0.45, 2.0
    R = oracle.radius(sigma)
    d = np.arange(-R, R + 1)
    g = np.array([oracle.gauss(k, sigma) for k in d])
    gx = np.sum(g * np.exp(1j * omega * np.cos(theta) * d))
    gy = np.sum(g * np.exp(1j * omega * np.sin(theta) * d))
    got = oracle.gabor_filter(np.full((9, 11), c), omega, theta, sigma, boundary=boundary)
    assert np.max(np.abs(got - c * gx * gy)) <= 1e-13


@pytest.mark.parametrize("boundary", ["replicate", "mirror"])
def test_sdft_boundary_equals_zero_padded_extended_image(boundary):
    rng = np.random.default_rng(32)
    img = rng.random((10, 13))
    M = 8
    ext = np.pad(img, M, mode=_PAD[boundary])
    got = oracle.sdft(img, 2.0, M, boundary=boundary)
    ref = oracle.sdft(ext, 2.0, M)[:, :, M:M + 10, M:M + 13]
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


# ---------------------------------------------------------------- recursive (IIR) variant
# The Young-van Vliet recursion is a linear, shift-invariant, zero-phase smoother with unit
# DC gain that approximates S_sigma; the IIR Gabor variant is Algorithm 1 with it.

@pytest.mark.parametrize("sigma", [1.0, 2.0, 4.0, 8.0, 16.0, 32.0])
def test_iir_smoother_gain_phase_and_shape(sigma):
    n = 8 * int(12 * sigma) + 64
    c = n // 2
    x = np.zeros(n)
    x[c] = 1.0
    h = oracle.iir_smooth(x, sigma)
    d = np.arange(n) - c
    g = np.exp(-d ** 2 / (2 * sigma ** 2)) / (math.sqrt(2 * math.pi) * sigma)
    assert abs(h.sum() - 1.0) <= 1e-10                          # unit DC gain
    k = min(200, c - 1)
    assert np.max(np.abs(h[c + 1:c + k] - h[c - 1:c - k:-1])) <= 1e-13   # zero phase
    # the core follows S_sigma (peak height 1 / (sqrt(2 pi) sigma) within 6%); the recursion's
    # exponential tails are heavier than the Gaussian's, so no second-moment match is expected
    assert abs(h[c] / g[c] - 1.0) <= 0.06
    assert np.max(np.abs(h - g)) <= (0.1 if sigma < 4 else 0.04) * g.max()
    assert np.allclose(oracle.iir_smooth(np.ones(4 * n), sigma)[n:3 * n], 1.0, atol=1e-10)


def test_iir_gabor_equals_direct_sum_with_the_recursive_kernel():
    # Linearity and shift invariance: the decomposition (Eq. 5-10) with the recursive smoother
    # equals the direct 2-D sum of Eq. 1 whose kernel uses the smoother's impulse response h.
    rng = np.random.default_rng(41)
    H, W, sigma, omega, theta = 14, 19, 2.0, 0.9, 0.7
    img = rng.random((H, W))
    P = oracle.iir_pad(sigma)
    n = 2 * P + 1
    imp = np.zeros(4 * n)
    imp[2 * n] = 1.0
    h = oracle.iir_smooth(imp, sigma)[2 * n - P:2 * n + P + 1]      # h(d), d = -P .. P
    d = np.arange(-P, P + 1)
    kx = h * np.exp(1j * omega * math.cos(theta) * d)
    ky = h * np.exp(1j * omega * math.sin(theta) * d)
    ref = np.zeros((H, W), dtype=np.complex128)
    for y in range(H):
        for x in range(W):
            ks = x - d            # k = x - dx
            ls = y - d
            vx = (ks >= 0) & (ks < W)
            vy = (ls >= 0) & (ls < H)
            ref[y, x] = np.sum(ky[vy][:, None] * kx[vx][None, :] * img[np.ix_(ls[vy], ks[vx])])
    got = oracle.iir_gabor_filter(img, omega, theta, sigma)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_iir_gabor_symmetries_and_approach_to_fir():
    from paper_1704_05231_gb300 import synth
    img = synth.pink_noise(3, 40, 52)
    a = oracle.iir_gabor_filter(img, 0.8, 0.4, 3.0)
    assert np.max(np.abs(oracle.iir_gabor_filter(img, 0.8, 0.4 + math.pi, 3.0) - np.conj(a))) <= 1e-13
    m = oracle.iir_gabor_filter(np.ascontiguousarray(img[:, ::-1]), 0.8, 0.4, 3.0)
    c = oracle.iir_gabor_filter(img, 0.8, math.pi - 0.4, 3.0)
    assert np.max(np.abs(c - m[:, ::-1])) <= 1e-13 * np.max(np.abs(c))
    # the recursive Gaussian approaches S_sigma as sigma grows: SER rises (imaginary parts)
    sers = [oracle.ser_db(oracle.iir_gabor_filter(img, math.pi / (2 * s), 0.5, s),
                          oracle.gabor_filter(img, math.pi / (2 * s), 0.5, s))[1] for s in (2.0, 4.0, 8.0)]
    assert sers[0] > 12 and sers[0] < sers[1] < sers[2]


# Young and van Vliet (1995) give their third-order recursive Gaussian in two forms: the decimal
# polynomials in q of b0 .. b3 that the oracle evaluates, and the poles m0, m1 +- i m2 of the
# continuous filter it was derived from, b0 ~ (m0 + q)(m1^2 + m2^2 + 2 m1 q + q^2),
# b1 ~ q (2 m0 m1 + m1^2 + m2^2 + (2 m0 + 4 m1) q + 3 q^2), b2 ~ -q^2 (m0 + 2 m1 + 3 q),
# b3 ~ q^3 (one common factor).  The recursion's ratios b_i / b0 must agree in both forms to the
# precision of the printed decimals (about 5e-6): a slipped or dropped digit in any of the
# oracle's eight polynomial constants moves them by 1e-4 or more.
_YVV_POLES = (1.16680, 1.10783, 1.40586)


def _yvv_pole_ratios(q):
    m0, m1, m2 = _YVV_POLES
    b0 = (m0 + q) * (m1 ** 2 + m2 ** 2 + 2 * m1 * q + q * q)
    b1 = q * (2 * m0 * m1 + m1 ** 2 + m2 ** 2 + (2 * m0 + 4 * m1) * q + 3 * q * q)
    b2 = -q * q * (m0 + 2 * m1 + 3 * q)
    return b1 / b0, b2 / b0, q ** 3 / b0


@pytest.mark.parametrize("sigma", [0.5, 0.7, 1.0, 2.0, 2.49, 2.5, 4.0, 16.0, 64.0, 150.0])
def test_iir_coefficients_match_the_pole_form(sigma):
    from scipy.optimize import brentq
    B, c1, c2, c3 = oracle.iir_coeffs(sigma)
    # the q at which the pole form has the oracle's b3 / b0 (monotonic in q)
    q = brentq(lambda t: _yvv_pole_ratios(t)[2] - c3, 1e-6, 1e4, xtol=1e-15)
    p1, p2, p3 = _yvv_pole_ratios(q)
    assert abs(c1 / p1 - 1) <= 2e-5 and abs(c2 / p2 - 1) <= 2e-5
    assert abs(B - (1 - p1 - p2 - p3)) <= 2e-5 * (abs(p1) + abs(p2) + p3)


@pytest.mark.parametrize("sigma", [1.0, 1.5, 2.0, 3.0, 5.0, 10.0, 20.0, 40.0])
def test_iir_smoother_width_fits_sigma(sigma):
    # q(sigma) (two fitted branches) is chosen so that the forward / backward pair approximates
    # the Gaussian of width sigma: the sampled Gaussian closest to the recursion's impulse
    # response (least squares) has a width within 4% of sigma (measured: -1% .. +3.5%), so a
    # slip in the branch constants that changes the width by more than that fails here.
    from scipy.optimize import minimize_scalar
    n = int(30 * sigma) + 200
    x = np.zeros(2 * n + 1)
    x[n] = 1.0
    h = oracle.iir_smooth(x, sigma)
    d = np.arange(-n, n + 1)

    def misfit(s):
        return float(np.sum((h - np.exp(-d * d / (2 * s * s)) / (math.sqrt(2 * math.pi) * s)) ** 2))

    best = minimize_scalar(misfit, bounds=(0.3 * sigma, 2 * sigma), method="bounded", options={"xatol": 1e-8}).x
    assert abs(best / sigma - 1) <= 0.04
