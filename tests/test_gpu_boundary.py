"""Boundary rules (zero, replicate, mirror) and the pixel-major output layout on the GPU.

The bank and the SDFT with a non-zero boundary rule are compared with the FP64 oracle's
direct sums over the extended image, element by element (FP32: 1e-5 * max|out|, tensor
cores: 2e-3 * max|out|); the pixel-major layout must hold exactly the plane-major values.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, TC_TOL, c2_bank, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [(37, 75), (129, 33), (3, 3), (1, 50)]


def _bank(precision, boundary, layout="planes"):
    from paper_1704_05231_gb300 import GaborBank
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6, 2.0]
    om, sg = [math.pi / 3, 0.4], [1.5, 5.0]   # R = 5 and 15: wider than the small images
    return GaborBank(th, om, sg, precision=precision, boundary=boundary, layout=layout), th, om, sg


@pytest.mark.parametrize("precision,tol", [("fp32", FP32_TOL), ("fp16_tc", TC_TOL), ("bf16_tc", TC_TOL)])
@pytest.mark.parametrize("boundary", ["replicate", "mirror"])
@pytest.mark.parametrize("H,W", SHAPES)
def test_bank_boundary_matches_oracle(precision, tol, boundary, H, W):
    import torch
    img = synth.pink_noise([11, H, W], H, W)
    gbk, th, om, sg = _bank(precision, boundary)
    with gbk:
        got = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
    ref = oracle.gabor_bank(img, th, om, sg, boundary=boundary)
    e = rel_err(got, ref)
    print(precision, boundary, H, W, "rel err", e)
    assert e <= tol


@pytest.mark.parametrize("precision,tol", [("fp32", FP32_TOL), ("fp16_tc", TC_TOL), ("bf16_tc", TC_TOL)])
@pytest.mark.parametrize("boundary", ["replicate", "mirror"])
def test_paper_bank_boundary_160x200(precision, tol, boundary):
    import torch
    from paper_1704_05231_gb300 import GaborBank
    img = synth.paper_like(0, 160, 200)
    th, om, sg = c2_bank()
    with GaborBank(th, om, sg, precision=precision, boundary=boundary) as gbk:
        got = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
    rng = np.random.default_rng(5)
    # every border pixel plus a random interior sample
    ys = np.concatenate([np.zeros(200), np.full(200, 159), np.arange(160), np.arange(160), rng.integers(0, 160, 300)])
    xs = np.concatenate([np.arange(200), np.arange(200), np.zeros(160), np.full(160, 199), rng.integers(0, 200, 300)])
    xs, ys = xs.astype(np.int32), ys.astype(np.int32)
    ref = oracle.gabor_bank(img, th, om, sg, points=(xs, ys), boundary=boundary)
    # scale = max|oracle| over the sampled pixels (every border pixel among them)
    assert rel_err(got[:, :, ys, xs], ref) <= tol


@pytest.mark.parametrize("precision,tol", [("fp32", FP32_TOL), ("fp16_tc", TC_TOL), ("bf16_tc", TC_TOL)])
@pytest.mark.parametrize("boundary", ["replicate", "mirror"])
def test_sdft_boundary_matches_oracle(precision, tol, boundary):
    import torch
    from paper_1704_05231_gb300 import GaborBank
    img = synth.pink_noise([12], 23, 41)
    with GaborBank(precision=precision, boundary=boundary) as gbk:
        got = gbk.sdft(torch.from_numpy(img).cuda(), 4.0, 16).cpu().numpy()
    ref = oracle.sdft(img, 4.0, 16, boundary=boundary)
    assert rel_err(got, ref) <= tol


@pytest.mark.parametrize("precision", ["fp32", "fp16_tc"])
@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_pixel_major_layout_is_the_transposed_planes(precision, boundary):
    import torch
    from paper_1704_05231_gb300 import GaborBank
    img = torch.from_numpy(synth.pink_noise([13], 70, 90)).cuda()
    th, om, sg = c2_bank()
    with GaborBank(th, om, sg, precision=precision, boundary=boundary) as a, \
            GaborBank(th, om, sg, precision=precision, boundary=boundary, layout="pixels") as b:
        planes = a.filter(img).cpu().numpy()
        pixels = b.filter(img).cpu().numpy()
        batch = [o.cpu().numpy() for o in b.filter_batch([img, img[:31, :57]])]
        small = a.filter(img[:31, :57]).cpu().numpy()
    assert pixels.shape == (70, 90, 4, 6)
    assert np.array_equal(np.moveaxis(planes, (0, 1), (2, 3)), pixels)
    assert np.array_equal(batch[0], pixels)
    assert np.array_equal(np.moveaxis(small, (0, 1), (2, 3)), batch[1])


def test_batch_with_boundary_equals_single_calls():
    import torch
    from paper_1704_05231_gb300 import GaborBank
    imgs = [torch.from_numpy(synth.pink_noise([14, i], h, w)).cuda()
            for i, (h, w) in enumerate([(40, 70), (128, 96), (33, 257)])]
    th, om, sg = c2_bank()
    with GaborBank(th, om, sg, boundary="replicate") as gbk:
        singles = [gbk.filter(t).cpu().numpy() for t in imgs]
        batch = [o.cpu().numpy() for o in gbk.filter_batch(imgs)]
    for s, b in zip(singles, batch):
        assert np.array_equal(s, b)
