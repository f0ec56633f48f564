"""The recursive-Gaussian bank (GB_SMOOTHER_IIR) on the GPU against the FP64 oracle of the
same recursion (Algorithm 1 with the Young-van Vliet smoother), element by element; and its
SER against the exact FIR bank (Sec. IV-C), reported and bounded from below.

Tolerance: the GPU evaluates the recursion in difference form (the state is the last output
and its last two first differences), so a step's rounding error is about half an ulp of the
signal, added to the carried output; the recursion's DC gain is one, so the error persists
along the line and grows as a random walk, about sqrt(n) ulps after n steps.  Two forward /
backward pass pairs (along x, then along y) over extended lines of at most n samples give the
bar max(1e-5 * max|out|, 4 * 2^-24 * sqrt(n) * max|f|) for max|err| per result tensor, for
every sigma.  (The direct form w = c0 x + c1 w1 + c2 w2 + c3 w3, whose feedback sums to
1 - c0 with c0 ~ 1 / sigma^3, measured 3e-3 in FP32 at sigma 32.)
"""
import math

import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, c1_bank, c2_bank, rel_err


def iir_bar(img, sigmas, boundary, ref):
    """The bar above for one result tensor."""
    H, W = img.shape
    P = max(math.ceil(12.0 * s) + 32 for s in sigmas)
    n = max(H, W) + (P if boundary == "zero" else 2 * P)
    return max(FP32_TOL * float(np.max(np.abs(ref))), 4 * 2.0 ** -24 * math.sqrt(n) * float(np.max(np.abs(img))))


def iir_check(got, ref, img, sigmas, boundary="zero"):
    err = float(np.max(np.abs(got - ref)))
    bar = iir_bar(img, sigmas, boundary, ref)
    print("IIR", img.shape, "sigma", max(sigmas), boundary, "max err", err, "bar", bar, "rel err", rel_err(got, ref))
    assert np.all(np.isfinite(got))
    assert err <= bar

pytestmark = pytest.mark.gpu


def _run(img, th, om, sg, **kw):
    import torch
    from paper_1704_05231_gb300 import GaborBank
    with GaborBank(th, om, sg, smoother="iir", **kw) as gbk:
        return gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()


def test_iir_c1_matches_recursive_oracle():
    img = synth.uniform01(0, 256, 256)
    th, om, sg = c1_bank()
    got = _run(img, th, om, sg)
    ref = oracle.iir_gabor_bank(img, th, om, sg)
    print("IIR C1 SER vs FIR", oracle.ser_db(got, oracle.gabor_bank(img, th, om, sg)))
    iir_check(got, ref, img, sg)


@pytest.mark.parametrize("boundary", ["zero", "replicate", "mirror"])
@pytest.mark.parametrize("H,W", [(37, 75), (129, 33), (3, 3), (1, 50)])
def test_iir_ragged_and_boundaries(boundary, H, W):
    img = synth.pink_noise([21, H, W], H, W)
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6]
    om, sg = [math.pi / 3, 0.4], [1.5, 5.0]
    got = _run(img, th, om, sg, boundary=boundary)
    ref = oracle.iir_gabor_bank(img, th, om, sg, boundary=boundary)
    iir_check(got, ref, img, sg, boundary)


@pytest.mark.parametrize("boundary,H,W,sg", [("zero", 300, 200, [16.0, 32.0]), ("mirror", 150, 170, [32.0]),
                                             ("replicate", 97, 701, [4.0, 32.0]), ("zero", 40, 1300, [2.0, 32.0])])
def test_iir_sigma_32(boundary, H, W, sg):
    # the largest sigma of the 64-image batch, rows and columns longer than one scan group
    img = synth.pink_noise([23, H, W], H, W)
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6]
    om = [math.pi / s for s in sg]
    got = _run(img, th, om, sg, boundary=boundary)
    iir_check(got, oracle.iir_gabor_bank(img, th, om, sg, boundary=boundary), img, sg, boundary)


def test_iir_paper_bank_and_ser_against_fir():
    img = synth.paper_like(0, 160, 200)
    th, om, sg = c2_bank()
    got = _run(img, th, om, sg)
    ref = oracle.iir_gabor_bank(img, th, om, sg)
    iir_check(got, ref, img, sg)
    fir = oracle.gabor_bank(img, th, om, sg)
    for s in range(len(om)):
        re_db, im_db = oracle.ser_db(got[s], fir[s])
        print(f"omega {om[s]:.4f} sigma {sg[s]:.2f}: SER re {re_db:.1f} dB im {im_db:.1f} dB")
        assert im_db > 10.0


def test_iir_layout_batch_and_reuse_off():
    import torch
    from paper_1704_05231_gb300 import GaborBank
    th, om, sg = c2_bank()
    imgs = [torch.from_numpy(synth.pink_noise([22, i], h, w)).cuda() for i, (h, w) in enumerate([(40, 70), (96, 64)])]
    with GaborBank(th, om, sg, smoother="iir") as a, GaborBank(th, om, sg, smoother="iir", layout="pixels") as b:
        singles = [a.filter(t).cpu().numpy() for t in imgs]
        batch = [o.cpu().numpy() for o in a.filter_batch(imgs)]
        pixels = b.filter(imgs[0]).cpu().numpy()
        a.set_option("reuse", 0)
        noreuse = a.filter(imgs[0]).cpu().numpy()
    for s_, b_ in zip(singles, batch):
        assert np.array_equal(s_, b_)
    assert np.array_equal(np.moveaxis(singles[0], (0, 1), (2, 3)), pixels)
    assert rel_err(noreuse, singles[0]) <= 2 * FP32_TOL


def test_iir_refused_on_tensor_cores():
    import torch
    from paper_1704_05231_gb300 import GaborBank, GBError
    th, om, sg = c1_bank()
    with GaborBank(th, om, sg, precision="fp16_tc", smoother="iir") as gbk:
        with pytest.raises(GBError) as ei:
            gbk.filter(torch.zeros((16, 16), dtype=torch.float32, device="cuda"))
        assert ei.value.status == -4
