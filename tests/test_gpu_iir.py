"""The recursive-Gaussian bank (GB_SMOOTHER_IIR) on the GPU against the FP64 oracle of the
same recursion (Algorithm 1 with the Young-van Vliet smoother), element by element; and its
SER against the exact FIR bank (Sec. IV-C), reported and bounded from below.

Tolerance: the recursion's feedback coefficients sum to 1 - B with B ~ 1 / sigma^3, so FP32
rounding errors circulate for ~sigma samples; one FP32 pass over a [0, 1] signal measures
4e-7 (sigma 2), 5e-6 (4), 3e-5 (8), 2.6e-4 (16), 3e-3 (32) relative to its FP64 result.  The
bar is max(1e-5, 2e-7 sigma_max^3) * max|out| per result tensor.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, c1_bank, c2_bank, rel_err


def iir_tol(sigmas):
    return max(FP32_TOL, 2e-7 * max(sigmas) ** 3)

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
    e = rel_err(got, ref)
    print("IIR C1 rel err", e, "SER vs FIR", oracle.ser_db(got, oracle.gabor_bank(img, th, om, sg)))
    assert e <= iir_tol(sg)


@pytest.mark.parametrize("boundary", ["zero", "replicate", "mirror"])
@pytest.mark.parametrize("H,W", [(37, 75), (129, 33), (3, 3), (1, 50)])
def test_iir_ragged_and_boundaries(boundary, H, W):
    img = synth.pink_noise([21, H, W], H, W)
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6]
    om, sg = [math.pi / 3, 0.4], [1.5, 5.0]
    got = _run(img, th, om, sg, boundary=boundary)
    ref = oracle.iir_gabor_bank(img, th, om, sg, boundary=boundary)
    assert rel_err(got, ref) <= iir_tol(sg)


def test_iir_paper_bank_and_ser_against_fir():
    img = synth.paper_like(0, 160, 200)
    th, om, sg = c2_bank()
    got = _run(img, th, om, sg)
    ref = oracle.iir_gabor_bank(img, th, om, sg)
    e = rel_err(got, ref)
    print("IIR paper bank 160x200 rel err", e, "bar", iir_tol(sg))
    assert e <= iir_tol(sg)
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
    assert rel_err(noreuse, singles[0]) <= iir_tol(sg)


def test_iir_refused_on_tensor_cores():
    import torch
    from paper_1704_05231_gb300 import GaborBank, GBError
    th, om, sg = c1_bank()
    with GaborBank(th, om, sg, precision="fp16_tc", smoother="iir") as gbk:
        with pytest.raises(GBError) as ei:
            gbk.filter(torch.zeros((16, 16), dtype=torch.float32, device="cuda"))
        assert ei.value.status == -4
