"""Uneven batches (the 64-image workload's shapes): one persistent launch, CUDA-graph replay,
autotuned tiling, and parity against the FP64 oracle on sampled pixels of a 8 x 5 bank."""
import math

import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, TC_TOL, rel_err, sample_points

pytestmark = pytest.mark.gpu


def c4_bank():
    thetas = [k * math.pi / 8 for k in range(8)]
    omegas = [math.pi / 2 ** (s + 1) for s in range(5)]      # pi/2 .. pi/32
    sigmas = [math.pi / w for w in omegas]                     # 2 .. 32 (R up to 96)
    return thetas, omegas, sigmas


def small_batch(n=4, lo=40, hi=220):
    return [synth.pink_noise([1, i], h, w) for i, (h, w) in enumerate(synth.batch_shapes(1, n, lo, hi))]


def test_batch_graph_and_autotune_bitwise():
    import torch
    from paper_1704_05231_gb300 import GaborBank, bank, tune
    imgs = small_batch()
    th, om, sg = c4_bank()
    with GaborBank(th, om, sg) as gbk:
        ts = [torch.from_numpy(i).cuda() for i in imgs]
        singles = [gbk.filter(t).clone() for t in ts]
        outs = [torch.empty_like(s) for s in singles]
        gbk.filter_batch(ts, outs)
        for a, b in zip(singles, outs):
            assert torch.equal(a, b)
        for o in outs:
            o.zero_()
        g = bank.capture_graph(lambda: gbk.filter_batch(ts, outs))
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(singles, outs):
            assert torch.equal(a, b)
        res = tune.autotune(gbk, ts, use_cache=False, steps=1)
        assert len(res["tiling"]) == len(om)
        gbk.filter_batch(ts, outs)
        torch.cuda.synchronize()
        for a, b in zip(singles, outs):
            assert torch.equal(a, b)


@pytest.mark.parametrize("precision,tol", [("fp32", FP32_TOL), ("fp16_tc", TC_TOL)])
def test_c4_shapes_sampled_parity(precision, tol):
    import torch
    from paper_1704_05231_gb300 import GaborBank
    shapes = sorted(synth.batch_shapes(1, 64, 128, 2048), key=lambda s: s[0] * s[1])[:3]
    th, om, sg = c4_bank()
    rng = np.random.default_rng(4)
    with GaborBank(th, om, sg, precision=precision) as gbk:
        imgs = [synth.pink_noise([1, 100 + i], h, w) for i, (h, w) in enumerate(shapes)]
        outs = gbk.filter_batch([torch.from_numpy(i).cuda() for i in imgs])
        gbk.device_status()
        for img, out in zip(imgs, outs):
            got = out.cpu().numpy()
            H, W = img.shape
            xs, ys = sample_points(rng, H, W, 120)
            ref = oracle.gabor_bank(img, th, om, sg, points=(xs, ys))
            scale = float(np.max(np.abs(got)))
            assert float(np.max(np.abs(ref))) <= scale * (1 + 1e-3)
            assert float(np.max(np.abs(got[:, :, ys, xs] - ref))) <= tol * scale


def test_tc_batch_matches_fp32_on_small_images():
    import torch
    from paper_1704_05231_gb300 import GaborBank
    imgs = small_batch(3)
    th, om, sg = c4_bank()
    ts = [torch.from_numpy(i).cuda() for i in imgs]
    with GaborBank(th, om, sg) as g32, GaborBank(th, om, sg, precision="fp16_tc") as g16:
        a = g32.filter_batch(ts)
        b = g16.filter_batch(ts)
        for x, y in zip(a, b):
            assert rel_err(y.cpu().numpy(), x.cpu().numpy()) <= TC_TOL
