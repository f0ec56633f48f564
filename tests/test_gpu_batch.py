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


@pytest.fixture(scope="module")
def c4_batch():
    """The 64-image batch exactly as the benchmark makes it (sides U[128, 2048] from seed 1,
    1/f noise synthesised on the device from seeds 1000 + i), run through the same
    gabor_bank_filter_batch call replayed from a captured CUDA graph, for the FP32 and the
    FP16 tensor-core handles.  Returns the host images and, per precision, the device outputs."""
    import torch
    from paper_1704_05231_gb300 import GaborBank
    from paper_1704_05231_gb300.bank import capture_graph
    shapes = synth.batch_shapes(1, 64, 128, 2048)
    imgs = [synth.pink_noise_device(1000 + i, h, w) for i, (h, w) in enumerate(shapes)]
    th, om, sg = c4_bank()
    outs = {}
    for prec in ("fp32", "fp16_tc"):
        with GaborBank(th, om, sg, precision=prec, max_shape=(2048, 2048)) as gbk:
            o = [torch.full(gbk.out_shape(h, w), float("nan"), dtype=torch.complex64, device="cuda")
                 for h, w in shapes]
            graph = capture_graph(lambda: gbk.filter_batch(imgs, o))
            for x in o:
                x.fill_(float("nan"))
            graph.replay()
            torch.cuda.synchronize()
            gbk.device_status()
            del graph
        outs[prec] = o
    host = [i.cpu().numpy() for i in imgs]
    del imgs
    return shapes, host, outs


@pytest.fixture(scope="module")
def c4_smallest_oracle(c4_batch):
    """The FP64 oracle in full on the 4 smallest images of the batch (by pixel count)."""
    shapes, host, _ = c4_batch
    th, om, sg = c4_bank()
    idx = sorted(range(len(shapes)), key=lambda i: shapes[i][0] * shapes[i][1])[:4]
    return {i: oracle.gabor_bank(host[i], th, om, sg) for i in idx}


@pytest.mark.parametrize("precision,tol", [("fp32", FP32_TOL), ("fp16_tc", TC_TOL)])
def test_c4_batch_smallest_images_full_oracle(c4_batch, c4_smallest_oracle, precision, tol):
    _, _, outs = c4_batch
    for i, ref in c4_smallest_oracle.items():
        got = outs[precision][i].cpu().numpy()
        assert np.all(np.isfinite(got))
        e = rel_err(got, ref)
        print("C4 image", i, got.shape, precision, "rel err (full oracle)", e)
        assert e <= tol


@pytest.mark.parametrize("precision,tol", [("fp32", FP32_TOL), ("fp16_tc", TC_TOL)])
def test_c4_batch_every_image_sampled_oracle(c4_batch, precision, tol):
    # 256 seeded pixels of every image (all 40 planes each, corners and border bands
    # included), against the oracle; scale = max|oracle| over the image's samples
    import torch
    shapes, host, outs = c4_batch
    th, om, sg = c4_bank()
    rng = np.random.default_rng(44)
    worst = 0.0
    for i, (H, W) in enumerate(shapes):
        xs, ys = sample_points(rng, H, W, 256)
        ix = torch.from_numpy(ys.astype(np.int64) * W + xs).cuda()
        got = outs[precision][i].reshape(len(om), len(th), H * W)[:, :, ix].cpu().numpy()
        ref = oracle.gabor_bank(host[i], th, om, sg, points=(xs, ys))
        e = rel_err(got, ref)
        worst = max(worst, e)
        assert e <= tol, (i, H, W, e)
    print("C4", precision, "worst sampled rel err over 64 images", worst)


def test_c4_batch_fp32_and_tc_agree_everywhere(c4_batch):
    # A property that holds at any size: on every image the two paths agree within the
    # tensor-core bound at every output, and no output is non-finite.
    import torch
    shapes, _, outs = c4_batch
    for i in range(len(shapes)):
        a, b = outs["fp32"][i], outs["fp16_tc"][i]
        assert bool(torch.isfinite(torch.view_as_real(a)).all()) and bool(torch.isfinite(torch.view_as_real(b)).all())
        scale = float(a.abs().max())
        assert float((a - b).abs().max()) <= TC_TOL * scale, i


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


@pytest.mark.parametrize("precision", ["fp16_tc", "bf16_tc"])
@pytest.mark.parametrize("boundary,layout", [("zero", "planes"), ("mirror", "planes"), ("zero", "pixels")])
def test_tc_batch_one_launch_set_bitwise_equals_single_calls(boundary, layout, precision):
    # Tensor-core batch: one k_minmax, one k_ones, one row and one column launch for all images;
    # every output takes the same MMAs as in a single-image call, so the results are bitwise
    # those of one call per image, also when replayed from a captured CUDA graph.
    import torch
    from paper_1704_05231_gb300 import GaborBank
    from paper_1704_05231_gb300.bank import capture_graph
    shapes = [(40, 70), (128, 96), (333, 257), (7, 300), (190, 41)]
    imgs = [torch.from_numpy(synth.pink_noise([61, i], h, w)).cuda() for i, (h, w) in enumerate(shapes)]
    th, om, sg = c4_bank()
    with GaborBank(th, om, sg, precision=precision, boundary=boundary, layout=layout) as gbk:
        singles = [gbk.filter(t).clone() for t in imgs]
        outs = [torch.full_like(s, float("nan")) for s in singles]
        gbk.filter_batch(imgs, outs)
        gbk.device_status()
        for a, b in zip(singles, outs):
            assert torch.equal(a, b)
        g = capture_graph(lambda: gbk.filter_batch(imgs, outs))
        for o in outs:
            o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        gbk.device_status()
        for a, b in zip(singles, outs):
            assert torch.equal(a, b)
    if layout == "planes":
        ref = oracle.gabor_bank(imgs[0].cpu().numpy(), th, om, sg, boundary=boundary)
        assert rel_err(singles[0].cpu().numpy(), ref) <= TC_TOL


@pytest.mark.parametrize("precision", ["fp16_tc", "bf16_tc"])
def test_tc_tile_choices_and_autotune_bitwise(precision):
    # GB_OPT_TC_TILES (rows per row item / column job: 32 or 64) changes no result; the
    # autotuner's tensor-core branch times the choices and applies one.
    import torch
    from paper_1704_05231_gb300 import GaborBank, tune
    th, om, sg = c4_bank()
    imgs = [torch.from_numpy(synth.pink_noise([71, i], h, w)).cuda() for i, (h, w) in enumerate([(150, 230), (97, 64)])]
    res = []
    with GaborBank(th, om, sg, precision=precision) as gbk:
        for r, c in ((64, 64), (32, 64), (64, 32), (32, 32)):
            gbk.set_option("tc_tiles", r + 256 * c)
            res.append([gbk.filter(t).clone() for t in imgs] + [o.clone() for o in gbk.filter_batch(imgs)])
            gbk.device_status()
        t = tune.autotune(gbk, imgs, use_cache=False, steps=1)
        assert t["tc_tiles"][0] in (32, 64) and t["tc_tiles"][1] in (32, 64)
        res.append([gbk.filter(t_).clone() for t_ in imgs])
        gbk.device_status()
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert torch.equal(a, b)
