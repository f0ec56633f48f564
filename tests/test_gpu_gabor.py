"""GPU parity of the FP32 Gabor bank (Algorithm 1, Eq. 1-16) against the FP64 oracle.

Every test calls the CUDA path through the C ABI (ctypes binding) and compares element by
element with the direct 2-D sum of Eq. 1 on the same seeded FP32 image; the bar is
max|err| <= 1e-5 * max|out| over each result tensor.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, c1_bank, c2_bank, plane_rel_errs, rel_err, sample_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def run_bank(torch, img, thetas, omegas, sigmas, **kw):
    from paper_1704_05231_gb300 import GaborBank
    with GaborBank(thetas, omegas, sigmas, **kw) as gbk:
        t = torch.from_numpy(img).cuda()
        out = gbk.filter(t)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def test_c1_full_parity(torch_cuda):
    img = synth.uniform01(0, 256, 256)
    th, om, sg = c1_bank()
    got = run_bank(torch_cuda, img, th, om, sg)
    ref = oracle.gabor_bank(img, th, om, sg)
    assert got.shape == (2, 4, 256, 256)
    e = rel_err(got, ref)
    print("C1 rel err", e, "worst plane", max(plane_rel_errs(got, ref)))
    assert e <= FP32_TOL


@pytest.mark.parametrize("H,W", [(37, 75), (1, 50), (50, 1), (3, 3), (64, 64), (129, 33), (200, 161)])
def test_ragged_and_degenerate_sizes(torch_cuda, H, W):
    img = synth.pink_noise([7, H, W], H, W)
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6, 2.0]
    om = [math.pi / 3, 0.4]
    sg = [1.5, 5.0]   # R = 5 and 15: radius above the image size for the small cases
    got = run_bank(torch_cuda, img, th, om, sg)
    ref = oracle.gabor_bank(img, th, om, sg)
    assert rel_err(got, ref) <= FP32_TOL


def test_pitch_and_strided_view(torch_cuda):
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    big = synth.uniform01(3, 90, 140)
    th, om, sg = c1_bank()
    view = torch.from_numpy(big).cuda()[5:80, 7:120]   # pitch 140 != W 113
    with GaborBank(th, om, sg) as gbk:
        got = gbk.filter(view).cpu().numpy()
    ref = oracle.gabor_bank(big[5:80, 7:120], th, om, sg)
    assert rel_err(got, ref) <= FP32_TOL


def test_row_loads_by_tma_follow_the_image(torch_cuda):
    # A one-image launch under the zero rule loads its row blocks as TMA boxes through maps that
    # the handle encodes once per image and tile geometry and keeps.  Calls on other buffers
    # must re-encode (each result equal to a fresh handle's), and views whose row pitch is not a
    # multiple of 16 bytes take the per-thread async copies instead, with the same arithmetic:
    # the same pixels give the same bits either way.
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    H, W = 150, 203
    th, om, sg = c2_bank()   # R up to 48: several row blocks per item, ragged last strip
    ta = torch.from_numpy(synth.paper_like(0, H, W)).cuda()
    tb = torch.from_numpy(synth.pink_noise([5, H, W], H, W)).cuda()
    wide = torch.zeros((H, W + 2), dtype=torch.float32, device="cuda")   # pitch 820 bytes
    wide[:, :W] = ta
    tc = wide[:, :W]
    wide2 = torch.zeros((H, W + 5), dtype=torch.float32, device="cuda")  # base 4 bytes past
    wide2[:, 1:W + 1] = ta
    td = wide2[:, 1:W + 1]
    with GaborBank(th, om, sg) as g:
        outs = [g.filter(t).cpu().numpy() for t in (ta, tb, ta, tc, td, tb)]
    fresh = {}
    for name, t in (("a", ta), ("b", tb)):
        with GaborBank(th, om, sg) as g:
            fresh[name] = g.filter(t).cpu().numpy()
    for got, name in zip(outs, ("a", "b", "a", "a", "a", "b")):
        assert np.array_equal(got, fresh[name])
    # and the first image against the FP64 oracle at sampled pixels
    xs, ys = sample_points(np.random.default_rng(3), H, W, 200)
    ref = oracle.gabor_bank(ta.cpu().numpy(), th, om, sg, points=(xs, ys))
    got = outs[0][:, :, ys, xs]
    assert rel_err(got, ref) <= FP32_TOL


def test_c2_bank_reduced_size_full_parity(torch_cuda):
    # The paper-size bank (sigma up to 16, R = 48) on a 160 x 200 image: halos wider than
    # a quarter of the image, several tiles and ragged edges.
    img = synth.paper_like(0, 160, 200)
    th, om, sg = c2_bank()
    got = run_bank(torch_cuda, img, th, om, sg)
    ref = oracle.gabor_bank(img, th, om, sg)
    e = rel_err(got, ref)
    print("C2-bank 160x200 rel err", e)
    assert e <= FP32_TOL


@pytest.fixture(scope="module")
def c2_full():
    """The paper-size bank's image (1024 x 1024, seed 0) and its FP64 oracle result in full:
    the direct 2-D sum of Eq. 1 at all 25.2 M outputs (all host cores)."""
    img = synth.paper_like(0, 1024, 1024)
    th, om, sg = c2_bank()
    return img, oracle.gabor_bank(img, th, om, sg)


def test_c2_full_size_full_oracle(torch_cuda, c2_full):
    # The benchmark's workload, every output against the oracle; scale = max|oracle|.
    img, ref = c2_full
    th, om, sg = c2_bank()
    got = run_bank(torch_cuda, img, th, om, sg)
    assert np.all(np.isfinite(got))
    e = rel_err(got, ref)
    print("C2 1024^2 FP32 rel err (full oracle)", e, "worst plane", max(plane_rel_errs(got, ref)))
    assert e <= FP32_TOL


def test_orientation_order_and_reuse_ablation(torch_cuda):
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    img = synth.pink_noise(5, 96, 130)
    th = [2 * math.pi / 3, 0.0, math.pi / 3, math.pi / 2, 5 * math.pi / 6, math.pi / 6]
    om, sg = [0.8], [2.5]
    t = torch.from_numpy(img).cuda()
    with GaborBank(th, om, sg) as gbk:
        a = gbk.filter(t).cpu().numpy()
        gbk.set_option("reuse", 0)          # recompute J for every orientation
        b = gbk.filter(t).cpu().numpy()
    ref = oracle.gabor_bank(img, th, om, sg)
    assert rel_err(a, ref) <= FP32_TOL
    assert rel_err(b, ref) <= FP32_TOL
    # reversing the orientation list permutes the planes only
    with GaborBank(th[::-1], om, sg) as gbk:
        c = gbk.filter(t).cpu().numpy()
    assert rel_err(c[:, ::-1], ref) <= FP32_TOL


def test_conjugate_symmetry_theta_plus_pi(torch_cuda):
    img = synth.pink_noise(9, 70, 90)
    th = [0.4, 0.4 + math.pi]
    got = run_bank(torch_cuda, img, th, [1.0], [2.0])
    assert rel_err(got[0, 1], np.conj(got[0, 0])) <= FP32_TOL


def test_batch_equals_single_bitwise_and_host_path(torch_cuda):
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    imgs = [synth.pink_noise([1, i], h, w) for i, (h, w) in enumerate([(40, 70), (128, 96), (33, 257)])]
    th, om, sg = c1_bank()
    with GaborBank(th, om, sg) as gbk:
        ts = [torch.from_numpy(i).cuda() for i in imgs]
        singles = [gbk.filter(t).cpu().numpy() for t in ts]
        batch = [o.cpu().numpy() for o in gbk.filter_batch(ts)]
        host = [gbk.filter_host(i) for i in imgs]
    for s, b, h in zip(singles, batch, host):
        assert np.array_equal(s, b)
        assert np.array_equal(s, h)


def test_impulse_response_on_gpu(torch_cuda):
    # The bank applied to an impulse reproduces the Gabor kernel of Eq. 1-2 (interior).
    H, W, x0, y0 = 64, 64, 30, 33
    img = synth.impulse(H, W, x0, y0)
    om, th, sg = 0.7, 0.5, 3.0
    got = run_bank(torch_cuda, img, [th], [om], [sg])[0, 0]
    ref = oracle.gabor_filter(img, om, th, sg)
    assert rel_err(got, ref) <= FP32_TOL


# ---------------------------------------------------------------- tensor-core bank

@pytest.mark.parametrize("precision", ["fp16_tc", "bf16_tc"])
def test_tc_bank_c1_full_parity(torch_cuda, precision):
    from tests.helpers import TC_TOL
    img = synth.uniform01(0, 256, 256)
    th, om, sg = c1_bank()
    got = run_bank(torch_cuda, img, th, om, sg, precision=precision)
    ref = oracle.gabor_bank(img, th, om, sg)
    e = rel_err(got, ref)
    print("TC C1", precision, "rel err", e, "worst plane", max(plane_rel_errs(got, ref)))
    assert e <= TC_TOL


@pytest.mark.parametrize("precision", ["fp16_tc", "bf16_tc"])
@pytest.mark.parametrize("H,W", [(37, 75), (160, 200), (1, 50), (129, 33)])
def test_tc_bank_ragged_and_c2_bank(torch_cuda, precision, H, W):
    from tests.helpers import TC_TOL
    img = synth.paper_like(0, H, W) if H > 8 and W > 8 else synth.pink_noise([3, H, W], H, W)
    th, om, sg = c2_bank()
    got = run_bank(torch_cuda, img, th, om, sg, precision=precision)
    ref = oracle.gabor_bank(img, th, om, sg)
    e = rel_err(got, ref)
    print("TC", precision, H, W, "rel err", e)
    assert e <= TC_TOL


@pytest.mark.parametrize("precision", ["fp16_tc", "bf16_tc"])
def test_tc_bank_c2_full_size_full_oracle(torch_cuda, c2_full, precision):
    from tests.helpers import TC_TOL
    img, ref = c2_full
    th, om, sg = c2_bank()
    got = run_bank(torch_cuda, img, th, om, sg, precision=precision)
    assert np.all(np.isfinite(got))
    e = rel_err(got, ref)
    print("C2 1024^2", precision, "rel err (full oracle)", e, "worst plane", max(plane_rel_errs(got, ref)))
    assert e <= TC_TOL


def test_tc_bank_unpaired_orientations_and_reuse_off(torch_cuda):
    from paper_1704_05231_gb300 import GaborBank
    from tests.helpers import TC_TOL
    torch = torch_cuda
    img = synth.pink_noise(17, 90, 140)
    th = [0.3, 1.2, math.pi - 0.3, 2.0]
    om, sg = [0.9, 0.45], [2.0, 4.5]
    t = torch.from_numpy(img).cuda()
    ref = oracle.gabor_bank(img, th, om, sg)
    with GaborBank(th, om, sg, precision="fp16_tc") as gbk:
        a = gbk.filter(t).cpu().numpy()
        gbk.set_option("reuse", 0)
        b = gbk.filter(t).cpu().numpy()
        gbk.device_status()
    assert rel_err(a, ref) <= TC_TOL
    assert rel_err(b, ref) <= TC_TOL


def test_tc_bank_bf16_hi_lo_and_its_limits(torch_cuda):
    # BF16 operands as hi + lo pairs (three products per K step): far inside the tensor-core
    # bound (well below the FP16 error), equal to the FP32 path to about 1e-5; the
    # step-by-step kernels take FP16 operands only, so that form refuses BF16.
    from paper_1704_05231_gb300 import GaborBank, GBError
    from tests.helpers import TC_TOL
    torch = torch_cuda
    img = synth.paper_like(9, 96, 130)
    th, om, sg = c2_bank()
    t = torch.from_numpy(img).cuda()
    ref = oracle.gabor_bank(img, th, om, sg)
    with GaborBank(th, om, sg, precision="bf16_tc") as gbk:
        b = gbk.filter(t).cpu().numpy()
        gbk.device_status()
        gbk.set_option("row_pass", 1)
        with pytest.raises(GBError) as ei:
            gbk.filter(t)
        assert ei.value.status == -4
    with GaborBank(th, om, sg, precision="fp16_tc") as gbk:
        h = gbk.filter(t).cpu().numpy()
    eb, eh = rel_err(b, ref), rel_err(h, ref)
    print("BF16 hi+lo rel err", eb, "FP16", eh)
    assert eb <= TC_TOL and eb <= 0.1 * eh


def _schedules(torch, imgs, th, om, sg, opts=(), **kw):
    """Outputs of the phased (GB_OPT_PIPELINE = 1) and pipelined (= 2) FP32 schedules."""
    from paper_1704_05231_gb300 import GaborBank
    res = []
    for sched in (1, 2):
        with GaborBank(th, om, sg, **kw) as gbk:
            gbk.set_option("pipeline", sched)
            for k, v in opts:
                gbk.set_option(k, v)
            outs = [gbk.filter(torch.from_numpy(i).cuda()).cpu().numpy() for i in imgs]
            gbk.device_status()
        res.append(outs)
    return res


@pytest.mark.parametrize("H,W", [(1, 50), (37, 75), (129, 33), (200, 161), (300, 96)])
def test_pipelined_schedule_matches_phased_and_oracle(torch_cuda, H, W):
    # Warp-specialised schedule: same operations per output, so the results are identical.
    img = synth.pink_noise([17, H, W], H, W)
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6, 2.0]
    om = [math.pi / 3, 0.4, 0.2]
    sg = [1.5, 5.0, 11.0]
    (a,), (b,) = _schedules(torch_cuda, [img], th, om, sg)
    assert np.array_equal(a, b)
    assert rel_err(b, oracle.gabor_bank(img, th, om, sg)) <= FP32_TOL


@pytest.mark.parametrize("tile_rows,segments", [(8, 0), (16, 3), (32, 1), (64, 2)])
def test_pipelined_schedule_tilings(torch_cuda, tile_rows, segments):
    img = synth.paper_like(4, 230, 170)
    th, om, sg = c2_bank()
    (a,), (b,) = _schedules(torch_cuda, [img], th, om, sg,
                            opts=(("tile_rows", tile_rows), ("segments", segments)))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("boundary", ["zero", "replicate", "mirror"])
@pytest.mark.parametrize("layout", ["planes", "pixels"])
def test_pipelined_schedule_boundary_and_layout(torch_cuda, boundary, layout):
    img = synth.pink_noise(23, 90, 140)
    th, om, sg = c1_bank()
    (a,), (b,) = _schedules(torch_cuda, [img], th, om, sg, boundary=boundary, layout=layout)
    assert np.array_equal(a, b)
    if layout == "planes":
        assert rel_err(b, oracle.gabor_bank(img, th, om, sg, boundary=boundary)) <= FP32_TOL


def test_pipelined_schedule_batch_and_large_radius(torch_cuda):
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    imgs = [synth.pink_noise([29, i], h, w) for i, (h, w) in enumerate([(40, 70), (128, 96), (333, 257)])]
    th = [0.3, math.pi - 0.3, math.pi / 2]
    om, sg = [0.05, 0.9], [53.0, 2.0]   # R = 159: the largest FP32 radius, pipelined tile of 8 rows
    (sa, sb) = _schedules(torch, imgs, th, om, sg)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    with GaborBank(th, om, sg) as gbk:
        gbk.set_option("pipeline", 2)
        batch = [o.cpu().numpy() for o in gbk.filter_batch([torch.from_numpy(i).cuda() for i in imgs])]
        gbk.device_status()
    for x, y in zip(sb, batch):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("row_pass", [1, 2])
@pytest.mark.parametrize("boundary", ["zero", "mirror"])
@pytest.mark.parametrize("H,W", [(1, 50), (37, 75), (200, 161)])
def test_row_pass_forms_match_oracle(torch_cuda, row_pass, boundary, H, W):
    # Eq. 5-6 as demodulate / smooth / remodulate (1) and as one modulated-tap pass (2);
    # radii 1, 5, 33 (tap chunks 1, 2, 9: both tap-split parities of the modulated form)
    from paper_1704_05231_gb300 import GaborBank
    img = synth.pink_noise([31, H, W], H, W)
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6, 2.0]
    om, sg = [2.5, 0.4, 0.15], [0.3, 1.5, 11.0]
    with GaborBank(th, om, sg, boundary=boundary) as gbk:
        gbk.set_option("row_pass", row_pass)
        got = gbk.filter(torch_cuda.from_numpy(img).cuda()).cpu().numpy()
        gbk.device_status()
    assert rel_err(got, oracle.gabor_bank(img, th, om, sg, boundary=boundary)) <= FP32_TOL


@pytest.mark.parametrize("row_pass", [1, 2])
def test_row_pass_forms_c2_full_and_large_radius_sampled(torch_cuda, c2_full, row_pass):
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    img, ref = c2_full
    with GaborBank(*c2_bank()) as gbk:
        gbk.set_option("row_pass", row_pass)
        got = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
    assert rel_err(got, ref) <= FP32_TOL
    # R = 159 (the largest FP32 radius) on sampled pixels; scale = max|oracle| over the samples
    rng = np.random.default_rng(5)
    th, om, sg = [0.3, math.pi - 0.3, math.pi / 2], [0.05], [53.0]
    img = synth.paper_like(2, 333, 257)
    with GaborBank(th, om, sg) as gbk:
        gbk.set_option("row_pass", row_pass)
        got = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
    xs, ys = sample_points(rng, 333, 257, 300)
    ref = oracle.gabor_bank(img, th, om, sg, points=(xs, ys))
    assert np.all(np.isfinite(got))
    assert rel_err(got[:, :, ys, xs], ref) <= FP32_TOL


def test_row_pass_forms_pipelined_bitwise(torch_cuda):
    img = synth.paper_like(6, 230, 170)
    th, om, sg = c2_bank()
    for form in (1, 2):
        (a,), (b,) = _schedules(torch_cuda, [img], th, om, sg, opts=(("row_pass", form),))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("row_pass", [1, 2])
@pytest.mark.parametrize("boundary", ["zero", "replicate"])
def test_two_ctas_per_sm_bitwise(torch_cuda, row_pass, boundary):
    # GB_OPT_BANK_CTAS = 2: two CTAs of 8 warps per SM (two row-pass sweeps per block, smaller
    # tiles for large radii); every output takes the same operations as with one CTA of 16.
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    imgs = [synth.pink_noise([37, i], h, w) for i, (h, w) in enumerate([(37, 75), (300, 161), (1, 40)])]
    th = [0.0, 0.6, math.pi / 2, math.pi - 0.6, 2.0]
    om, sg = [2.5, 0.4, 0.15, 0.05], [0.3, 1.5, 11.0, 40.0]   # R up to 120
    res = []
    for ctas in (1, 2):
        with GaborBank(th, om, sg, boundary=boundary) as gbk:
            gbk.set_option("row_pass", row_pass)
            gbk.set_option("bank_ctas", ctas)
            ts = [torch.from_numpy(i).cuda() for i in imgs]
            res.append([gbk.filter(t).cpu().numpy() for t in ts] +
                       [o.cpu().numpy() for o in gbk.filter_batch(ts)])
            gbk.device_status()
    for x, y in zip(*res):
        assert np.array_equal(x, y)
    ref = oracle.gabor_bank(imgs[0], th, om, sg, boundary=boundary)
    assert rel_err(res[1][0], ref) <= FP32_TOL


def test_c2_full_size_tuned_geometry_bitwise(torch_cuda):
    # The geometry the benchmark's autotuner picks (two CTAs of 8 warps per SM, per-frequency
    # tiles and segments) gives the same bits as the default geometry on the full-size bank.
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    img = torch.from_numpy(synth.paper_like(0, 1024, 1024)).cuda()
    th, om, sg = c2_bank()
    with GaborBank(th, om, sg) as gbk:
        ref = gbk.filter(img).cpu().numpy()
        gbk.set_option("bank_ctas", 2)
        for s, (tr, seg) in enumerate([(0, 2), (0, 2), (0, 0), (32, 2)]):
            gbk.set_tiling(s, tr, seg)
        got = gbk.filter(img).cpu().numpy()
        gbk.device_status()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("row_pass", [1, 2])
@pytest.mark.parametrize("boundary", ["zero", "mirror"])
@pytest.mark.parametrize("H,W", [(37, 75), (160, 200), (129, 33)])
def test_tc_bank_row_pass_forms(torch_cuda, row_pass, boundary, H, W):
    # Tensor-core bank: row pass as demodulated operand x Toeplitz (1) or modulated-tap operand
    # x patch (2); both within the tensor-core bound of the FP64 oracle.
    from paper_1704_05231_gb300 import GaborBank
    from tests.helpers import TC_TOL
    img = synth.paper_like([43, H, W], H, W)
    th, om, sg = c2_bank()
    with GaborBank(th, om, sg, precision="fp16_tc", boundary=boundary) as gbk:
        gbk.set_option("row_pass", row_pass)
        got = gbk.filter(torch_cuda.from_numpy(img).cuda()).cpu().numpy()
        gbk.device_status()
    e = rel_err(got, oracle.gabor_bank(img, th, om, sg, boundary=boundary))
    print("TC row pass", row_pass, boundary, H, W, "rel err", e)
    assert e <= TC_TOL


@pytest.mark.parametrize("row_pass,precision", [(1, "fp16_tc"), (2, "fp16_tc"), (2, "bf16_tc")])
@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_tc_bank_large_radius_sampled(torch_cuda, row_pass, precision, boundary):
    # Batched-bank frequencies pi/2 .. pi/32 (sigma = pi / omega, radii 6 .. 96): with radius
    # 96 the modulated-tap column pass takes 32-row jobs (the 64-row operands exceed shared
    # memory); ragged sizes put partial jobs at both image edges.
    from paper_1704_05231_gb300 import GaborBank
    from tests.helpers import TC_TOL
    torch = torch_cuda
    rng = np.random.default_rng(23)
    th = [k * math.pi / 8 for k in range(8)]
    om = [math.pi / 2 ** k for k in range(1, 6)]
    sg = [math.pi / w for w in om]
    for H, W in [(333, 257), (97, 530)]:
        img = synth.paper_like([47, H, W], H, W)
        with GaborBank(th, om, sg, precision=precision, boundary=boundary) as gbk:
            gbk.set_option("row_pass", row_pass)
            got = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
            gbk.device_status()
        with GaborBank(th, om, sg, boundary=boundary) as gbk:
            f32 = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
        e = rel_err(got, f32)
        print("TC large radius", row_pass, precision, boundary, H, W, "rel err vs FP32", e)
        assert e <= TC_TOL
        xs, ys = sample_points(rng, H, W, 200)
        ref = oracle.gabor_bank(img, th, om, sg, points=(xs, ys), boundary=boundary)
        # scale = max|oracle| over the samples (at most the result's max: a stricter bound)
        assert rel_err(got[:, :, ys, xs], ref) <= TC_TOL
        assert rel_err(f32[:, :, ys, xs], ref) <= FP32_TOL


@pytest.mark.parametrize("layout", ["planes", "pixels"])
def test_host_path_per_frequency_copies_bitwise(torch_cuda, layout):
    # gabor_bank_filter_host on pinned buffers: per-frequency launches whose planes are copied
    # back while the next frequency computes (plane-major layout), or one launch (pixel-major);
    # bitwise the device call's result either way, and repeated calls give the same bits.
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    img = synth.paper_like(3, 300, 410)
    th, om, sg = c2_bank()
    with GaborBank(th, om, sg, layout=layout) as gbk:
        dev = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
        h_img = torch.from_numpy(img).pin_memory()
        h_out = torch.full(gbk.out_shape(300, 410), float("nan"), dtype=torch.complex64).pin_memory()
        for _ in range(2):
            gbk.filter_host_ptr(h_img.data_ptr(), 300, 410, 410, h_out.data_ptr())
            assert np.array_equal(h_out.numpy(), dev)
            h_out.fill_(float("nan"))
