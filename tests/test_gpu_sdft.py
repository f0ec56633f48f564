"""GPU parity of the localized sliding DFT (Algorithm 2, Eq. 17-26) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def run_sdft(torch, img, sigma, M, half=False, precision="fp32"):
    from paper_1704_05231_gb300 import GaborBank
    with GaborBank(precision=precision) as gbk:
        out = gbk.sdft(torch.from_numpy(img).cuda(), sigma, M, half_spectrum=half)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("H,W,M,sigma", [(64, 80, 16, 4.0), (37, 45, 8, 1.5), (5, 70, 16, 4.0),
                                         (100, 3, 4, 0.8), (33, 129, 12, 2.0)])
def test_sdft_fp32_full_parity(torch_cuda, H, W, M, sigma):
    img = synth.pink_noise([3, H, W], H, W)
    got = run_sdft(torch_cuda, img, sigma, M)
    ref = oracle.sdft(img, sigma, M)
    assert got.shape == ref.shape
    e = rel_err(got, ref)
    print("SDFT", H, W, M, "rel err", e)
    assert e <= FP32_TOL


def test_sdft_nonsquare_window(torch_cuda):
    img = synth.pink_noise(4, 48, 72)
    got = run_sdft(torch_cuda, img, 2.0, (8, 16))
    ref = oracle.sdft(img, 2.0, 8, 16)
    assert rel_err(got, ref) <= FP32_TOL
    got = run_sdft(torch_cuda, img, 2.0, (16, 6))
    ref = oracle.sdft(img, 2.0, 16, 6)
    assert rel_err(got, ref) <= FP32_TOL


def test_sdft_half_spectrum_and_conjugate_fill(torch_cuda):
    img = synth.pink_noise(6, 40, 56)
    M = 16
    full = run_sdft(torch_cuda, img, 4.0, M)
    half = run_sdft(torch_cuda, img, 4.0, M, half=True)
    assert half.shape[0] == M // 2 + 1
    assert np.array_equal(half, full[:M // 2 + 1])
    for v in range(M):
        for u in range(M):
            assert np.array_equal(full[(M - v) % M, (M - u) % M], np.conj(full[v, u])) or v in (0, M // 2)


@pytest.fixture(scope="module")
def c3_full():
    """The SDFT workload's image (512 x 512 1/f noise, seed 0) and the FP64 oracle's direct
    windowed DFT of Eq. 17 at every pixel and all 256 bins of the 16 x 16 window, sigma 4."""
    img = synth.pink_noise(0, 512, 512)
    return img, oracle.sdft(img, 4.0, 16)


def test_sdft_c3_full_size_full_oracle(torch_cuda, c3_full):
    img, ref = c3_full
    got = run_sdft(torch_cuda, img, 4.0, 16)
    assert np.all(np.isfinite(got))
    e = rel_err(got, ref)
    print("SDFT 512^2 16x16 FP32 rel err (full oracle)", e)
    assert e <= FP32_TOL


# ---------------------------------------------------------------- tensor-core path

@pytest.mark.parametrize("precision", ["fp16_tc", "bf16_tc"])
@pytest.mark.parametrize("H,W,M,sigma", [(40, 300, 16, 4.0), (7, 129, 8, 1.5), (64, 64, (8, 16), 2.0),
                                         (20, 140, 12, 2.0), (33, 150, (8, 32), 2.5), (45, 131, (32, 8), 2.5)])
def test_sdft_tc_parity(torch_cuda, precision, H, W, M, sigma):
    # 16 x 16, 8 x 8, 8 x 16, 8 x 32 and 32 x 8 run the TMA-fed kernel (the last two only
    # there: their operands exceed shared memory with a staged patch); 12 x 12 the im2col one.
    from tests.helpers import TC_TOL
    img = synth.pink_noise([8, H, W], H, W)
    got = run_sdft(torch_cuda, img, sigma, M, precision=precision)
    My, Mx = (M, M) if isinstance(M, int) else M
    ref = oracle.sdft(img, sigma, My, Mx)
    e = rel_err(got, ref)
    print("TC SDFT", precision, H, W, M, "rel err", e)
    assert e <= TC_TOL


@pytest.mark.parametrize("M", [16, 12])
@pytest.mark.parametrize("gain", [1.0e6, 1.0e4, 1.0e-6])
def test_sdft_tc_scaled_input_and_status(torch_cuda, M, gain):
    # The power-of-two operand scale (per image on the TMA-fed path, M = 16; per tile on the
    # im2col path, M = 12): images far above the FP16 range (1e6) or deep in its subnormals
    # (1e-6) keep the tensor-core bound.
    from paper_1704_05231_gb300 import GaborBank
    from tests.helpers import TC_TOL
    torch = torch_cuda
    img = (synth.pink_noise(12, 33, 200) * gain).astype(np.float32)
    with GaborBank(precision="fp16_tc") as gbk:
        got = gbk.sdft(torch.from_numpy(img).cuda(), 4.0, M).cpu().numpy()
        gbk.device_status()
    ref = oracle.sdft(img, 4.0, M)
    assert rel_err(got, ref) <= TC_TOL


def test_sdft_tc_workspace_growth_and_pitch(torch_cuda):
    # The TMA-fed path's unfolded-image workspace grows with the image and is reused for a
    # smaller one; strided views (pitch 260 > W) read the same pixels as contiguous copies.
    # Every result equals a fresh handle's on the contiguous copy, bitwise, and the half
    # spectrum is the first My/2 + 1 planes of the full one.
    from paper_1704_05231_gb300 import GaborBank
    torch = torch_cuda
    t = torch.from_numpy(synth.pink_noise([51], 150, 260)).cuda()
    shapes = [(40, 70), (150, 260), (33, 129)]
    with GaborBank(precision="fp16_tc") as gbk:
        outs = [gbk.sdft(t[:h, :w], 4.0, 16).cpu().numpy() for h, w in shapes]
        half = gbk.sdft(t[:33, :129], 4.0, 16, half_spectrum=True).cpu().numpy()
        gbk.device_status()
    for (h, w), got in zip(shapes, outs):
        with GaborBank(precision="fp16_tc") as fresh:
            ref = fresh.sdft(t[:h, :w].contiguous(), 4.0, 16).cpu().numpy()
        assert np.array_equal(got, ref)
    assert np.array_equal(half, outs[2][:9])


@pytest.mark.parametrize("precision", ["fp16_tc", "bf16_tc"])
def test_sdft_tc_c3_full_oracle_and_vs_fp32(torch_cuda, c3_full, precision):
    from tests.helpers import TC_TOL
    img, ref = c3_full
    got = run_sdft(torch_cuda, img, 4.0, 16, precision=precision)
    assert np.all(np.isfinite(got))
    e = rel_err(got, ref)
    print("SDFT 512^2 16x16", precision, "rel err (full oracle)", e)
    assert e <= TC_TOL
    f32 = run_sdft(torch_cuda, img, 4.0, 16)
    assert rel_err(got, f32) <= TC_TOL


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("My,Mx", [(16, 4), (12, 6), (4, 16)])
def test_filter_order_non_square_windows(order, My, Mx):
    # Sec. III-B: either pass order gives the same F_{u,v}; the vertical-first order runs on the
    # transposed image.  Both must match the direct windowed DFT.
    import torch
    from paper_1704_05231_gb300 import GaborBank
    img = synth.pink_noise([31, My, Mx], 45, 70)
    with GaborBank() as gbk:
        gbk.set_option("sdft_order", order)
        got = gbk.sdft(torch.from_numpy(img).cuda(), 3.0, (My, Mx)).cpu().numpy()
        mirror = GaborBank(boundary="mirror")
        mirror.set_option("sdft_order", order)
        gm = mirror.sdft(torch.from_numpy(img).cuda(), 3.0, (My, Mx)).cpu().numpy()
        mirror.close()
    assert rel_err(got, oracle.sdft(img, 3.0, My, Mx)) <= FP32_TOL
    assert rel_err(gm, oracle.sdft(img, 3.0, My, Mx, boundary="mirror")) <= FP32_TOL


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("boundary", ["zero", "replicate"])
@pytest.mark.parametrize("H,W,M,sigma", [(64, 80, 16, 4.0), (5, 70, 16, 4.0), (100, 3, 4, 0.8),
                                         (33, 129, 12, 2.0), (40, 50, (8, 16), 2.0), (90, 40, 32, 6.0)])
def test_sdft_forms_match_oracle(torch_cuda, form, boundary, H, W, M, sigma):
    # GB_OPT_SDFT_FORM: 1 the passes step by step (demodulate, smooth, remodulate), 2 one
    # modulated-tap convolution per pass with J_{Mx-u} = J*_u folded into the column sums.
    from paper_1704_05231_gb300 import GaborBank
    img = synth.pink_noise([41, H, W], H, W)
    My, Mx = (M, M) if isinstance(M, int) else M
    with GaborBank(boundary=boundary) as gbk:
        gbk.set_option("sdft_form", form)
        got = gbk.sdft(torch_cuda.from_numpy(img).cuda(), sigma, M).cpu().numpy()
        half = gbk.sdft(torch_cuda.from_numpy(img).cuda(), sigma, M, half_spectrum=True).cpu().numpy()
    ref = oracle.sdft(img, sigma, My, Mx, boundary=boundary)
    assert rel_err(got, ref) <= FP32_TOL
    assert np.array_equal(half, got[:My // 2 + 1])


@pytest.mark.parametrize("order", [1, 2])
def test_sdft_forms_c3_full_oracle_and_order(torch_cuda, c3_full, order):
    from paper_1704_05231_gb300 import GaborBank
    img, ref = c3_full
    res = {}
    for form in (1, 2):
        with GaborBank() as gbk:
            gbk.set_option("sdft_form", form)
            gbk.set_option("sdft_order", order)
            res[form] = gbk.sdft(torch_cuda.from_numpy(img).cuda(), 4.0, 16).cpu().numpy()
    for form in (1, 2):
        assert rel_err(res[form], ref) <= FP32_TOL
    assert rel_err(res[2], res[1]) <= FP32_TOL


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("H,W,M,sigma,half,boundary", [(64, 80, 16, 4.0, False, "zero"),
                                                        (37, 45, (8, 12), 1.5, False, "mirror"),
                                                        (50, 33, (12, 6), 2.0, True, "replicate"),
                                                        (5, 70, 16, 4.0, False, "zero")])
def test_sdft_no_reuse_ablation_matches_oracle(torch_cuda, form, H, W, M, sigma, half, boundary):
    # GB_OPT_SDFT_REUSE = 0: J_u recomputed for every (u, v), F_{Mx-u,v} not taken from J*_u
    # (the paper's comparison without the reuse of Sec. III-B); the same result as the oracle.
    from paper_1704_05231_gb300 import GaborBank
    My, Mx = (M, M) if isinstance(M, int) else M
    img = synth.pink_noise([9, H, W], H, W)
    with GaborBank(boundary=boundary) as gbk:
        gbk.set_option("sdft_form", form)
        gbk.set_option("sdft_reuse", 0)
        got = gbk.sdft(torch_cuda.from_numpy(img).cuda(), sigma, (My, Mx), half_spectrum=half).cpu().numpy()
        gbk.set_option("sdft_reuse", 1)
        again = gbk.sdft(torch_cuda.from_numpy(img).cuda(), sigma, (My, Mx), half_spectrum=half).cpu().numpy()
    ref = oracle.sdft(img, sigma, My, Mx, boundary=boundary)[:got.shape[0]]
    assert rel_err(got, ref) <= FP32_TOL
    assert rel_err(again, ref) <= FP32_TOL


def test_sdft_no_reuse_c3_full_oracle(torch_cuda, c3_full):
    from paper_1704_05231_gb300 import GaborBank
    img, ref = c3_full
    with GaborBank() as gbk:
        gbk.set_option("sdft_reuse", 0)
        got = gbk.sdft(torch_cuda.from_numpy(img).cuda(), 4.0, 16).cpu().numpy()
    assert rel_err(got, ref) <= FP32_TOL


def test_store_probe_writes_every_output(torch_cuda):
    # The store-pattern probe (the tensor-core SDFT's output stream without arithmetic) writes
    # every element of its plane-major output exactly: out[p][y][x] = (p + 1, x + 1).
    import torch
    from paper_1704_05231_gb300 import GBError
    from paper_1704_05231_gb300.bank import store_probe
    nplanes, H, W = 19, 37, 256
    out = torch.full((nplanes, H, W), float("nan"), dtype=torch.complex64, device="cuda")
    store_probe(out, ctas=5)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = (np.arange(1, nplanes + 1, dtype=np.float32)[:, None, None]
            + 1j * np.arange(1, W + 1, dtype=np.float32)[None, None, :]) * np.ones((1, H, 1), np.float32)
    assert np.array_equal(got, want.astype(np.complex64))
    with pytest.raises(GBError):
        store_probe(torch.empty((2, 4, 100), dtype=torch.complex64, device="cuda"))
