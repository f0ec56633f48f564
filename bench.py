#!/usr/bin/env python
"""Benchmark of the GB300 Gabor filter bank (arXiv 1704.05231, Algorithm 1).

Workload (default): the paper-size bank - one 1024 x 1024 FP32 image (1/f^2 noise plus eight
oriented sinusoids, seed 0), 6 orientations k pi / 6 x 4 frequencies pi/2 .. pi/16 with
sigma = pi / omega and radius 3 sigma, complex64 outputs: 24 pixel-filter outputs per pixel.
A step is one call of the bank on that image (every row of the hot path: tables are built
before timing; horizontal pass, orientation reuse, vertical pass and stores inside).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead, on a
bounded pixel sample of the same workload.  Multi-GPU runs are independent replicas (weak
scaling): the bank has no exchange step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gabor bank pixel·filter outputs/s, plain vs TC at ≤2e-3 rel err; serve p99 ms"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_gabor_fp32 launch on this
# workload from an ncu capture of the current kernel; None once the kernel changes.
K_GABOR_FP32_TRAFFIC = 143858176   # 4390656 read + 139467520 written (autotuned k_gabor_fp32<0, 1, 8, 1>, one ncu pass)
UNIT = "outputs/s"
H = W = 1024


def workload():
    from paper_1704_05231_gb300 import synth
    thetas = [k * math.pi / 6 for k in range(6)]
    omegas = [math.pi / 2, math.pi / 4, math.pi / 8, math.pi / 16]
    sigmas = [math.pi / w for w in omegas]
    img = synth.paper_like(0, H, W)
    return img, thetas, omegas, sigmas


def workload_config(extra=None):
    cfg = {"workload": "paper-size Gabor bank: 1024x1024 FP32 1/f^2 noise + 8 sinusoids (seed 0), "
                       "6 orientations k*pi/6 x 4 frequencies pi/2..pi/16, sigma=pi/omega, radius 3 sigma, "
                       "complex64 out",
           "H": H, "W": W, "n_theta": 6, "n_freq": 4, "outputs_per_step": 24 * H * W,
           "l2": "flushed between steps (256 MiB write); output 201 MB > L2"}
    if extra:
        cfg.update(extra)
    return cfg


def radius(sigma, rf=3.0):
    return int(math.ceil(rf * sigma - 1e-9))


def algorithmic_flops(thetas, omegas, sigmas, Hh=H, Ww=W):
    """FLOPs of the decomposition (FIR form): per pixel and frequency (3N+1) T FMAs."""
    n = len(thetas)
    fma = sum((3 * n + 1) * (2 * radius(s) + 1) for s in sigmas) * Hh * Ww
    return 2.0 * fma


def fp32_nominal_tflops(torch):
    """Nominal FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP x max SM clock."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


_FP32_PEAK = None


def fp32_peak_tflops(torch):
    """Measured FP32 CUDA-core peak (the library's FMA probe, best of scalar and packed FMA),
    and a note with the nominal figure beside it."""
    global _FP32_PEAK
    if _FP32_PEAK is None:
        from paper_1704_05231_gb300.bank import fp32_fma_peak
        m = fp32_fma_peak()
        nom, sms, mhz = fp32_nominal_tflops(torch)
        _FP32_PEAK = (m["peak"], f"FMA probe: scalar {m['scalar']:.1f}, packed {m['packed']:.1f} TFLOP/s; "
                                 f"nominal {nom:.1f} ({sms} SMs, {mhz:.0f} MHz)")
    return _FP32_PEAK


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml, read-only queries)
    every `period_s` from a host thread during the timed region, plus once at its start and
    end, so that even a region of a few milliseconds has samples."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, torch, dev, period_s=0.002):
        import ctypes
        import threading
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        uuid = ("GPU-" + str(torch.cuda.get_device_properties(dev).uuid)).encode()
        if self.lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(uuid), ctypes.byref(self.h)) != 0:
            raise RuntimeError("NVML handle not found")
        self.reason_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.period = period_s
        self.samples = []
        self.stop_ev = threading.Event()
        self.thread = threading.Thread(target=self._loop, daemon=True)

    def _sample(self):
        c, r = self.ct.c_uint(), self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(c)) == 0 and \
                self.reason_fn(self.h, self.ct.byref(r)) == 0:
            self.samples.append((c.value, r.value))

    def _loop(self):
        while not self.stop_ev.is_set():
            self._sample()
            self.stop_ev.wait(self.period)

    def start(self):
        self._sample()
        self.thread.start()

    def stop(self):
        self.stop_ev.set()
        self.thread.join()
        self._sample()
        mx = self.ct.c_uint()
        sm_max = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.ct.byref(mx)) == 0 else None
        sm = [c for c, _ in self.samples]
        reasons = sorted({n for _, r in self.samples for bit, n in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": sm_max, "reasons": reasons,
                "samples": len(self.samples), "source": "nvml"}


def clock_sampler(torch, dev):
    try:
        return NvmlClockSampler(torch, dev)
    except Exception:
        return ClockSampler(dev)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _oracle_rate(img, thetas, omegas, sigmas, seconds, threads, seed):
    """Outputs/s of the FP64 oracle on random pixels of the image, for about `seconds`."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    n_px = 0
    t0 = time.perf_counter()
    while True:
        xs = rng.integers(0, W, 256).astype(np.int32)
        ys = rng.integers(0, H, 256).astype(np.int32)
        oracle.gabor_bank(img, thetas, omegas, sigmas, points=(xs, ys), threads=threads)
        n_px += 256
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return n_px * len(thetas) * len(omegas) / el, n_px, el


def cpu_baseline(img, thetas, omegas, sigmas, seconds):
    """The FP64 oracle as it stands, on a time-boxed random pixel sample: all host cores, and
    one core for a fifth of the time."""
    cores = os.cpu_count() or 1
    v, n_px, el = _oracle_rate(img, thetas, omegas, sigmas, seconds, cores, 123)
    v1, n1, el1 = _oracle_rate(img, thetas, omegas, sigmas, max(1.0, seconds / 5), 1, 124)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_px} random pixels x {len(thetas) * len(omegas)} filters of the 1024x1024 "
                      f"bank (direct FP64 sums), {el:.1f} s",
            "one_core": {"value": v1, "sample": f"{n1} px, {el1:.1f} s"}}


def run_reference(args):
    """--impl reference: the FP64 oracle on bounded samples, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    img, thetas, omegas, sigmas = workload()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(321)
    per_step = 256

    def step():
        xs = rng.integers(0, W, per_step).astype(np.int32)
        ys = rng.integers(0, H, per_step).astype(np.int32)
        oracle.gabor_bank(img, thetas, omegas, sigmas, points=(xs, ys), threads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    nout = per_step * len(thetas) * len(omegas)
    value = nout * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config({"sample_per_step": f"{per_step} random pixels x 24 filters"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} random pixels x 24 filters per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class nvtx_range:
    """An NVTX push/pop range around a leg's warm-up and timed steps, so that a profiler can
    select the launches of one leg (`ncu --nvtx --nvtx-include "<name>/"`); a no-op where
    torch has no NVTX."""

    def __init__(self, torch, name):
        self.nvtx = getattr(torch.cuda, "nvtx", None) if name else None
        self.name = name

    def __enter__(self):
        if self.nvtx is not None:
            try:
                self.nvtx.range_push(self.name)
            except Exception:
                self.nvtx = None
        return self

    def __exit__(self, *exc):
        if self.nvtx is not None:
            self.nvtx.range_pop()
        return False


def time_device(torch, fn, steps, warmup, flush, stream, name=None):
    """CUDA-event time of fn() per step (ms), L2 flushed before each step, after warm-up."""
    with nvtx_range(torch, name):
        for _ in range(max(3, warmup)):
            fn()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for k in range(steps):
            if flush is not None:
                flush.zero_()
            starts[k].record(stream)
            fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def c1_leg(torch, steps, warmup, stream):
    """The smallest bank (256 x 256 uniform image, seed 0; 4 orientations x 2 frequencies,
    sigma 4, radius 12): latency-bound, working set inside L2, so no flush between steps.
    Timed per call and as a replayed one-call CUDA graph (no host launch cost)."""
    from paper_1704_05231_gb300 import GaborBank, synth
    from paper_1704_05231_gb300.bank import capture_graph
    Hc = Wc = 256
    img = torch.from_numpy(synth.uniform01(0, Hc, Wc)).cuda()
    th = [0.0, math.pi / 4, math.pi / 2, 3 * math.pi / 4]
    om = [math.pi / 4, math.pi / 8]
    n_out = len(th) * len(om) * Hc * Wc
    res = {"workload": "256x256 uniform [0,1) (seed 0), 4 orientations x 2 frequencies, sigma 4, radius 12; "
                       "L2-resident, latency-bound", "outputs_per_step": n_out}
    for prec in ("fp32", "fp16_tc"):
        gbk = GaborBank(th, om, [4.0, 4.0], precision=prec, max_shape=(Hc, Wc))
        out = torch.empty(gbk.out_shape(Hc, Wc), dtype=torch.complex64, device="cuda")
        ms = statistics.median(time_device(torch, lambda: gbk.filter(img, out), max(steps, 50), warmup, None,
                                           stream))
        graph = capture_graph(lambda: gbk.filter(img, out))
        gms = statistics.median(time_device(torch, graph.replay, max(steps, 50), warmup, None, stream))
        gbk.device_status()
        res[prec] = {"us": ms * 1e3, "graph_us": gms * 1e3, "value": n_out / (gms * 1e-3), "unit": UNIT}
        del graph
        gbk.close()
    return res


def bank_tc_leg(torch, d_img, thetas, omegas, sigmas, ref_out, n_out, steps, warmup, flush, stream):
    """The same bank on tensor cores (FP16 operands, and BF16 operands as hi + lo pairs; FP32
    accumulation): outputs/s, rel. error against the FP32 path on this image, HBM roofline of
    the whole step."""
    from paper_1704_05231_gb300 import GaborBank
    peak, kind = hbm_peak_gbs()
    res = {}
    ref = ref_out.clone()
    for prec in ("fp16_tc", "bf16_tc"):
        try:
            gbk = GaborBank(thetas, omegas, sigmas, precision=prec, max_shape=(H, W))
            from paper_1704_05231_gb300.tune import autotune
            tiles = autotune(gbk, d_img, steps=3)["tc_tiles"]
            out = torch.empty_like(ref)
            ms = statistics.mean(time_device(torch, lambda: gbk.filter(d_img, out), steps, warmup, flush, stream,
                                             name=prec))
            gbk.device_status()
            bytes_ = n_out * 8 + H * W * 4
            res[prec] = {"value": n_out / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "tc_tiles": tiles,
                         "rel_err_vs_fp32": float((out - ref).abs().max() / ref.abs().max()),
                         "roofline": {"bound": "hbm", "achieved": bytes_ / (ms * 1e-3) / 1e9, "peak": peak,
                                      "unit": "GB/s", "frac": bytes_ / (ms * 1e-3) / 1e9 / peak,
                                      "peak_kind": kind, "algorithmic_bytes": bytes_}}
            gbk.close()
        except Exception as exc:  # reported, not hidden
            res[prec] = {"error": str(exc)}
    return res


def sdft_leg(torch, steps, warmup, flush, stream):
    """Localized SDFT, 512 x 512 1/f noise, 16 x 16 window, sigma 4, all 256 bins: FP32
    separable path (Algorithm 2) and the tensor-core windowed-DFT contraction."""
    from paper_1704_05231_gb300 import GaborBank, synth
    Hs = Ws = 512
    img = torch.from_numpy(synth.pink_noise(0, Hs, Ws)).cuda()
    n_out = 256 * Hs * Ws
    bytes_ = n_out * 8 + Hs * Ws * 4
    peak, kind = hbm_peak_gbs()
    res = {"workload": "512x512 1/f noise (seed 0), 16x16 window, sigma 4, 256 bins, complex64 out",
           "outputs_per_step": n_out}
    # write bandwidth of the same output volume, for context: a zero fill (torch; faster than
    # the memory's raw rate through zero compression) and the library's store probe (the
    # tensor-core SDFT's own store pattern and CTA shape, non-zero values, no arithmetic): the
    # ceiling of that pattern
    from paper_1704_05231_gb300.bank import store_probe
    fill = torch.empty((16, 16, Hs, Ws), dtype=torch.complex64, device="cuda")
    fms = statistics.mean(time_device(torch, lambda: fill.zero_(), steps, warmup, flush, stream))
    res["fill_same_bytes"] = {"ms": fms, "GB/s": n_out * 8 / (fms * 1e-3) / 1e9, "values": "zeros"}
    pv = fill.view(256, Hs, Ws)
    pms = statistics.mean(time_device(torch, lambda: store_probe(pv), steps, warmup, flush, stream))
    res["store_pattern"] = {"ms": pms, "GB/s": n_out * 8 / (pms * 1e-3) / 1e9,
                            "frac_of_peak": n_out * 8 / (pms * 1e-3) / 1e9 / peak,
                            "note": "the TC SDFT's output stream alone: 16 storing warps, one CTA per SM, non-zero values"}
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    p2 = statistics.mean(time_device(torch, lambda: store_probe(pv, ctas=2 * nsm), steps, warmup, flush, stream))
    res["store_pattern"]["two_ctas_per_sm_GB/s"] = n_out * 8 / (p2 * 1e-3) / 1e9
    del fill, pv
    ref = None
    for prec in ("fp32", "fp16_tc", "bf16_tc"):
        gbk = GaborBank(precision=prec)
        out = torch.empty((16, 16, Hs, Ws), dtype=torch.complex64, device="cuda")
        ms = statistics.mean(time_device(torch, lambda: gbk.sdft(img, 4.0, 16, out=out), steps, warmup, flush, stream,
                                         name="sdft_" + prec))
        gbk.device_status()
        ent = {"value": n_out / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
               "roofline": {"bound": "hbm", "achieved": bytes_ / (ms * 1e-3) / 1e9, "peak": peak,
                            "unit": "GB/s", "frac": bytes_ / (ms * 1e-3) / 1e9 / peak, "peak_kind": kind,
                            "algorithmic_bytes": bytes_}}
        if ref is None:
            ref = out.clone()
        else:
            ent["rel_err_vs_fp32"] = float((out - ref).abs().max() / ref.abs().max())
            ent["frac_of_store_pattern"] = pms / ms
        res[prec] = ent
        gbk.close()
        del out
    # Reuse of Sec. III-B (J_u once per u for every v, F_{Mx-u,v} from J*_u) on and off: the
    # GPU analogue of the paper's SDFT reuse gain (Table III), FP32 path
    ent = {}
    for reuse in (1, 0):
        gbk = GaborBank(precision="fp32")
        gbk.set_option("sdft_reuse", reuse)
        out = torch.empty((16, 16, Hs, Ws), dtype=torch.complex64, device="cuda")
        ms = statistics.mean(time_device(torch, lambda: gbk.sdft(img, 4.0, 16, out=out), steps, warmup, flush, stream))
        ent["reuse" if reuse else "no_reuse"] = {"ms_per_step": ms, "value": n_out / (ms * 1e-3)}
        gbk.close()
        del out
    ent["speedup_from_reuse"] = ent["no_reuse"]["ms_per_step"] / ent["reuse"]["ms_per_step"]
    res["reuse"] = ent
    # Non-square windows (My x Mx, same 256 bins): the FP32 kernel always runs the horizontal
    # pass first; its FMA count differs by window orientation, its output bytes do not.
    from paper_1704_05231_gb300 import GBError
    for (My, Mx) in ((8, 32), (32, 8)):
        # FP32: both pass orders (Sec. III-B filter order) and the automatic choice
        for prec, order in (("fp32", 1), ("fp32", 2), ("fp32", 0), ("fp16_tc", 0)):
            gbk = GaborBank(precision=prec)
            gbk.set_option("sdft_order", order)
            out = torch.empty((My, Mx, Hs, Ws), dtype=torch.complex64, device="cuda")
            key = f"{prec}_{My}x{Mx}" + {0: "_auto", 1: "_horizontal_first", 2: "_vertical_first"}[order]
            try:
                ms = statistics.mean(time_device(torch, lambda: gbk.sdft(img, 4.0, (My, Mx), out=out), steps,
                                                 warmup, flush, stream))
                res[key] = {"ms_per_step": ms, "value": n_out / (ms * 1e-3),
                            "hbm_frac": bytes_ / (ms * 1e-3) / 1e9 / peak}
            except GBError as exc:   # reported, not hidden
                res[key] = {"unsupported": str(exc)}
            gbk.close()
            del out
    return res


def ablation_leg(torch, d_img, thetas, omegas, sigmas, steps, warmup, flush, stream):
    """Orientation reuse on and off (J_{pi-theta} = J*_theta, Eq. 13-16): the GPU analogue of
    the paper's reuse speed-up, FP32 and FP16-TC, same image and bank as the main line."""
    from paper_1704_05231_gb300 import GaborBank
    res = {}
    for prec in ("fp32", "fp16_tc"):
        gbk = GaborBank(thetas, omegas, sigmas, precision=prec, max_shape=(H, W))
        out = torch.empty(gbk.out_shape(H, W), dtype=torch.complex64, device="cuda")
        ent = {}
        for reuse in (1, 0):
            gbk.set_option("reuse", reuse)
            ms = statistics.mean(time_device(torch, lambda: gbk.filter(d_img, out), steps, warmup, flush, stream))
            ent["reuse" if reuse else "no_reuse"] = {"ms_per_step": ms, "value": len(thetas) * len(omegas) * H * W / (ms * 1e-3)}
        ent["speedup_from_reuse"] = ent["no_reuse"]["ms_per_step"] / ent["reuse"]["ms_per_step"]
        gbk.close()
        res[prec] = ent
    return res


def iir_leg(torch, d_img, thetas, omegas, sigmas, fir_out, steps, warmup, flush, stream):
    """The recursive-Gaussian bank (Young-van Vliet, the paper's own smoother; cost per output
    independent of sigma) on the paper-size bank and on the 64-image batch: time, outputs/s and
    the SER of Sec. IV-C of each frequency's outputs against the exact FIR bank on the GPU."""
    from paper_1704_05231_gb300 import GaborBank, synth
    res = {}
    gbk = GaborBank(thetas, omegas, sigmas, smoother="iir", max_shape=(H, W))
    out = torch.empty(gbk.out_shape(H, W), dtype=torch.complex64, device="cuda")
    ms = statistics.mean(time_device(torch, lambda: gbk.filter(d_img, out), steps, warmup, flush, stream,
                                     name="iir_bank"))
    n_out = len(thetas) * len(omegas) * H * W
    ser = []
    for s in range(len(omegas)):
        f, t = out[s], fir_out[s]
        ser.append([10 * math.log10(float((part(f) ** 2).sum() / ((part(f) - part(t)) ** 2).sum()))
                    for part in (torch.real, torch.imag)])
    res["paper_bank"] = {"ms_per_step": ms, "value": n_out / (ms * 1e-3), "unit": UNIT,
                         "ser_db_re_im_per_frequency": ser}
    gbk.close()
    del out
    shapes = synth.batch_shapes(1, 64, 128, 2048)
    imgs = [synth.pink_noise_device(1000 + i, h, w) for i, (h, w) in enumerate(shapes)]
    th, om, sg = synth.octave_bank(8, 5)
    gbk = GaborBank(th, om, sg, smoother="iir", max_shape=(2048, 2048))
    outs = [torch.empty(gbk.out_shape(h, w), dtype=torch.complex64, device="cuda") for h, w in shapes]
    ms = statistics.mean(time_device(torch, lambda: gbk.filter_batch(imgs, outs), min(steps, 3), 3, flush, stream,
                                     name="iir_batch"))
    n_out = sum(len(th) * len(om) * h * w for h, w in shapes)
    res["batch_64"] = {"ms_per_step": ms, "value": n_out / (ms * 1e-3), "unit": UNIT, "launches_per_step": 2 * len(shapes)}
    gbk.close()
    del outs, imgs
    torch.cuda.empty_cache()
    return res


def batch_leg(torch, steps, warmup, flush, stream):
    """64 uneven 1/f-noise images (sides uniform in [128, 2048], seed 1), 8 orientations x 5
    octave frequencies (sigma = pi/omega, R up to 96): one persistent launch per step for FP32
    (tile geometry from the autotuner), replayed from a captured CUDA graph; the FP16-TC bank
    takes four launches per step for all 64 images (min / max, F[1] tables, row pass, column
    pass), in the same kind of graph."""
    from paper_1704_05231_gb300 import GaborBank, synth
    from paper_1704_05231_gb300.bank import capture_graph
    from paper_1704_05231_gb300.tune import autotune
    shapes = synth.batch_shapes(1, 64, 128, 2048)
    imgs = [synth.pink_noise_device(1000 + i, h, w) for i, (h, w) in enumerate(shapes)]
    th, om, sg = synth.octave_bank(8, 5)
    n_out = sum(len(th) * len(om) * h * w for h, w in shapes)
    flops = sum(algorithmic_flops(th, om, sg, h, w) for h, w in shapes)
    res = {"workload": "64 images, sides U[128,2048] (seed 1), 1/f noise made on the device; 8 orientations "
                       "k*pi/8 x 5 frequencies pi/2..pi/32, sigma=pi/omega",
           "outputs_per_step": n_out, "pixels": sum(h * w for h, w in shapes)}
    peak_hbm, kind = hbm_peak_gbs()
    peak_alu, _ = fp32_peak_tflops(torch)
    for prec in ("fp32", "fp16_tc", "bf16_tc"):
        gbk = GaborBank(th, om, sg, precision=prec, max_shape=(2048, 2048))
        outs = [torch.empty(gbk.out_shape(h, w), dtype=torch.complex64, device="cuda") for h, w in shapes]
        ent = {}
        if prec == "fp32":
            t = autotune(gbk, imgs, steps=1, tile_rows=(0,), segments=(0, 1, 2, 4))
            ent["tiling"], ent["ctas_per_sm"] = t["tiling"], t["ctas"]
        else:
            ent["tc_tiles"] = autotune(gbk, imgs, steps=1)["tc_tiles"]
        graph = capture_graph(lambda: gbk.filter_batch(imgs, outs))
        ms = statistics.mean(time_device(torch, graph.replay, steps, warmup, flush, stream))
        gbk.device_status()
        ent.update({"value": n_out / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                    "launches_per_step": 1 if prec == "fp32" else 4})
        if prec == "fp32":
            a = flops / (ms * 1e-3) / 1e12
            ent["roofline"] = {"bound": "alu", "achieved": a, "peak": peak_alu, "unit": "TFLOP/s", "frac": a / peak_alu}
        else:
            b = n_out * 8 + res["pixels"] * 4
            a = b / (ms * 1e-3) / 1e9
            ent["roofline"] = {"bound": "hbm", "achieved": a, "peak": peak_hbm, "unit": "GB/s", "frac": a / peak_hbm,
                               "peak_kind": kind}
        res[prec] = ent
        del graph, outs
        gbk.close()
        torch.cuda.empty_cache()
    return res


def serve_leg(args):
    """Served stream: Poisson arrivals at 0.7x the closed-loop saturation rate, 256-4096 px
    sides, 90% banks / 10% 16x16 SDFT, 96 GiB budget, 4 slots (continuous batching)."""
    from paper_1704_05231_gb300 import serve
    pool = serve.ImagePool(n=4, side=4096, seed=3)
    res = {"workload": f"{args.serve_warm} warm-up + {args.serve_n} measured requests (seed 2), sides log-U[256,4096], "
                       "banks N~U{4..8} x S~U{2..5} octaves sigma=pi/omega, 10% SDFT M=16 sigma=4; images are "
                       "crops of device-resident 4096^2 1/f noise; outputs stay in device memory",
           "budget_gib": 96, "slots": 4}
    for prec in ("fp32", "fp16_tc"):
        r = serve.measure(prec, n_warm=args.serve_warm, n_meas=args.serve_n, rate_fracs=(0.7, 0.5, 0.9), pool=pool,
                          n_sat=min(300, args.serve_n), log=lambda m: print(m, file=sys.stderr, flush=True))
        ent = {"saturation_req_s": r["saturation_req_s"]}
        for frac, s in r["rates"].items():
            ent[f"{frac:.1f}x"] = {"rate_req_s": s["rate_req_s"], "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"],
                                   "outputs_per_s": s["outputs_per_s"], "served": s["served"],
                                   "rejected": s["rejected"]}
        ent.update({k: ent["0.7x"][k] for k in ("p50_ms", "p99_ms", "outputs_per_s")})
        res[prec] = ent
    return res


LEG_KEYS = ("c1", "tc", "sdft", "ablation", "batch", "iir", "serve")


def _r(x, nd=4):
    """x rounded to nd significant digits (None and non-numbers unchanged)."""
    if isinstance(x, bool) or not isinstance(x, (int, float)) or x == 0 or x != x:
        return x
    return float(f"{x:.{nd}g}")


def _g(x):
    """outputs/s in units of 1e9."""
    return _r(x / 1e9) if isinstance(x, (int, float)) else x


def _get(d, *path):
    for p in path:
        if not isinstance(d, dict) or p not in d:
            return None
        d = d[p]
    return d


def leg_summary(line):
    """One short entry per leg: times in ms (us where named), rates in 1e9 outputs/s (gout_s),
    fractions of the stated roof."""
    out = {}
    c1 = line.get("c1")
    if c1:
        for p in ("fp32", "fp16_tc"):
            if p in c1:
                out[f"c1_256_{p}"] = {"us": _r(c1[p]["us"]), "graph_us": _r(c1[p]["graph_us"]),
                                      "gout_s": _g(c1[p]["value"])}
    tc = line.get("tc")
    if tc:
        for p, e in tc.items():
            if "error" in e:
                out[f"bank_{p}"] = {"error": e["error"][:80]}
            else:
                out[f"bank_{p}"] = {"ms": _r(e["ms_per_step"]), "gout_s": _g(e["value"]),
                                    "hbm_frac": _r(e["roofline"]["frac"], 3), "err_vs_fp32": _r(e["rel_err_vs_fp32"], 3)}
    sd = line.get("sdft")
    if sd:
        for p in ("fp32", "fp16_tc", "bf16_tc"):
            if p in sd:
                e = sd[p]
                out[f"sdft512_m16_{p}"] = {"ms": _r(e["ms_per_step"]), "gout_s": _g(e["value"]),
                                           "hbm_frac": _r(e["roofline"]["frac"], 3)}
        if "reuse" in sd:
            out["sdft_reuse_speedup"] = _r(sd["reuse"]["speedup_from_reuse"], 3)
        if "fill_same_bytes" in sd:
            out["sdft_zero_fill_gbs"] = _r(sd["fill_same_bytes"]["GB/s"])
        if "store_pattern" in sd:
            out["sdft_store_pattern_gbs"] = _r(sd["store_pattern"]["GB/s"])
            if "fp16_tc" in sd:
                out["sdft512_m16_fp16_tc"]["frac_of_store_pattern"] = _r(sd["fp16_tc"]["frac_of_store_pattern"], 3)
    ab = line.get("ablation")
    if ab:
        out["bank_reuse_speedup"] = {p: _r(e["speedup_from_reuse"], 3) for p, e in ab.items()}
    bt = line.get("batch")
    if bt:
        for p in ("fp32", "fp16_tc", "bf16_tc"):
            e = bt.get(p)
            if e:
                out[f"batch64_{p}"] = {"ms": _r(e["ms_per_step"]), "gout_s": _g(e["value"]),
                                       "launches": e.get("launches_per_step"),
                                       "frac": _r(_get(e, "roofline", "frac"), 3),
                                       "bound": _get(e, "roofline", "bound")}
    ir = line.get("iir")
    if ir:
        out["iir"] = {"bank_ms": _r(_get(ir, "paper_bank", "ms_per_step")),
                      "batch64_ms": _r(_get(ir, "batch_64", "ms_per_step"))}
    sv = line.get("serve")
    if sv:
        for p in ("fp32", "fp16_tc"):
            e = sv.get(p)
            if e:
                out[f"serve_{p}"] = {"p50_ms": _r(e["p50_ms"]), "p99_ms": _r(e["p99_ms"]),
                                     "gout_s": _g(e["outputs_per_s"]), "sat_req_s": _r(e["saturation_req_s"]),
                                     "p99_ms_0.9x": _r(_get(e, "0.9x", "p99_ms"))}
    return out


def compact_line(line):
    """The stdout JSON line: every contract key, legs replaced by their summary."""
    c = {k: v for k, v in line.items() if k not in LEG_KEYS}
    if "roofline" in c:
        c["roofline"] = {k: (_r(v) if isinstance(v, float) else v) for k, v in c["roofline"].items()}
    legs = leg_summary(line)
    if legs:
        c["legs"] = legs
    return c


def max_over_ranks(ms, dist, device):
    """The slowest rank's step time (ms): every replica runs the same work, so the job's
    step ends when the last one does."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(n_out_per_rank, world, ms):
    """Whole-job outputs/s: every rank filters its own image (weak scaling, no exchange)."""
    return n_out_per_rank * world / (ms * 1e-3)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1704_05231_gb300 import GaborBank

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    img, thetas, omegas, sigmas = workload()
    n_out = len(thetas) * len(omegas) * H * W
    gbk = GaborBank(thetas, omegas, sigmas, precision="fp32", max_shape=(H, W))
    d_img = torch.from_numpy(img).cuda()
    out = torch.empty(gbk.out_shape(H, W), dtype=torch.complex64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    tiling, ctas = None, 1
    if not args.no_tune:
        from paper_1704_05231_gb300.tune import autotune
        tuned = autotune(gbk, d_img, steps=3)
        tiling, ctas = tuned["tiling"], tuned["ctas"]
    headline = nvtx_range(torch, "fp32_bank").__enter__()
    for _ in range(max(3, args.warmup)):
        gbk.filter(d_img, out)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = clock_sampler(torch, local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        gbk.filter(d_img, out)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    headline.__exit__()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = statistics.mean(step_ms)
    ms = max_over_ranks(ms, dist, "cuda")
    value = replica_throughput(n_out, world, ms)

    # End to end through the C ABI on host buffers (pinned): H2D image, bank, D2H result.
    e2e_s = float("nan")
    if not args.no_e2e:
        h_img = torch.from_numpy(img).pin_memory()
        h_out = torch.empty(gbk.out_shape(H, W), dtype=torch.complex64).pin_memory()
        gbk.filter_host_ptr(h_img.data_ptr(), H, W, W, h_out.data_ptr())
        e2e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(e2e_steps):
            gbk.filter_host_ptr(h_img.data_ptr(), H, W, W, h_out.data_ptr())
        e2e_s = (time.perf_counter() - t1) / e2e_steps
        # the copy ceiling: the same host<->device bytes as plain pinned copies, no compute
        d_out_c = torch.empty_like(out)
        copy_stream = torch.cuda.current_stream()
        for _ in range(2):
            d_img.copy_(h_img, non_blocking=True)
            h_out.copy_(d_out_c, non_blocking=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for _ in range(e2e_steps):
            d_img.copy_(h_img, non_blocking=True)
            h_out.copy_(d_out_c, non_blocking=True)
            copy_stream.synchronize()
        copy_s = (time.perf_counter() - t2) / e2e_steps
        del d_out_c

    flops = algorithmic_flops(thetas, omegas, sigmas)
    peak, peak_note = fp32_peak_tflops(torch)
    achieved = flops / (ms * 1e-3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"path": "FP32 CUDA-core fused bank kernel", "parallelism": f"replicas x{world}",
                                       "tiling": tiling, "ctas_per_sm": ctas}),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": K_GABOR_FP32_TRAFFIC,
                         "kernel": "k_gabor_fp32 (one persistent launch per step)",
                         "peak_note": peak_note,
                         "algorithmic": "(3N+1)(2R+1) FMA per pixel per frequency"},
            "e2e": None if args.no_e2e else {
                "value": n_out / e2e_s, "unit": UNIT, "h2d_bytes_per_step": H * W * 4,
                "d2h_bytes_per_step": n_out * 8, "ms": e2e_s * 1e3,
                "path": "gabor_bank_filter_host, pinned buffers (per-frequency launches, D2H overlapped)",
                "copy_ceiling": {"ms": copy_s * 1e3, "value": n_out / copy_s,
                                 "d2h_gb_s": n_out * 8 / copy_s / 1e9,
                                 "note": "the same H2D + D2H bytes as plain pinned copies, no compute"},
                "frac_of_copy_ceiling": copy_s / e2e_s},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "wall_s": wall}
    legs = set() if args.no_extra else set(args.legs.split(","))
    if "c1" in legs:
        line["c1"] = c1_leg(torch, args.steps, args.warmup, stream)
    if "tc" in legs:
        line["tc"] = bank_tc_leg(torch, d_img, thetas, omegas, sigmas, out, n_out, args.steps, args.warmup, flush,
                                 stream)
    if "sdft" in legs:
        line["sdft"] = sdft_leg(torch, args.steps, args.warmup, flush, stream)
    if "ablation" in legs:
        line["ablation"] = ablation_leg(torch, d_img, thetas, omegas, sigmas, args.steps, args.warmup, flush, stream)
    if "batch" in legs:
        line["batch"] = batch_leg(torch, min(args.steps, 5), 3, flush, stream)
    if "iir" in legs:
        line["iir"] = iir_leg(torch, d_img, thetas, omegas, sigmas, out, args.steps, args.warmup, flush, stream)
    if "serve" in legs and not args.no_serve and world == 1:
        line["serve"] = serve_leg(args)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(img, thetas, omegas, sigmas, args.cpu_seconds)
    if rank == 0:
        # every leg in full on stderr; the stdout line keeps the headline and one compact
        # summary per leg, short enough to survive a log tail of a few kilobytes
        for k in LEG_KEYS:
            if k in line:
                print("leg " + json.dumps({k: line[k]}), file=sys.stderr, flush=True)
        print(json.dumps(compact_line(line)), flush=True)
    gbk.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-extra", action="store_true", help="skip every extra leg (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true", help="default tile geometry instead of the autotuner's")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream leg")
    ap.add_argument("--legs", default="c1,tc,sdft,ablation,batch,iir,serve",
                    help="comma list of extra legs: c1, tc, sdft, ablation, batch, iir, serve")
    ap.add_argument("--serve-n", type=int, default=2000, help="measured requests of the served stream")
    ap.add_argument("--serve-warm", type=int, default=200)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
