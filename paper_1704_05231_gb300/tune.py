"""Autotuner for the tile geometry of the filter-bank kernels.

FP32 handles: for every frequency of a plan it picks the rows per streamed chunk (TH) and the
number of row segments per column strip, and for the whole plan the CTAs per SM (one of 16
warps or two of 8), by timing the whole bank on the caller's images (coordinate descent over
the frequencies for each CTA setting, CUDA events, L2 flushed between timings).  The choice
trades the 2R-row vertical halo recomputed per segment against load balance across the SMs.
Tensor-core handles: the rows per row-pass item and per column-pass job of the modulated-tap
kernels (32 or 64 each, GB_OPT_TC_TILES), timed the same way.  No choice changes any result
(every output's arithmetic is the same).  Choices are cached in a JSON file keyed by GPU name,
image-size classes, radii, orientation count and precision.
"""
from __future__ import annotations

import json
import math
import os
import statistics

TILE_ROWS = (0, 32, 64)
SEGMENTS = (0, 1, 2, 4, 8)
CTAS = (1, 2)
TC_TILES = ((64, 64), (32, 64), (64, 32), (32, 32))   # (row-pass rows, column-pass rows)


def default_cache_path():
    return os.environ.get("GABORBANK_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gaborbank_tune.json"))


def size_class(n):
    return 1 << max(0, int(n - 1).bit_length())


def cache_key(gbk, shapes, gpu_name):
    radii = [int(math.ceil(3.0 * s - 1e-9)) for s in gbk.sigmas]
    classes = sorted({(size_class(h), size_class(w)) for h, w in shapes})
    return f"{gpu_name}|{classes}|R={radii}|N={len(gbk.thetas)}|{gbk.precision}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(gbk, imgs, cache_path=None, steps=3, use_cache=True, tile_rows=TILE_ROWS, segments=SEGMENTS,
             ctas=CTAS):
    """Choose the tile geometry for `imgs` (a CUDA tensor or a list of them).

    FP32 handles: (tile_rows, segments) per frequency and the CTAs per SM; returns {"key",
    "tiling": [[tile_rows, segments], ...], "ctas", "ms"} (`tile_rows`, `segments` and `ctas`
    are the candidate values searched).  Tensor-core handles: the modulated-tap tile rows;
    returns {"key", "tc_tiles": [row, column], "ms"}.  The choice is applied to `gbk`.
    """
    import torch
    batch = isinstance(imgs, (list, tuple))
    ims = list(imgs) if batch else [imgs]
    shapes = [tuple(t.shape) for t in ims]
    nf = len(gbk.omegas)
    if nf == 0:
        return {"key": None, "tiling": [], "ctas": None, "ms": None}
    tc = gbk.precision != "fp32"
    path = cache_path or default_cache_path()
    key = cache_key(gbk, shapes, torch.cuda.get_device_name()) + (
        f"|tc{list(TC_TILES)}" if tc else f"|{list(tile_rows)}|{list(segments)}|{list(ctas)}")
    cache = _load(path) if use_cache else {}
    if key in cache:
        if tc:
            r, c = cache[key]["tc_tiles"]
            gbk.set_option("tc_tiles", r + 256 * c)
        else:
            gbk.set_option("bank_ctas", cache[key]["ctas"])
            for s, (tr, sg) in enumerate(cache[key]["tiling"]):
                gbk.set_tiling(s, tr, sg)
        return dict(cache[key], key=key, cached=True)

    outs = [torch.empty(gbk.out_shape(*sh), dtype=torch.complex64, device=t.device) for t, sh in zip(ims, shapes)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=ims[0].device)

    def run():
        if batch:
            gbk.filter_batch(ims, outs)
        else:
            gbk.filter(ims[0], outs[0])

    def timed():
        run()                       # rebuilds tables / work lists after a tiling change
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            run()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    if tc:
        best = None
        for r, c in TC_TILES:
            gbk.set_option("tc_tiles", r + 256 * c)
            ms = timed()
            if best is None or ms < best[2]:
                best = (r, c, ms)
        gbk.set_option("tc_tiles", best[0] + 256 * best[1])
        entry = {"tc_tiles": [best[0], best[1]], "ms": best[2]}
        if use_cache:
            cache = _load(path)
            cache[key] = entry
            _save(path, cache)
        return dict(entry, key=key, cached=False)

    best = None
    for c in ctas:
        gbk.set_option("bank_ctas", c)
        # start from the best uniform segment count, then descend frequency by frequency
        start, best_ms = None, None
        for sg in segments:
            gbk.set_tiling(-1, 0, sg)
            ms = timed()
            if best_ms is None or ms < best_ms:
                start, best_ms = sg, ms
        tiling = [[0, start] for _ in range(nf)]
        gbk.set_tiling(-1, 0, start)
        for s in sorted(range(nf), key=lambda i: -gbk.sigmas[i]):
            for tr in tile_rows:
                for sg in segments:
                    if [tr, sg] == tiling[s]:
                        continue
                    gbk.set_tiling(s, tr, sg)
                    ms = timed()
                    if ms < best_ms:
                        best_ms = ms
                        tiling[s] = [tr, sg]
            gbk.set_tiling(s, *tiling[s])
        if best is None or best_ms < best[2]:
            best = (c, tiling, best_ms)
    c, tiling, best_ms = best
    gbk.set_option("bank_ctas", c)
    for s, (tr, sg) in enumerate(tiling):
        gbk.set_tiling(s, tr, sg)
    entry = {"tiling": tiling, "ctas": c, "ms": best_ms}
    if use_cache:
        cache = _load(path)
        cache[key] = entry
        _save(path, cache)
    return dict(entry, key=key, cached=False)
