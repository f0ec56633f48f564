"""Continuous-batching server for filter-bank and localized-SDFT requests on one GPU.

Requests arrive over time (Poisson arrivals in the benchmark's served stream).  Images and
results stay in device memory.  A waiting request is admitted, first come first served, as
soon as a slot (a CUDA stream with its own library handles) is free and its output, plus
the tensor-core intermediate for a GB_FP16_TC bank, fits the HBM budget; it is launched at
once, so the work of requests admitted while others run overlaps on the GPU.  All request
memory comes from one fixed-budget arena (``gabor_arena_*`` of the C ABI), so admission
never allocates device memory and a request that does not fit waits instead of failing.

Latency is measured on the device clock: from the request's arrival (host time mapped onto
a reference CUDA event recorded when the run starts) to the CUDA event recorded after the
request's last kernel.
"""
from __future__ import annotations

import time
from collections import deque

import numpy as np

from .bank import Arena, GaborBank


class ImagePool:
    """Device-resident 1/f-noise source images; a request's image is a seeded crop of one.

    A crop is a strided view (row pitch = the source width), which the library reads in
    place, so serving a request moves no image bytes.
    """

    def __init__(self, n=4, side=4096, seed=3, device="cuda"):
        from .synth import pink_noise_device
        self.side = side
        self.images = [pink_noise_device(seed * 1000 + i, side, side, device) for i in range(n)]

    def crop(self, req):
        H, W = req["H"], req["W"]
        if H > self.side or W > self.side:
            raise ValueError("request larger than the source images")
        rng = np.random.default_rng(req["seed"])
        k = int(rng.integers(len(self.images)))
        y0 = int(rng.integers(self.side - H + 1))
        x0 = int(rng.integers(self.side - W + 1))
        return self.images[k][y0:y0 + H, x0:x0 + W]


def request_outputs(req):
    """Complex outputs (pixel x filter) of a request."""
    if req["kind"] == "bank":
        return len(req["thetas"]) * len(req["omegas"]) * req["H"] * req["W"]
    return req["M"] * req["M"] * req["H"] * req["W"]


class Server:
    """Slots x (stream, handles) over one arena of `budget_bytes` of device memory.

    precision: 'fp32' or 'fp16_tc' for the filter banks; SDFT requests use
    `sdft_precision` (default: the same).
    """

    def __init__(self, precision="fp32", slots=4, budget_bytes=96 << 30, max_side=4096, pool=None,
                 sdft_precision=None, device="cuda"):
        import torch
        self.torch = torch
        self.precision = precision
        self.sdft_precision = sdft_precision or precision
        self.max_side = max_side
        self.arena = Arena(budget_bytes, device=device)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.banks = [dict() for _ in range(slots)]
        self.sdfts = [None] * slots
        self.pool = pool if pool is not None else ImagePool(side=max_side, device=device)

    # -- handles (one set per slot: a handle is used on one stream at a time)
    def _bank(self, slot, req):
        key = (tuple(req["thetas"]), tuple(req["omegas"]), tuple(req["sigmas"]))
        b = self.banks[slot].get(key)
        if b is None:
            b = GaborBank(*key, precision=self.precision, max_shape=(self.max_side, self.max_side))
            self.banks[slot][key] = b
        return b

    def _sdft(self, slot):
        if self.sdfts[slot] is None:
            self.sdfts[slot] = GaborBank(precision=self.sdft_precision)
        return self.sdfts[slot]

    def prepare(self, reqs):
        """Create every handle the requests need on every slot (outside any timed region)."""
        for slot in range(len(self.streams)):
            self._sdft(slot)
            for r in reqs:
                if r["kind"] == "bank":
                    self._bank(slot, r)

    def request_bytes(self, req):
        """(output bytes, workspace bytes) the request holds while it runs."""
        out = request_outputs(req) * 8
        ws = self._bank(0, req).workspace_bytes(req["H"], req["W"]) if req["kind"] == "bank" else 0
        return out, ws

    # -- one request
    def _launch(self, slot, req, out_off, ws_off, ws_bytes):
        torch = self.torch
        st = self.streams[slot]
        img = self.pool.crop(req)
        H, W = req["H"], req["W"]
        with torch.cuda.stream(st):
            if req["kind"] == "bank":
                b = self._bank(slot, req)
                if ws_bytes:
                    b.set_workspace(self.arena.ptr(ws_off), ws_bytes)
                out = self.arena.view(out_off, b.out_shape(H, W), torch.complex64)
                b.filter(img, out=out, stream=st)
            else:
                M = req["M"]
                out = self.arena.view(out_off, (M, M, H, W), torch.complex64)
                self._sdft(slot).sdft(img, req["sigma"], M, out=out, stream=st)
            done = torch.cuda.Event(enable_timing=True)
            done.record(st)
        return out, done

    # -- the serving loop
    def run(self, reqs, on_done=None, max_inflight=None):
        """Serve `reqs` (dicts with arrival time ``t`` in seconds, sorted or not).

        Returns a list of per-request records: rid, kind, outputs, t_arrival, t_admit,
        t_done (seconds from the start of the run), latency_ms, or ``rejected`` for a request
        larger than the whole budget.  ``on_done(req, out)`` sees each result (a device
        tensor over arena memory) before its memory returns to the arena.
        """
        torch = self.torch
        order = sorted(range(len(reqs)), key=lambda i: reqs[i]["t"])
        pending = deque(order)
        waiting = deque()
        free_slots = deque(range(len(self.streams)))
        limit = max_inflight or len(self.streams)
        inflight = []
        records = [None] * len(reqs)
        cap = self.arena.stats()["capacity"]
        torch.cuda.synchronize()
        ref = torch.cuda.Event(enable_timing=True)
        ref.record()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and reqs[pending[0]]["t"] <= now:
                waiting.append(pending.popleft())
            progressed = False
            # retire finished requests (their memory goes back to the arena)
            still = []
            for job in inflight:
                i, slot, out, done, offs, t_admit = job
                if done.query():
                    t_done = ref.elapsed_time(done) / 1e3
                    if on_done is not None:
                        on_done(reqs[i], out)
                    for off in offs:
                        self.arena.free(off)
                    free_slots.append(slot)
                    r = reqs[i]
                    records[i] = dict(rid=i, kind=r["kind"], outputs=request_outputs(r), t_arrival=r["t"],
                                      t_admit=t_admit, t_done=t_done, latency_ms=(t_done - r["t"]) * 1e3)
                    progressed = True
                else:
                    still.append(job)
            inflight = still
            # admit waiting requests in arrival order while a slot and the budget allow
            while waiting and free_slots and len(inflight) < limit:
                i = waiting[0]
                out_b, ws_b = self.request_bytes(reqs[i])
                if out_b + ws_b > cap:
                    waiting.popleft()
                    records[i] = dict(rid=i, kind=reqs[i]["kind"], rejected=True)
                    continue
                out_off = self.arena.alloc(out_b)
                if out_off is None:
                    break
                ws_off = None
                if ws_b:
                    ws_off = self.arena.alloc(ws_b)
                    if ws_off is None:
                        self.arena.free(out_off)
                        break
                waiting.popleft()
                slot = free_slots.popleft()
                t_admit = time.perf_counter() - t0
                out, done = self._launch(slot, reqs[i], out_off, ws_off, ws_b)
                offs = [out_off] + ([ws_off] if ws_off is not None else [])
                inflight.append((i, slot, out, done, offs, t_admit))
                progressed = True
            if not progressed:
                if inflight or (pending and reqs[pending[0]]["t"] <= time.perf_counter() - t0 + 1e-4):
                    time.sleep(0)
                elif pending:
                    time.sleep(max(0.0, min(1e-3, reqs[pending[0]]["t"] - (time.perf_counter() - t0))))
        torch.cuda.synchronize()
        return records

    def close(self):
        for d in self.banks:
            for b in d.values():
                b.close()
            d.clear()
        for i, h in enumerate(self.sdfts):
            if h is not None:
                h.close()
            self.sdfts[i] = None
        self.arena.close()


def summarize(records):
    """p50 / p99 latency (ms) and outputs/s over the served (not rejected) requests."""
    done = [r for r in records if r is not None and not r.get("rejected")]
    if not done:
        return {"served": 0}
    lat = np.array([r["latency_ms"] for r in done])
    t_first = min(r["t_arrival"] for r in done)
    t_last = max(r["t_done"] for r in done)
    outs = sum(r["outputs"] for r in done)
    return {
        "served": len(done),
        "rejected": sum(1 for r in records if r is not None and r.get("rejected")),
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "outputs_per_s": outs / max(t_last - t_first, 1e-9),
        "requests_per_s": len(done) / max(t_last - t_first, 1e-9),
        "span_s": t_last - t_first,
    }


def with_rate(reqs, rate_hz):
    """The same requests with arrival times rescaled to a Poisson rate of `rate_hz` (the
    generator's times are for 1 request/s)."""
    return [dict(r, t=r["t"] / rate_hz) for r in reqs]


def closed_loop(reqs):
    """Every request arrives at t = 0 (saturation measurement)."""
    return [dict(r, t=0.0) for r in reqs]


def served_stream(seed=2, n=2200, lo=256, hi=4096, p_sdft=0.1):
    """The served-stream workload at 1 request/s (rescale with `with_rate`)."""
    from .synth import request_stream
    return request_stream(seed=seed, n=n, rate_hz=1.0, lo=lo, hi=hi, p_sdft=p_sdft)


def measure(precision, n_warm=200, n_meas=2000, rate_fracs=(0.7,), n_sat=300, budget_bytes=96 << 30,
            slots=4, seed=2, pool=None, log=None):
    """Served-stream measurement: closed-loop saturation rate, then Poisson arrivals at each
    fraction of it.  Returns {"saturation_req_s", "rates": {frac: summary}}."""
    reqs = served_stream(seed=seed, n=n_warm + n_meas)
    warm, meas = reqs[:n_warm], reqs[n_warm:]
    srv = Server(precision=precision, slots=slots, budget_bytes=budget_bytes, pool=pool)
    try:
        srv.prepare(reqs)
        srv.run(closed_loop(warm))
        sat = summarize(srv.run(closed_loop(meas[:n_sat])))
        sat_rate = sat["requests_per_s"]
        if log:
            log(f"serve {precision}: saturation {sat_rate:.1f} req/s")
        out = {"saturation_req_s": sat_rate, "rates": {}}
        for frac in rate_fracs:
            srv.run(with_rate(warm, frac * sat_rate))
            s = summarize(srv.run(with_rate(meas, frac * sat_rate)))
            s["rate_req_s"] = frac * sat_rate
            out["rates"][frac] = s
            if log:
                log(f"serve {precision} at {frac:.1f}x: p50 {s['p50_ms']:.2f} ms p99 {s['p99_ms']:.2f} ms "
                    f"{s['outputs_per_s']:.3e} outputs/s")
        return out
    finally:
        srv.close()


def _main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="served-stream measurement (continuous batching)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16_tc"])
    ap.add_argument("--n", type=int, default=2000)
    ap.add_argument("--warm", type=int, default=200)
    ap.add_argument("--rates", default="0.5,0.7,0.9")
    ap.add_argument("--budget-gib", type=float, default=96)
    ap.add_argument("--slots", type=int, default=4)
    a = ap.parse_args()
    res = measure(a.precision, n_warm=a.warm, n_meas=a.n, rate_fracs=[float(x) for x in a.rates.split(",")],
                  budget_bytes=int(a.budget_gib * (1 << 30)), slots=a.slots, log=print)
    print(json.dumps(res))


if __name__ == "__main__":
    _main()
