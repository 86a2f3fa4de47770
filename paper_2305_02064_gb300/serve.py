"""Continuous-batching server for imaging requests.

Requests (scans of different sizes) arrive over time.  The scheduler admits a
waiting request as soon as a stream slot is free and the device memory it
needs fits under the admission cap together with everything already
admitted; admitted requests run concurrently on their own streams, so work
that arrives while others are on the GPU overlaps with them.  Each request's
latency runs from its arrival to the completion of its volume.

The scheduling logic (``Scheduler``) is independent of CUDA: it drives an
executor object with ``start(req) -> handle``, ``done(handle) -> bool`` and
``finish(handle)``; ``GpuExecutor`` is the CUDA one (pinned host echo ->
device on the request's stream -- for FP16/BF16 storage the echo is kept as
scaled pairs, quantised once per scan on the device --, imaging, completion
event; each stream slot reuses its own device buffers, so steady-state
serving allocates no device memory).  Tests drive the scheduler
with a fake executor.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time


@dataclasses.dataclass
class ServeRequest:
    rid: int
    scan: object
    arrival: float              # seconds since the start of the run
    footprint: int = 0          # device bytes while admitted
    admitted: float = math.nan
    completed: float = math.nan
    result: object = None
    pinned: object = None       # page-locked host copies of the inputs (GpuExecutor.pin)

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


class Scheduler:
    """Admission by memory and slots, FIFO among arrived requests."""

    def __init__(self, executor, slots: int, mem_cap: int, clock=time.perf_counter):
        self.ex = executor
        self.slots = slots
        self.mem_cap = mem_cap
        self.clock = clock
        self.in_use = 0
        self.peak_in_use = 0
        self.running = []            # (req, handle)
        self.max_concurrent = 0

    def run(self, requests, poll_sleep=0.0):
        """Serve ``requests`` (sorted by arrival); returns them with times set."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        done = []
        t0 = self.clock()
        for r in pending:
            if r.footprint > self.mem_cap:
                raise ValueError(f"request {r.rid} needs {r.footprint} bytes, above the admission cap")
        while pending or waiting or self.running:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # retire finished work first: it frees slots and memory
            still = []
            for req, h in self.running:
                if self.ex.done(h):
                    self.ex.finish(h)
                    req.completed = self.clock() - t0
                    self.in_use -= req.footprint
                    done.append(req)
                else:
                    still.append((req, h))
            self.running = still
            # admit in arrival order while a slot and the memory allow
            while waiting and len(self.running) < self.slots and \
                    self.in_use + waiting[0].footprint <= self.mem_cap:
                req = waiting.popleft()
                req.admitted = self.clock() - t0
                self.in_use += req.footprint
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                self.running.append((req, self.ex.start(req)))
                self.max_concurrent = max(self.max_concurrent, len(self.running))
            if not self.running and not waiting and pending:
                # idle until the next arrival
                delay = pending[0].arrival - (self.clock() - t0)
                if delay > 0:
                    time.sleep(min(delay, 0.01))
            elif poll_sleep:
                time.sleep(poll_sleep)
        return done


def poisson_arrivals(n, rate_hz, seed=0):
    import numpy as np
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def latency_summary(reqs):
    import numpy as np
    lat = np.array([r.latency for r in reqs])
    span = max(r.completed for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "images_per_s": len(reqs) / span, "n": len(reqs)}


class GpuExecutor:
    """CUDA executor: one stream per running request, pinned host echoes.

    Per request, on its stream: echo and geometry host -> device, FP16/BF16
    quantisation with a per-scan scale (unless complex64), the image, and the
    volume device -> host into a pinned buffer from a pool recycled by size;
    the request is done when that copy has landed.  ``finish`` hands the
    buffer back to the pool (keyed by volume shape) (``keep_results`` keeps a copy of the volume on
    the request first, for checks outside timed runs)."""

    def __init__(self, device, dtype="f16", n_streams=8, keep_results=False):
        import torch
        self.dev = torch.device(device)
        self.dtype = dtype
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_streams)]
        self.free_streams = list(range(n_streams))
        self.keep = keep_results
        self._out_pool = collections.defaultdict(list)   # volume shape -> free pinned volumes
        # per slot: device buffers reused by every request the slot serves
        # (grown to the largest request seen, or sized up front by reserve):
        # no device allocation in steady state, so no allocator stall
        self._slot_bufs = [{} for _ in range(n_streams)]

    def footprint(self, scan):
        from .batch import plan_for
        p = plan_for(scan, dtype=self.dtype)
        T, R, P, Nk = scan.echo.shape
        echo_dev = T * R * P * Nk * (8 if self.dtype == "c64" else 4)   # complex64, or FP16/BF16 pairs
        g = scan.grid
        return int(p.workspace_bytes + echo_dev + 8 * g.nx * g.ny * g.nz + 48 * (P + T + R))

    def pin(self, req):
        """Page-locked host copies of a request's inputs.  For FP16/BF16 storage
        the echo is stored reduced: it goes to the device once, the library's
        quantisation kernel turns it into scaled pairs, and those (with the
        scale) come back to pinned host memory -- every request of the scan
        then moves half the echo bytes."""
        import numpy as np
        import torch
        from . import quantize_echo
        s = req.scan
        geo = [torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory() for a in (s.pos, s.tx, s.rx)]
        echo_h = torch.from_numpy(np.ascontiguousarray(s.echo)).pin_memory()
        if self.dtype == "c64":
            req.pinned = [echo_h, None] + geo
            return
        st = self.streams[0]
        with torch.cuda.stream(st):
            q, scale = quantize_echo(echo_h.to(self.dev, non_blocking=True), self.dtype, stream=st)
            q_h = torch.empty(q.shape, dtype=q.dtype).pin_memory()
            scale_h = torch.empty(1, dtype=torch.float32).pin_memory()
            q_h.copy_(q, non_blocking=True)
            scale_h.copy_(scale, non_blocking=True)
        st.synchronize()
        req.pinned = [q_h, scale_h] + geo

    def _sizes(self, scan):
        from .batch import plan_for
        p = plan_for(scan, dtype=self.dtype)
        T, R, P, Nk = scan.echo.shape
        g = scan.grid
        echo = (T * R * P * Nk, "c64") if self.dtype == "c64" else (T * R * P * Nk * 2, self.dtype)
        return {"echo": echo, "geo": (3 * (P + T + R), "f64"), "ws": (p.workspace_bytes, "u8"),
                "vol": (g.nx * g.ny * g.nz, "c64")}

    def _take(self, si, name, numel, kind):
        import torch
        dt = {"c64": torch.complex64, "f16": torch.float16, "bf16": torch.bfloat16, "f64": torch.float64,
              "u8": torch.uint8, "f32": torch.float32, "i32": torch.int32}[kind]
        bufs = self._slot_bufs[si]
        t = bufs.get(name)
        if t is None or t.numel() < numel:
            with torch.cuda.stream(self.streams[si]):
                t = torch.empty(max(numel, 1), dtype=dt, device=self.dev)
            bufs[name] = t
        return t[:numel]

    def reserve(self, scans):
        """Size every slot's buffers for the largest of ``scans`` (before serving)."""
        need = {}
        for sc in scans:
            for name, (n, kind) in self._sizes(sc).items():
                need[name] = (max(n, need.get(name, (0, kind))[0]), kind)
        for si in range(len(self.streams)):
            for name, (n, kind) in need.items():
                self._take(si, name, n, kind)
            self._take(si, "scale", 1, "f32")

    def _out_buffer(self, shape):
        import torch
        free = self._out_pool[tuple(shape)]
        if free:
            return free.pop()
        return torch.empty(shape, dtype=torch.complex64).pin_memory()

    def start(self, req):
        import torch
        from .batch import plan_for
        si = self.free_streams.pop()
        st = self.streams[si]
        plan = plan_for(req.scan, dtype=self.dtype)
        if req.pinned is None:
            self.pin(req)
        echo_h, scale_h, pos_h, tx_h, rx_h = req.pinned
        vol_h = self._out_buffer(plan.volume_shape)
        sz = self._sizes(req.scan)
        echo = self._take(si, "echo", *sz["echo"]).view(echo_h.shape)
        geo = self._take(si, "geo", *sz["geo"])
        ws = self._take(si, "ws", *sz["ws"])
        vol = self._take(si, "vol", *sz["vol"]).view(plan.volume_shape)
        scale = None if scale_h is None else self._take(si, "scale", 1, "f32")
        with torch.cuda.stream(st):
            echo.copy_(echo_h, non_blocking=True)
            if scale is not None:
                scale.copy_(scale_h, non_blocking=True)
            pos, tx, rx = (geo[o:o + t.numel()].view(t.shape) for o, t in
                           zip((0, pos_h.numel(), pos_h.numel() + tx_h.numel()), (pos_h, tx_h, rx_h)))
            for d, h in zip((pos, tx, rx), (pos_h, tx_h, rx_h)):
                d.copy_(h, non_blocking=True)
            plan.image(ws, echo, pos, tx, rx, vol, echo_scale=scale, stream=st)
            vol_h.copy_(vol, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"req": req, "si": si, "ev": ev, "bufs": (echo, pos, tx, rx, ws, scale, vol), "vol_h": vol_h,
                "plan": plan}

    def done(self, h):
        return h["ev"].query()

    def finish(self, h):
        h["plan"].poll_error(h["bufs"][4], stream=self.streams[h["si"]])
        vol_h = h["vol_h"]
        if self.keep:
            h["req"].result = vol_h.clone()
        self._out_pool[tuple(vol_h.shape)].append(vol_h)
        self.free_streams.append(h["si"])
        h.clear()
