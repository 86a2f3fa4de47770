"""Continuous-batching server for imaging requests.

Requests (scans of different sizes) arrive over time.  The scheduler admits a
waiting request as soon as a stream slot is free and the device memory it
needs fits under the admission cap together with everything already
admitted; admitted requests run concurrently on their own streams, so work
that arrives while others are on the GPU overlaps with them.  Each request's
latency runs from its arrival to the completion of its volume.

Device memory is one arena: ``GpuExecutor`` allocates a single buffer of
``mem_cap`` bytes before serving, and ``Arena`` (host-side bookkeeping, first
fit, 256-byte aligned blocks, freed neighbours merged) places each admitted
request's echo, geometry, scale, workspace and volume in it.  A waiting
request is admitted when a stream slot is free and the arena can place all
its blocks; they return to the arena when its volume has reached the host.
Serving therefore never allocates device memory, and what is resident is
bounded by the cap by construction.

The scheduling logic (``Scheduler``) is independent of CUDA: it drives an
executor object with ``start(req) -> handle``, ``done(handle) -> bool`` and
``finish(handle)`` (and, for arena admission, ``block_sizes(req)``);
``GpuExecutor`` is the CUDA one (pinned host echo -> device on the request's
stream -- for FP16/BF16 storage the echo is kept as scaled pairs, quantised
once per scan on the device --, imaging, completion event).  Tests drive the
scheduler and the arena with a fake executor.
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
    placement: object = None    # the request's blocks in the arena while admitted

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


class Arena:
    """First-fit placement of blocks in one buffer of ``capacity`` bytes
    (host-side bookkeeping of byte offsets; every block starts on
    ``align`` bytes).  ``place`` puts all of a request's blocks or none;
    ``release`` returns them and merges free neighbours."""

    def __init__(self, capacity: int, align: int = 256):
        self.capacity = int(capacity)
        self.align = int(align)
        self.free = [(0, self.capacity)]     # (offset, size), sorted by offset, disjoint, merged
        self.in_use = 0
        self.peak = 0

    def _round(self, n):
        return max(self.align, (int(n) + self.align - 1) // self.align * self.align)

    def place(self, sizes):
        """Offsets of blocks of the given byte sizes, or None if they do not all fit."""
        free = list(self.free)
        offs = []
        for n in sizes:
            n = self._round(n)
            for i, (o, sz) in enumerate(free):
                if sz >= n:
                    offs.append((o, n))
                    free[i] = (o + n, sz - n)
                    if free[i][1] == 0:
                        del free[i]
                    break
            else:
                return None
        self.free = free
        self.in_use += sum(n for _, n in offs)
        self.peak = max(self.peak, self.in_use)
        return offs

    def release(self, blocks):
        for o, n in blocks:
            self.in_use -= n
            self.free.append((o, n))
        self.free.sort()
        merged = []
        for o, n in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + n)
            else:
                merged.append((o, n))
        self.free = merged

    def largest_free(self) -> int:
        return max((n for _, n in self.free), default=0)


class Scheduler:
    """Admission by memory and slots, FIFO among arrived requests.  With an
    ``arena`` (the executor's), a request is admitted when the arena can place
    its blocks (``executor.block_sizes(req)``); without one, when the sum of
    the admitted footprints stays within ``mem_cap``."""

    def __init__(self, executor, slots: int, mem_cap: int, clock=time.perf_counter, arena=None):
        self.ex = executor
        self.slots = slots
        self.mem_cap = mem_cap
        self.clock = clock
        self.arena = arena if arena is not None else getattr(executor, "arena", None)
        self.in_use = 0
        self.peak_in_use = 0
        self.running = []            # (req, handle)
        self.max_concurrent = 0

    def _admit(self, req) -> bool:
        if self.arena is None:
            if self.in_use + req.footprint > self.mem_cap:
                return False
            req.placement = None
        else:
            req.placement = self.arena.place(self.ex.block_sizes(req))
            if req.placement is None:
                return False
        self.in_use += req.footprint
        self.peak_in_use = max(self.peak_in_use, self.in_use if self.arena is None else self.arena.in_use)
        return True

    def _retire(self, req):
        self.in_use -= req.footprint
        if self.arena is not None and req.placement is not None:
            self.arena.release(req.placement)
            req.placement = None

    def run(self, requests, poll_sleep=0.0):
        """Serve ``requests`` (sorted by arrival); returns them with times set."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        done = []
        t0 = self.clock()
        for r in pending:
            if self.arena is None and r.footprint > self.mem_cap:
                raise ValueError(f"request {r.rid} needs {r.footprint} bytes, above the admission cap")
            if self.arena is not None:
                need = sum(self.arena._round(n) for n in self.ex.block_sizes(r))
                if need > self.arena.capacity:
                    raise ValueError(f"request {r.rid} needs {need} bytes, above the arena of "
                                     f"{self.arena.capacity} bytes")
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
                    self._retire(req)
                    done.append(req)
                else:
                    still.append((req, h))
            self.running = still
            # admit in arrival order while a slot and the memory allow
            while waiting and len(self.running) < self.slots and self._admit(waiting[0]):
                req = waiting.popleft()
                req.admitted = self.clock() - t0
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
    """CUDA executor: one stream per running request, pinned host echoes, and
    every device buffer a request uses placed in one arena.

    The arena is a single device buffer of ``mem_cap`` bytes allocated when the
    executor is made; ``arena`` places the blocks of each admitted request
    (``block_sizes``: echo, geometry, scale, workspace, volume) and
    ``start`` images into views of them.  Per request, on its stream: echo
    and geometry host -> device, the image, and the volume device -> host into
    a pinned buffer from a pool recycled by size; the request is done when
    that copy has landed.  ``finish`` hands the host buffer back to the pool
    (``keep_results`` keeps a copy of the volume on the request first, for
    checks outside timed runs); the scheduler returns the blocks to the
    arena."""

    def __init__(self, device, dtype="f16", n_streams=8, keep_results=False, mem_cap=40 << 30):
        import torch
        self.dev = torch.device(device)
        self.dtype = dtype
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_streams)]
        self.free_streams = list(range(n_streams))
        self.keep = keep_results
        self._out_pool = collections.defaultdict(list)   # volume shape -> free pinned volumes
        self.mem_cap = int(mem_cap)
        self.buf = torch.empty(self.mem_cap, dtype=torch.uint8, device=self.dev)   # the arena, allocated once
        self.arena = Arena(self.mem_cap)

    def _sizes(self, scan):
        from .batch import plan_for
        p = plan_for(scan, dtype=self.dtype)
        T, R, P, Nk = scan.echo.shape
        g = scan.grid
        echo = T * R * P * Nk * (8 if self.dtype == "c64" else 4)   # complex64, or FP16/BF16 pairs
        return [echo, 8 * 3 * (P + T + R), 4, p.workspace_bytes, 8 * g.nx * g.ny * g.nz]

    def block_sizes(self, req):
        """Bytes of the request's device blocks: echo, geometry, scale, workspace, volume."""
        return self._sizes(req.scan)

    def footprint(self, scan):
        return int(sum(self.arena._round(n) for n in self._sizes(scan)))

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

    def _view(self, block, dtype, shape):
        import torch
        o, _ = block
        n = int(torch.Size(shape).numel()) * torch.empty(0, dtype=dtype).element_size()
        return self.buf[o:o + n].view(dtype).view(shape)

    def _out_buffer(self, shape):
        import torch
        free = self._out_pool[tuple(shape)]
        if free:
            return free.pop()
        return torch.empty(shape, dtype=torch.complex64).pin_memory()

    def start(self, req):
        import torch
        from .batch import plan_for
        if req.placement is None:
            raise RuntimeError("request started without a placement in the arena")
        si = self.free_streams.pop()
        st = self.streams[si]
        plan = plan_for(req.scan, dtype=self.dtype)
        if req.pinned is None:
            self.pin(req)
        echo_h, scale_h, pos_h, tx_h, rx_h = req.pinned
        vol_h = self._out_buffer(plan.volume_shape)
        b_echo, b_geo, b_scale, b_ws, b_vol = req.placement
        echo = self._view(b_echo, echo_h.dtype, echo_h.shape)
        geo = self._view(b_geo, torch.float64, (pos_h.numel() + tx_h.numel() + rx_h.numel(),))
        ws = self._view(b_ws, torch.uint8, (max(plan.workspace_bytes, 1),))
        vol = self._view(b_vol, torch.complex64, plan.volume_shape)
        scale = None if scale_h is None else self._view(b_scale, torch.float32, (1,))
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
        return {"req": req, "si": si, "ev": ev, "ws": ws, "vol_h": vol_h, "plan": plan}

    def done(self, h):
        return h["ev"].query()

    def finish(self, h):
        h["plan"].poll_error(h["ws"], stream=self.streams[h["si"]])
        vol_h = h["vol_h"]
        if self.keep:
            h["req"].result = vol_h.clone()
        self._out_pool[tuple(vol_h.shape)].append(vol_h)
        self.free_streams.append(h["si"])
        h.clear()
