"""Batched imaging of many independent scans of uneven sizes.

Each scan becomes a ``ScanJob``: its plan, its echo/geometry resident on the
device (optionally stored as FP16/BF16 with a per-scan scale), a private
workspace and an output volume.  ``image_batch`` enqueues all jobs through
``mmsar_image_batch`` round-robin over several CUDA streams so that small
scans overlap on the GPU; ``image_batch_fused`` enqueues them through
``mmsar_image_batch_fused`` instead, one launch per stage and kernel shape for
the whole batch; ``BatchGraph`` captures either form once into a CUDA graph
and replays it with a single launch.  Every kernel that runs is the
library's; this module only marshals pointers and streams.
"""
from __future__ import annotations

import collections
import ctypes
import threading

from . import Plan, _lib, _ptr, quantize_echo

# Plans are host-only and reusable: the imaging calls only read a plan, so
# one plan serves every scan of its shape on any stream (each call with its
# own workspace).  The cache keeps the most recently used PLAN_CACHE_MAX
# plans; an evicted plan lives on while a job still holds it.
PLAN_CACHE_MAX = 256
_PLAN_CACHE: "collections.OrderedDict" = collections.OrderedDict()
_PLAN_LOCK = threading.Lock()


def plan_for(scan, dtype="c64", **kw):
    """A plan per (shape, grid, dtype, options), from a bounded LRU cache."""
    T, R, P, Nk = scan.echo.shape
    g = scan.grid
    key = (T, R, P, Nk, scan.f0, scan.df, g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, g.nx, g.ny, g.nz, dtype,
           tuple(sorted(kw.items())))
    with _PLAN_LOCK:
        p = _PLAN_CACHE.get(key)
        if p is not None:
            _PLAN_CACHE.move_to_end(key)
            return p
    p = Plan.for_scan(scan, dtype=dtype, **kw)
    with _PLAN_LOCK:
        p = _PLAN_CACHE.setdefault(key, p)
        _PLAN_CACHE.move_to_end(key)
        while len(_PLAN_CACHE) > PLAN_CACHE_MAX:
            _PLAN_CACHE.popitem(last=False)
    return p


class ScanJob:
    """One scan resident on the device with everything its image needs."""

    def __init__(self, scan, device, dtype="c64", stream=None, **plan_kw):
        import numpy as np
        import torch
        self.scan = scan
        self.dtype = dtype
        self.plan = plan_for(scan, dtype=dtype, **plan_kw)
        s = stream or torch.cuda.current_stream(device)
        with torch.cuda.stream(s):
            echo = torch.from_numpy(np.ascontiguousarray(scan.echo)).to(device, non_blocking=True)
            if dtype == "c64":
                self.echo, self.scale = echo, None
            else:
                self.echo, self.scale = quantize_echo(echo, dtype, stream=s)
            self.pos = torch.from_numpy(np.ascontiguousarray(scan.pos, np.float64)).to(device)
            self.tx = torch.from_numpy(np.ascontiguousarray(scan.tx, np.float64)).to(device)
            self.rx = torch.from_numpy(np.ascontiguousarray(scan.rx, np.float64)).to(device)
            self.ws = self.plan.new_workspace(device)
            self.vol = self.plan.new_volume(device)

    @property
    def footprint(self) -> int:
        return int(self.ws.numel() + self.echo.numel() * self.echo.element_size() +
                   self.vol.numel() * 8 + 24 * (self.pos.shape[0] + 16))

    def request(self) -> _lib.Request:
        import torch
        return _lib.Request(self.plan._h.value, self.ws.data_ptr(), self.ws.numel(), self.echo.data_ptr(),
                            self.scale.data_ptr() if self.scale is not None else None, self.pos.data_ptr(),
                            self.tx.data_ptr(), self.rx.data_ptr(), self.vol.data_ptr())

    def tune(self, stream=None):
        """Autotune the gridding launch shape of this job's plan on its own data
        (once per plan: jobs of one shape share it)."""
        from .tune import autotune
        if self.plan.tuned is None:
            autotune(self.plan, self.ws, self.echo, self.pos, self.tx, self.rx, self.vol, echo_scale=self.scale,
                     stream=stream)
        return self.plan.tuned

    def image(self, stream=None):
        self.plan.image(self.ws, self.echo, self.pos, self.tx, self.rx, self.vol, echo_scale=self.scale,
                        stream=stream)


def image_batch(jobs, streams):
    """Enqueue every job through mmsar_image_batch, job i on streams[i % len]."""
    lib = _lib.load()
    reqs = (_lib.Request * len(jobs))(*[j.request() for j in jobs])
    hs = (ctypes.c_void_p * len(streams))(*[ctypes.c_void_p(s.cuda_stream) for s in streams])
    _lib.check(lib.mmsar_image_batch(reqs, len(jobs), hs, len(streams)))


def image_batch_fused(jobs, stream=None) -> int:
    """Enqueue every job through mmsar_image_batch_fused on one stream (one
    launch per stage and kernel shape); returns the kernels enqueued."""
    import torch
    lib = _lib.load()
    reqs = (_lib.Request * len(jobs))(*[j.request() for j in jobs])
    s = stream or torch.cuda.current_stream()
    n = ctypes.c_int()
    _lib.check(lib.mmsar_image_batch_fused(reqs, len(jobs), ctypes.c_void_p(s.cuda_stream), ctypes.byref(n)))
    return n.value


class BatchGraph:
    """A fixed batch captured once into a CUDA graph and replayed with one
    launch: forked onto n_streams streams, either ten launches per job
    (round-robin), or with ``fused`` the jobs split round-robin into
    n_streams sub-batches, each as the fused launches of
    mmsar_image_batch_fused on its own stream (so the stages of different
    sub-batches overlap)."""

    def __init__(self, jobs, n_streams=4, device=None, fused=False):
        import torch
        self.jobs = list(jobs)
        self.fused = fused
        dev = device or self.jobs[0].vol.device
        self.main = torch.cuda.Stream(device=dev)
        self.side = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]
        self.launches = 0
        # one eager pass first (kernel attributes are set outside the capture)
        self._enqueue()
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.main):
            self._enqueue()

    def _enqueue(self):
        import torch
        cur = torch.cuda.current_stream()
        for s in self.side:
            s.wait_stream(cur)
        if self.fused:
            k = len(self.side)
            self.launches = sum(image_batch_fused(self.jobs[i::k], self.side[i]) for i in range(k)
                                if self.jobs[i::k])
        else:
            image_batch(self.jobs, self.side)
            self.launches = sum(j.plan.kernels_per_image for j in self.jobs)
        for s in self.side:
            cur.wait_stream(s)

    def replay(self):
        self.graph.replay()
