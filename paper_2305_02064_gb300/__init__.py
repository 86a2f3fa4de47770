"""GB300 multi-planar multistatic MIMO-SAR imaging (Smith & Torlak, IEEE Access 2022).

Python face of libmmsar (include/mmsar.h).  PyTorch supplies device memory
and streams; every step of the image formation runs in the library's CUDA
kernels for sm_103a.

    plan = Plan.from_scan_shape(T, R, P, Nk, f0, df, grid)
    ws = plan.new_workspace()                 # torch.uint8 CUDA tensor
    vol = plan.new_volume()                   # torch.complex64 [nx, ny, nz]
    plan.image(ws, echo, pos, tx, rx, vol)    # stream-ordered
    plan.poll_error(ws)                       # device-side conditions
"""
from __future__ import annotations

import ctypes
import math

from . import _lib
from ._lib import MmsarError, library_path  # noqa: F401

__all__ = ["Plan", "MmsarError", "peak", "quantize_echo", "library_path", "version"]


def version() -> str:
    return _lib.load().mmsar_version().decode()


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, what, dtype=None, numel=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise ValueError(f"{what} has dtype {t.dtype}, expected {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Host-side plan for one acquisition shape and voxel grid.  ``compensate``:
    1 (or True) applies Eq. 11-12 as the paper does, 2 uses the residual of
    Eq. 5 evaluated at the scene centre, 0 (or False) skips compensation."""

    def __init__(self, n_tx, n_rx, n_pos, n_k, f0_hz, df_hz, grid, dtype="c64", z_ref=None, z_scene=None,
                 compensate=True, nufft_tol=1e-3, mx=0, my=0):
        lib = _lib.load()
        self._lib = lib
        self.shape = _lib.Shape(int(n_tx), int(n_rx), int(n_pos), int(n_k), float(f0_hz), float(df_hz),
                                _lib.DTYPES[dtype])
        g = grid
        self.grid = _lib.Grid(float(g.x0), float(g.y0), float(g.z0), float(g.dx), float(g.dy), float(g.dz),
                              int(g.nx), int(g.ny), int(g.nz))
        self.opt = _lib.Options(_lib._nan(z_ref), _lib._nan(z_scene), int(compensate), float(nufft_tol),
                                int(mx), int(my))
        self.dtype = dtype
        h = ctypes.c_void_p()
        _lib.check(lib.mmsar_plan_create(ctypes.byref(h), ctypes.byref(self.shape), ctypes.byref(self.grid),
                                         ctypes.byref(self.opt)))
        self._h = h
        n = ctypes.c_size_t()
        _lib.check(lib.mmsar_plan_workspace_bytes(h, ctypes.byref(n)))
        self.workspace_bytes = int(n.value)
        w, mxv, myv, kpi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(lib.mmsar_plan_info(h, ctypes.byref(w), ctypes.byref(mxv), ctypes.byref(myv), ctypes.byref(kpi)))
        self.kernel_width, self.mx, self.my = w.value, mxv.value, myv.value
        self.kernels_per_image = kpi.value
        self._events = None
        self.tuned = None       # set by tune.autotune

    @classmethod
    def for_scan(cls, scan, **kw):
        """Plan matching a synthetic scan object (echo/pos/tx/rx/f0/df/grid)."""
        T, R, P, Nk = scan.echo.shape
        return cls(T, R, P, Nk, scan.f0, scan.df, scan.grid, **kw)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.mmsar_plan_destroy(h)
            self._h = None

    def set_tiles(self, freqs_per_lane: int, warps_per_cta: int, grouped: int = 0, tensor_cores: int = 0):
        """Gridding form and launch shape (see mmsar_plan_set_tiles; tune.autotune
        picks one): tensor_cores=1..5 selects a tensor-core gridding (the other
        fields are then ignored), 0 the FP32 FMA form given by the others."""
        _lib.check(self._lib.mmsar_plan_set_tiles(self._h, ctypes.byref(
            _lib.Tiles(int(freqs_per_lane), int(warps_per_cta), int(grouped), int(tensor_cores)))))

    def set_wait_test(self, on: bool):
        """Exercise the bounded-wait expiry of the tensor-core gridding on the
        next images (see mmsar_plan_set_wait_test; tests only)."""
        _lib.check(self._lib.mmsar_plan_set_wait_test(self._h, 1 if on else 0))

    @property
    def tiles(self):
        """(frequencies per lane, warps per CTA, grouped, tensor cores) of the gridding."""
        t = _lib.Tiles()
        _lib.check(self._lib.mmsar_plan_get_tiles(self._h, ctypes.byref(t)))
        return (t.grid_freqs_per_lane, t.grid_warps_per_cta, t.grid_grouped, t.grid_tensor_cores)

    @property
    def volume_shape(self):
        return (self.grid.nx, self.grid.ny, self.grid.nz)

    @property
    def n_samples(self):
        return self.shape.n_tx * self.shape.n_rx * self.shape.n_pos

    def new_workspace(self, device=None):
        import torch
        # 256-byte aligned: the caching allocator returns 512-byte aligned blocks
        return torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=device or "cuda")

    def new_volume(self, device=None):
        import torch
        return torch.empty(self.volume_shape, dtype=torch.complex64, device=device or "cuda")

    def image(self, workspace, echo, pos, tx, rx, vol, echo_scale=None, stream=None):
        """Run the whole imaging path on ``stream`` (default: torch's current)."""
        import torch
        s = self.shape
        n_echo = s.n_tx * s.n_rx * s.n_pos * s.n_k
        if self.dtype == "c64":
            e = _ptr(echo, "echo", torch.complex64, n_echo)
        else:
            want = torch.float16 if self.dtype == "f16" else torch.bfloat16
            e = _ptr(echo, "echo", want, 2 * n_echo)
        code = self._lib.mmsar_image(
            self._h, _ptr(workspace, "workspace", torch.uint8), ctypes.c_size_t(workspace.numel()), e,
            _ptr(echo_scale, "echo_scale", torch.float32, 1), _ptr(pos, "pos", torch.float64, 3 * s.n_pos),
            _ptr(tx, "tx", torch.float64, 3 * s.n_tx), _ptr(rx, "rx", torch.float64, 3 * s.n_rx),
            _ptr(vol, "vol", torch.complex64, self.grid.nx * self.grid.ny * self.grid.nz), _stream_handle(stream))
        _lib.check(code)
        return vol

    @staticmethod
    def stage_names():
        lib = _lib.load()
        return [lib.mmsar_stage_name(i).decode() for i in range(lib.mmsar_stage_count())]

    def set_stage_events(self, events):
        """Record the given torch.cuda.Event objects around each stage of
        every later image() call (len == number of stages + 1); None: off."""
        if events is None:
            _lib.check(self._lib.mmsar_plan_set_stage_events(self._h, None, 0))
            self._events = None
            return
        import torch
        for e in events:
            if not e.cuda_event:       # torch creates the CUDA event on its first record
                e.record(torch.cuda.current_stream())
        arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        _lib.check(self._lib.mmsar_plan_set_stage_events(self._h, arr, len(events)))
        self._events = list(events)

    def backproject(self, echo, pos, tx, rx, out=None, voxels=None, stream=None):
        """Direct back-projection at ``voxels`` (device float64 [n, 3]) or at
        every voxel of the plan's grid; returns complex64 [n] (or the grid)."""
        import torch
        s = self.shape
        n = voxels.shape[0] if voxels is not None else self.grid.nx * self.grid.ny * self.grid.nz
        if out is None:
            shape = (n,) if voxels is not None else self.volume_shape
            out = torch.empty(shape, dtype=torch.complex64, device=echo.device)
        _lib.check(self._lib.mmsar_backproject(
            self._h, _ptr(echo, "echo", torch.complex64, s.n_tx * s.n_rx * s.n_pos * s.n_k),
            _ptr(pos, "pos", torch.float64, 3 * s.n_pos), _ptr(tx, "tx", torch.float64, 3 * s.n_tx),
            _ptr(rx, "rx", torch.float64, 3 * s.n_rx), _ptr(voxels, "voxels", torch.float64),
            ctypes.c_int64(n), _ptr(out, "out", torch.complex64, n), _stream_handle(stream)))
        return out

    def poll_error(self, workspace, stream=None):
        _lib.check(self._lib.mmsar_poll_error(_ptr(workspace, "workspace"), _stream_handle(stream)))


def peak(vol, scratch=None, stream=None):
    """(linear index, max |o|) of a complex64 CUDA volume, computed on device."""
    import torch
    lib = _lib.load()
    n = vol.numel()
    if scratch is None:
        scratch = torch.empty(int(lib.mmsar_peak_scratch_bytes(n)), dtype=torch.uint8, device=vol.device)
    res = torch.empty(2, dtype=torch.int64, device=vol.device)
    _lib.check(lib.mmsar_peak(_ptr(vol, "vol", torch.complex64), ctypes.c_int64(n), _ptr(scratch, "scratch"),
                              _ptr(res, "result"), _stream_handle(stream)))
    r = res.cpu()
    idx = int(r[0])
    mag = float(r[1:2].view(torch.float32)[0])
    return idx, mag


def quantize_echo(echo, dtype="f16", out=None, scale=None, scratch=None, stream=None):
    """Per-scan max-abs scaling of a complex64 CUDA echo into FP16 or BF16
    pairs on the device.  Returns (out, scale): out has the echo's shape plus
    a trailing axis of 2 (re, im); scale is a 1-element float32 tensor."""
    import torch
    lib = _lib.load()
    if echo.dtype != torch.complex64:
        raise ValueError("echo must be complex64")
    want = torch.float16 if dtype == "f16" else torch.bfloat16
    dev = echo.device
    if out is None:
        out = torch.empty(tuple(echo.shape) + (2,), dtype=want, device=dev)
    if scale is None:
        scale = torch.empty(1, dtype=torch.float32, device=dev)
    if scratch is None:
        scratch = torch.empty(1, dtype=torch.int32, device=dev)
    _lib.check(lib.mmsar_quantize_echo(_ptr(echo, "echo"), ctypes.c_int64(echo.numel()), _lib.DTYPES[dtype],
                                       _ptr(out, "out", want, 2 * echo.numel()), _ptr(scale, "scale", torch.float32, 1),
                                       _ptr(scratch, "scratch", torch.int32, 1), _stream_handle(stream)))
    return out, scale
