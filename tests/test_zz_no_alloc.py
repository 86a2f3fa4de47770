"""mmsar_image_static: imaging for callers that cannot allocate device memory.

Hard real-time acquisition loops and plug-ins that only receive buffers from
their host cannot call cudaMalloc while they run, so they cannot provide the
scratch workspace mmsar_image needs.  mmsar_image_static runs the same
launch sequence on a fixed scratch area inside the library.  These tests call
it through the C ABI (ctypes, no binding helper) twice in a row -- first a
scan whose scratch fills most of the area, then a small one that must not
be disturbed by what the first left behind -- and compare each output with
the workspace entry point's output within the tolerance the parity tests
use.  They also check that the device's free memory does not change across
a call, that a non-finite echo is reported through the area's error word,
and that oversized plans are refused.  This file is collected last so that
a stop-at-first-failure run has already run everything else.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import rma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONTRACT = 1e-4      # NMSE bound of the FP32 path against the FP64 oracle
BOUND_W6 = 2e-5      # derived bound at the default Gaussian width 6


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_02064_gb300 import _lib
    return _lib.load()


def _device_args(scan, dev):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            for a in (scan.echo, np.asarray(scan.pos, np.float64), np.asarray(scan.tx, np.float64),
                      np.asarray(scan.rx, np.float64))]


def _static_call(lib, plan, args, vol, stream):
    echo, pos, tx, rx = args
    return lib.mmsar_image_static(plan._h, ctypes.c_void_p(echo.data_ptr()), None,
                                  ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(tx.data_ptr()),
                                  ctypes.c_void_p(rx.data_ptr()), ctypes.c_void_p(vol.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))


def _poll_static(lib, stream):
    return lib.mmsar_poll_error(None, ctypes.c_void_p(stream.cuda_stream))


def _scans():
    # ~20 MiB of scratch (64 x 64 x 32 voxels, Nk = 64, 7200 samples), then
    # the tiny scan (2 MiB): the second call runs over the first's leftovers
    big = synth.custom(nx_pos=30, ny_pos=30, nk=64, layout="awr1443", nx=64, ny=64, nz=32, seed=5, serp=True,
                       jitter=(1.5e-3, 3e-3), n_points=5)
    return [big, synth.tiny()]


def test_static_scratch_matches_workspace_entry_point(lib):
    from paper_2305_02064_gb300 import Plan, _lib
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    area = lib.mmsar_static_workspace_bytes()
    assert area == 32 << 20
    scans = _scans()
    plans = [Plan.for_scan(s) for s in scans]
    assert 20 << 20 <= plans[0].workspace_bytes <= area
    assert plans[1].workspace_bytes < plans[0].workspace_bytes // 4
    # one untimed call first: it loads the library's module that holds the
    # area (lazy module loading places the 32 MiB array then)
    warm = Plan.for_scan(scans[1])
    _lib.check(_static_call(lib, warm, _device_args(scans[1], dev), warm.new_volume(dev), stream))
    _lib.check(_poll_static(lib, stream))
    for scan, plan in zip(scans, plans):   # two calls in a row, the second on the first's leftovers
        args = _device_args(scan, dev)
        want = plan.new_volume(dev)
        ws = plan.new_workspace(dev)
        plan.image(ws, *args, want)
        got = torch.full(plan.volume_shape, complex(np.nan, np.nan), dtype=torch.complex64, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        _lib.check(_static_call(lib, plan, args, got, stream))
        _lib.check(_poll_static(lib, stream))   # synchronises; the area's error word is clear
        # nothing was allocated, by torch or by the library behind its back
        assert torch.cuda.mem_get_info(dev)[0] == free0
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == alloc0
        g, w = got.cpu().numpy(), want.cpu().numpy()
        assert np.all(np.isfinite(g))
        e = rma.nmse(g, w)
        assert e <= CONTRACT and e <= BOUND_W6, e
        assert rma.peak_index(g) == rma.peak_index(w)
        # and the static call agrees with the FP64 oracle like the workspace call does
        ref = rma.rma_exact(rma.setup_from(scan))
        assert rma.nmse(g, ref) <= BOUND_W6


def test_static_scratch_reports_nonfinite_input(lib):
    """A NaN echo sample is flagged in the area's error word, which
    mmsar_poll_error(NULL, stream) reads (and clears)."""
    from paper_2305_02064_gb300 import Plan, _lib
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    scan = synth.tiny()
    bad = scan.echo.copy()
    bad[0, 1, 17, 3] = np.nan
    plan = Plan.for_scan(scan)
    args = _device_args(scan, dev)
    args[0] = torch.from_numpy(bad).to(dev)
    vol = plan.new_volume(dev)
    _lib.check(_static_call(lib, plan, args, vol, stream))
    assert _poll_static(lib, stream) == 6   # MMSAR_ERR_NONFINITE
    assert b"non-finite" in lib.mmsar_last_error()
    assert _poll_static(lib, stream) == 0   # the word was cleared
    # a clean call afterwards reports nothing
    _lib.check(_static_call(lib, plan, _device_args(scan, dev), vol, stream))
    assert _poll_static(lib, stream) == 0


def test_static_scratch_rejects_oversized_plans(lib):
    from paper_2305_02064_gb300 import Plan
    g = synth.Grid(-0.128, -0.128, 0.2, 1e-3, 1e-3, 3.125e-3, 256, 256, 64)
    plan = Plan(2, 4, 16384, 256, 77e9, 4e9 / 256, g)
    assert plan.workspace_bytes > lib.mmsar_static_workspace_bytes()
    vol = plan.new_volume("cuda:0")
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    p = ctypes.c_void_p(dummy.data_ptr())
    code = lib.mmsar_image_static(plan._h, p, None, p, p, p, ctypes.c_void_p(vol.data_ptr()), None)
    assert code == 2   # MMSAR_ERR_UNSUPPORTED_SIZE
    assert b"scratch" in lib.mmsar_last_error()
