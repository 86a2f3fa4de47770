"""mmsar_image_static: imaging for callers that cannot allocate device memory.

Hard real-time acquisition loops and plug-ins that only receive buffers from
their host cannot call cudaMalloc while they run, so they cannot provide the
scratch workspace mmsar_image needs.  mmsar_image_static runs the same
launch sequence on a fixed scratch area inside the library.  These tests call
it through the C ABI (ctypes, no binding helper) twice in a row, on two
different scans, and compare each output with the workspace entry point's
output within the tolerance the parity tests use.  This file is collected
last so that a stop-at-first-failure run has already run everything else.
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


def test_static_scratch_matches_workspace_entry_point(lib):
    from paper_2305_02064_gb300 import Plan, _lib
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    scans = [synth.tiny(),
             synth.custom(nx_pos=7, ny_pos=5, nk=20, layout="awr1443", nx=24, ny=12, nz=10, seed=9,
                          jitter=(0.7e-3, 4e-3), snr_db=20)]
    assert lib.mmsar_static_workspace_bytes() == 32 << 20
    for scan in scans:   # two calls in a row, the second on different sizes
        plan = Plan.for_scan(scan)
        assert plan.workspace_bytes <= lib.mmsar_static_workspace_bytes()
        args = _device_args(scan, dev)
        want = plan.new_volume(dev)
        ws = plan.new_workspace(dev)
        plan.image(ws, *args, want)
        got = torch.full(plan.volume_shape, complex(np.nan, np.nan), dtype=torch.complex64, device=dev)
        torch.cuda.synchronize()
        before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        _lib.check(_static_call(lib, plan, args, got, stream))
        torch.cuda.synchronize()
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
        g, w = got.cpu().numpy(), want.cpu().numpy()
        assert np.all(np.isfinite(g))
        e = rma.nmse(g, w)
        assert e <= CONTRACT and e <= BOUND_W6, e
        assert rma.peak_index(g) == rma.peak_index(w)
        # and the static call agrees with the FP64 oracle like the workspace call does
        ref = rma.rma_exact(rma.setup_from(scan))
        assert rma.nmse(g, ref) <= BOUND_W6


def test_static_scratch_rejects_oversized_plans(lib):
    from paper_2305_02064_gb300 import Plan, _lib
    g = synth.Grid(-0.128, -0.128, 0.2, 1e-3, 1e-3, 3.125e-3, 256, 256, 64)
    plan = Plan(2, 4, 16384, 256, 77e9, 4e9 / 256, g)
    assert plan.workspace_bytes > lib.mmsar_static_workspace_bytes()
    vol = plan.new_volume("cuda:0")
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    p = ctypes.c_void_p(dummy.data_ptr())
    code = lib.mmsar_image_static(plan._h, p, None, p, p, p, ctypes.c_void_p(vol.data_ptr()), None)
    assert code == 2   # MMSAR_ERR_UNSUPPORTED_SIZE
    assert b"scratch" in lib.mmsar_last_error()
