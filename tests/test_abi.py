"""CPU checks of the C ABI: the library builds, loads and exports every
function include/mmsar.h declares, and the host-side plan logic (validation,
kernel width, spectral grid, workspace size) behaves as documented.  No
compute call is made here (there is no GPU in this suite)."""
import math
import os
import re
import subprocess

import pytest

import synth
from paper_2305_02064_gb300 import Plan, _lib, MmsarError

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mmsar.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mmsar_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.library_path()], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for name in declared_functions():
        assert name in exported, name


def test_version_string():
    assert b"sm_103a" in _lib.load().mmsar_version()


def _plan(**kw):
    g = synth.centred_grid(32, 32, 16, 1e-3, 5e-3, 0.26)
    args = dict(n_tx=1, n_rx=2, n_pos=256, n_k=32, f0_hz=77e9, df_hz=125e6, grid=g)
    args.update(kw)
    return Plan(**args)


def test_defaults_and_kernel_width():
    p = _plan()
    assert (p.mx, p.my) == (32, 32)
    assert p.kernel_width == 6
    assert _plan(nufft_tol=1e-4).kernel_width == 8
    assert _plan(nufft_tol=1e-6).kernel_width == 12
    assert _plan(nufft_tol=0.01).kernel_width == 4


def test_spectral_grid_rounding():
    g = synth.Grid(0, 0, 0.2, 1e-3, 1e-3, 1e-3, 24, 12, 10)
    p = Plan(2, 4, 35, 20, 77e9, 2e8, g)
    assert (p.mx, p.my) == (32, 16)
    with pytest.raises(MmsarError):
        Plan(2, 4, 35, 20, 77e9, 2e8, g, mx=48)
    with pytest.raises(MmsarError):
        Plan(2, 4, 35, 20, 77e9, 2e8, g, mx=16)


@pytest.mark.parametrize("bad", [dict(n_tx=0), dict(n_k=0), dict(n_k=5000), dict(f0_hz=-1.0), dict(df_hz=0.0),
                                 dict(n_pos=-1), dict(dtype="bogus"), dict(z_ref=0.3, z_scene=0.2)])
def test_plan_rejects_bad_arguments(bad):
    with pytest.raises((MmsarError, KeyError)):
        _plan(**bad)


def test_plan_rejects_bad_grid():
    for g in (synth.Grid(0, 0, 0, 0.0, 1e-3, 1e-3, 8, 8, 8), synth.Grid(0, 0, 0, 1e-3, 1e-3, 1e-3, 8, 8, 0),
              synth.Grid(0, 0, 0, 1e-3, 1e-3, 1e-3, 2048, 8, 8), synth.Grid(0, 0, math.nan, 1e-3, 1e-3, 1e-3, 8, 8, 8)):
        with pytest.raises(MmsarError):
            Plan(1, 1, 4, 4, 77e9, 1e9, g)


def test_workspace_grows_with_the_problem():
    small = _plan().workspace_bytes
    more_k = _plan(n_k=64).workspace_bytes
    more_pos = _plan(n_pos=1024).workspace_bytes
    assert small > 0 and more_k > small and more_pos > small
    assert small % 256 == 0


def test_empty_scan_plan_is_valid():
    p = _plan(n_pos=0)
    assert p.workspace_bytes > 0


def test_realistic_workspace_fits_hbm():
    s = synth.Grid(-0.128, -0.128, 0.2, 1e-3, 1e-3, 3.125e-3, 256, 256, 64)
    p = Plan(2, 4, 16384, 256, 77e9, 4e9 / 256, s)
    assert p.workspace_bytes < 2 * 1024 ** 3


def test_gridding_launch_shape_setter():
    """mmsar_plan_set_tiles accepts the gridding forms and launch shapes and
    rejects everything else (the grouped form takes 1 or 2 frequencies per
    lane); the default is the warp-specialised tensor-core form (5)."""
    from paper_2305_02064_gb300._lib import MmsarError
    p = _plan()
    assert p.tiles == (2, 4, 0, 5)
    for shp in ((1, 4, 0), (2, 4, 1), (4, 4, 0), (1, 8, 1), (4, 8, 0), (2, 8, 0)):
        p.set_tiles(*shp)
        assert p.tiles == shp + (0,)
    for v in (1, 2, 3, 4, 5):
        p.set_tiles(2, 4, 0, v)
        assert p.tiles == (2, 4, 0, v)
    p.set_tiles(2, 8, 0)
    for bad in ((0, 8, 0), (3, 8, 0), (8, 4, 0), (4, 4, 1), (2, 2, 0), (2, 16, 0), (-1, 4, 0), (2, 8, 2),
                (2, 4, 0, 6), (2, 4, 0, -1)):
        with pytest.raises(MmsarError, match="INVALID_ARG"):
            p.set_tiles(*bad)
    assert p.tiles == (2, 8, 0, 0)   # the last valid setting stays


def test_wait_test_switch():
    """mmsar_plan_set_wait_test takes 0 or 1 (the GPU test of the timeout path
    is in test_gpu_timeout.py)."""
    from paper_2305_02064_gb300 import _lib
    from paper_2305_02064_gb300._lib import MmsarError
    p = _plan()
    for on in (1, 0):
        _lib.check(p._lib.mmsar_plan_set_wait_test(p._h, on))
    for bad in (2, -1):
        with pytest.raises(MmsarError, match="INVALID_ARG"):
            _lib.check(p._lib.mmsar_plan_set_wait_test(p._h, bad))
