"""GPU parity at the plan's size limits, against the FP64 oracle.

Every kernel instance the plan can select is run here on a scan small
enough for the exact oracle (or the fast oracle, itself pinned to the exact
sums): the 512-point Stolt grid (nz 129..256), the largest frequency counts
(Nk up to 1024, even, odd and not a multiple of 32), the largest spectral
grid on both axes together (Mx = My = 1024: FFTs of 2048 points along x'
and y', inverse FFTs of 1024 points along k_y and k_x), and the wider
Gaussian kernels (w = 8, 10, 12: Stolt register windows of 10, 12 and 14
points) on a scan that spans many gridding tiles.

Tolerances: the contract is NMSE <= 1e-4 (FP32 path); each test also
asserts the bound derived from the Gaussian gridding error of its kernel
width (three transforms, x10 margin: 2e-5 at w = 6, 2e-7 at w = 8, the FP32
floor of 1e-8 beyond), as the other parity tests do.
"""
import numpy as np
import pytest

import synth
from oracle import rma

from test_gpu_parity import CONTRACT, assert_parity, dev, near_tie, run_gpu  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND_WIDE = {8: 2e-7, 10: 1e-8, 12: 1e-8}


def exact(scan, **kw):
    return rma.rma_exact(rma.setup_from(scan, **kw))


@pytest.mark.parametrize("nz", [129, 200, 256])
def test_deepest_z_grids(dev, nz):
    """nz in 129..256 selects the 512-point z gridding grid of the Stolt step."""
    scan = synth.custom(nx_pos=6, ny_pos=5, nk=24, layout="awr1443", nx=16, ny=16, nz=nz, dz=2e-3, z0=0.1,
                        seed=nz, n_points=4)
    got, plan = run_gpu(scan, dev)
    assert plan.kernel_width == 6
    assert_parity(got, exact(scan), plan.kernel_width)


TC = (2, 4, 0, 2)   # tensor-core gridding (staged)
WS = (2, 4, 0, 5)   # tensor-core gridding (warp-specialised)


def run_with(scan, dev, tiles=None, **plan_kw):
    """run_gpu with an explicit gridding form."""
    if tiles is None:
        return run_gpu(scan, dev, **plan_kw)
    from paper_2305_02064_gb300 import Plan
    plan = Plan.for_scan(scan, **plan_kw)
    plan.set_tiles(*tiles)
    ws = plan.new_workspace(dev)
    vol = torch.full(plan.volume_shape, complex(np.nan, np.nan), dtype=torch.complex64, device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    plan.image(ws, t(scan.echo), t(np.asarray(scan.pos, np.float64)), t(np.asarray(scan.tx, np.float64)),
               t(np.asarray(scan.rx, np.float64)), vol)
    plan.poll_error(ws)
    return vol.cpu().numpy(), plan


@pytest.mark.parametrize("tiles", [None, TC, WS], ids=["fp32", "tc", "ws"])
@pytest.mark.parametrize("nk", [1024, 1000, 1023])
def test_largest_frequency_counts(dev, nk, tiles):
    """Nk at the limit (1024: sixteen 64-frequency groups), below it (1000,
    even), odd and ragged (1023), for both gridding forms."""
    scan = synth.custom(nx_pos=4, ny_pos=4, nk=nk, layout="tiny", nx=16, ny=16, nz=8, seed=nk, snr_db=30)
    got, plan = run_with(scan, dev, tiles)
    assert_parity(got, exact(scan), plan.kernel_width)


def test_too_many_frequencies_are_refused(dev):
    from paper_2305_02064_gb300 import MmsarError, Plan
    g = synth.centred_grid(16, 16, 8, 1e-3, 5e-3, 0.26)
    with pytest.raises(MmsarError, match="UNSUPPORTED_SIZE"):
        Plan(1, 2, 16, 1025, 77e9, 4e6, g)
    with pytest.raises(MmsarError, match="UNSUPPORTED_SIZE"):
        Plan(1, 2, 16, 32, 77e9, 1e8, synth.centred_grid(16, 16, 257, 1e-3, 5e-3, 0.26))


@pytest.mark.parametrize("tiles", [None, TC, WS], ids=["fp32", "tc", "ws"])
def test_largest_spectral_grid_on_both_axes(dev, tiles):
    """Mx = My = 1024 (the plan's largest) on a small voxel grid: 2048-point
    FFTs along x' and y', 1024-point inverse FFTs along k_y and k_x, a
    2048 x 2048 gridding grid."""
    scan = synth.custom(nx_pos=4, ny_pos=4, nk=8, layout="tiny", nx=24, ny=20, nz=6, seed=41, jitter=(0.5e-3, 1e-3))
    got, plan = run_with(scan, dev, tiles, mx=1024, my=1024)
    assert (plan.mx, plan.my) == (1024, 1024)
    ref = rma.rma_exact(rma.setup_from(scan, Mx=1024, My=1024))
    assert_parity(got, ref, plan.kernel_width)


@pytest.mark.slow
def test_largest_voxel_grid(dev):
    """A 1024 x 1024 voxel grid (Mx = My = 1024 by default) against the fast
    oracle (FP64 Gaussian gridding, w = 16)."""
    scan = synth.custom(nx_pos=8, ny_pos=8, nk=8, layout="tiny", nx=1024, ny=1024, nz=4, dz=8e-3, z0=0.27,
                        seed=43, jitter=(0.5e-3, 1e-3), n_points=3)
    got, plan = run_gpu(scan, dev)
    assert (plan.mx, plan.my) == (1024, 1024)
    ref = rma.rma_fast(rma.setup_from(scan), w=16)
    assert_parity(got, ref, plan.kernel_width)


def _multi_tile_scan():
    # 64 x 64 voxels: a 128 x 128 gridding grid of 8 x 8-cell tiles, samples
    # wrapping around the periodic window (as in the parity suite)
    return synth.custom(nx_pos=40, ny_pos=36, nk=48, layout="awr1443", nx=64, ny=64, nz=24, dz=4e-3, z0=0.24,
                        seed=21, serp=True, jitter=(1.5e-3, 3e-3), n_points=6)


@pytest.fixture(scope="module")
def multi_tile():
    scan = _multi_tile_scan()
    return scan, rma.rma_fast(rma.setup_from(scan), w=16)


@pytest.mark.parametrize("tiles", [None, TC, WS], ids=["fp32", "tc", "ws"])
@pytest.mark.parametrize("tol,w", [(1e-4, 8), (1e-5, 10), (1e-6, 12)])
def test_wide_kernels_on_many_tiles(dev, multi_tile, tol, w, tiles):
    scan, ref = multi_tile
    got, plan = run_with(scan, dev, tiles, nufft_tol=tol)
    assert plan.kernel_width == w
    e = assert_parity(got, ref, w, contract=CONTRACT)
    assert e <= BOUND_WIDE[w], (e, w)


def test_stolt_phase_at_the_deepest_scene(dev):
    """The k_z phase of Eq. 15 grows with the depth below the plane (about
    270 turns at 0.5 m for the upper band edge).  One point at 0.5 m, the
    widest kernel (w = 12, gridding error ~1e-13 in NMSE) and the exact
    oracle: what remains is the arithmetic of the k_z phase."""
    scan = synth.custom(nx_pos=12, ny_pos=12, nk=64, layout="awr1443", nx=16, ny=16, nz=32, dz=3.125e-3,
                        z0=0.45, seed=5, scatterers=[[0.0, 0.0, 0.5, 1.0]], jitter=(0.5e-3, 1e-3))
    got, plan = run_gpu(scan, dev, nufft_tol=1e-6)
    assert plan.kernel_width == 12
    ref = exact(scan)
    e = rma.nmse(got, ref)
    assert e <= 1e-7, e
    assert rma.peak_index(got) == rma.peak_index(ref)
