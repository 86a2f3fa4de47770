"""GPU direct back-projection against the FP64 oracle's back-projection, and
its peaks against the RMA image's (the paper compares the two by image
peaks, Sec. V)."""
import numpy as np
import pytest

import synth
from oracle import bpa as obpa
from oracle import rma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _dev_args(scan, dev):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
            (scan.echo, np.asarray(scan.pos, np.float64), np.asarray(scan.tx, np.float64),
             np.asarray(scan.rx, np.float64))]


def test_bpa_full_grid_matches_oracle(dev, tiny_scan):
    from paper_2305_02064_gb300 import Plan
    plan = Plan.for_scan(tiny_scan)
    got = plan.backproject(*_dev_args(tiny_scan, dev)).cpu().numpy()
    ref = obpa.bpa(tiny_scan)
    assert rma.nmse(got, ref) < 1e-9
    assert rma.peak_index(got) == rma.peak_index(ref) == np.ravel_multi_index(
        tiny_scan.grid.centre_index(0.0, 0.0, 0.3), ref.shape)


def test_bpa_voxel_subset_on_realistic_geometry(dev):
    """Random voxels of the 2 Tx x 4 Rx serpentine geometry (Nk = 64 to keep
    the FP64 oracle quick) plus the scatterer voxels."""
    from paper_2305_02064_gb300 import Plan
    scan = synth.custom(nx_pos=40, ny_pos=40, nk=64, layout="awr1443", nx=64, ny=64, nz=16, dz=5e-3, z0=0.26,
                        seed=41, serp=True, jitter=(2e-3, 3e-3), n_points=4)
    plan = Plan.for_scan(scan)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(0, scan.grid.n_voxels, 200),
                          [np.ravel_multi_index(scan.grid.centre_index(*p[:3]), (64, 64, 16))
                           for p in scan.scatterers]])
    vox = obpa.voxel_centres(scan.grid, idx)
    got = plan.backproject(*_dev_args(scan, dev), voxels=torch.from_numpy(vox).to(dev)).cpu().numpy()
    ref = obpa.bpa(scan, idx)
    assert rma.nmse(got, ref) < 1e-9


def test_bpa_and_rma_agree_on_the_peak(dev):
    """A point target below the centre of a 48 x 48-position aperture with
    +-4 mm of z jitter: the compensated RMA image and the back-projection
    peak on the target voxel.  (Off the aperture centre the finite aperture
    skews the RMA's broad cross-range PSF -- 12 mm here -- by a voxel or two
    while back-projection, the matched filter, stays on the target.)"""
    from paper_2305_02064_gb300 import Plan
    scan = synth.custom(nx_pos=48, ny_pos=48, nk=32, layout="awr1443", nx=64, ny=64, nz=16, dz=5e-3, z0=0.26,
                        seed=43, jitter=(0.3e-3, 4e-3), scatterers=[[0.0, 0.0, 0.29, 1.0]])
    plan = Plan.for_scan(scan)
    args = _dev_args(scan, dev)
    b = plan.backproject(*args).cpu().numpy()
    ws, vol = plan.new_workspace(dev), plan.new_volume(dev)
    plan.image(ws, *args, vol)
    o = vol.cpu().numpy()
    pb = np.array(np.unravel_index(rma.peak_index(b), b.shape))
    po = np.array(np.unravel_index(rma.peak_index(o), o.shape))
    truth = np.array(scan.grid.centre_index(0.0, 0.0, 0.29))
    assert np.all(pb == truth)
    assert np.all(np.abs(po - truth) <= 1)
