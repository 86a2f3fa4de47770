"""Direct back-projection oracle (the paper's gold-standard baseline, Sec. III).

TEST INFRASTRUCTURE ONLY (see the package docstring).

o_BP(r) = sum_{t, r, p, k} s(t, r, p, k) exp(+j k (|T_tp - r| + |R_rp - r|)),
with the round-trip distance of Eq. 2 and k = 2 pi f / c (Eq. 9), evaluated
term by term in FP64.  It is a different operator from the RMA (no Eq. 7
approximation, no k_z weight), so it is compared with the RMA by peak
positions only.
"""
from __future__ import annotations

import numpy as np

from . import _native


def voxel_centres(grid, idx=None):
    """Centres of the voxels (all of them, or linear indices ``idx``) as [n, 3]."""
    if idx is None:
        idx = np.arange(grid.nx * grid.ny * grid.nz)
    idx = np.asarray(idx)
    i, rem = np.divmod(idx, grid.ny * grid.nz)
    j, q = np.divmod(rem, grid.nz)
    return np.stack([grid.x0 + i * grid.dx, grid.y0 + j * grid.dy, grid.z0 + q * grid.dz], 1)


def bpa(scan, idx=None):
    """Back-projected image at the voxels ``idx`` (default: all, shaped
    [nx, ny, nz])."""
    freq = scan.f0 + scan.df * np.arange(scan.echo.shape[3])
    vox = voxel_centres(scan.grid, idx)
    out = _native.bpa(scan.echo, scan.pos, scan.tx, scan.rx, freq, vox)
    if idx is None:
        return out.reshape(scan.grid.nx, scan.grid.ny, scan.grid.nz)
    return out
