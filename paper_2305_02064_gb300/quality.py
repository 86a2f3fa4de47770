"""Image-quality measures of a reconstructed point target (host side, numpy).

Used by the point-spread study (Sec. V-A: main-lobe widths along the cross
range y and the range z for growing deviation of the samples from the
reference plane) on volumes the library produced; nothing here touches the
device or the imaging path.
"""
from __future__ import annotations

import numpy as np


def _width(profile: np.ndarray, idx: int, level: float, pitch: float) -> float:
    """Width (same unit as pitch) of the main lobe of `profile` around its
    maximum at `idx` where it stays >= level, with linear interpolation of
    the two crossings; the lobe is cut at the ends of the profile."""
    n = profile.size
    lo = idx
    while lo > 0 and profile[lo - 1] >= level:
        lo -= 1
    hi = idx
    while hi < n - 1 and profile[hi + 1] >= level:
        hi += 1
    left = float(lo)
    if lo > 0:
        a, b = profile[lo - 1], profile[lo]
        left = lo - (b - level) / (b - a)
    right = float(hi)
    if hi < n - 1:
        a, b = profile[hi], profile[hi + 1]
        right = hi + (a - level) / (a - b)
    return (right - left) * pitch


def _pslr_db(profile: np.ndarray, idx: int) -> float:
    """Peak-to-sidelobe ratio: the largest value outside the main lobe
    (bounded by the first local minima on either side) over the peak, in dB."""
    n = profile.size
    lo = idx
    while lo > 0 and profile[lo - 1] <= profile[lo]:
        lo -= 1
    hi = idx
    while hi < n - 1 and profile[hi + 1] <= profile[hi]:
        hi += 1
    side = np.concatenate([profile[:lo], profile[hi + 1:]])
    if side.size == 0:
        return -np.inf
    return float(20.0 * np.log10(side.max() / profile[idx]))


def psf_metrics(vol: np.ndarray, grid, target) -> dict:
    """Point-target measures of |vol| ([nx][ny][nz], voxel (i, j, q) at
    x0 + i dx, y0 + j dy, z0 + q dz): the peak's offset from `target`
    (x, y, z in metres), its amplitude, the -3 dB main-lobe widths along y
    and z through the peak, and the peak-to-sidelobe ratio along y.
    Lengths are returned in millimetres."""
    a = np.abs(np.asarray(vol))
    i, j, q = np.unravel_index(int(np.argmax(a)), a.shape)
    peak = float(a[i, j, q])
    level = peak / np.sqrt(2.0)
    py = a[i, :, q]
    pz = a[i, j, :]
    return {
        "peak": peak,
        "peak_offset_y_mm": (grid.y0 + j * grid.dy - target[1]) * 1e3,
        "peak_offset_z_mm": (grid.z0 + q * grid.dz - target[2]) * 1e3,
        "width_y_mm": _width(py, j, level, grid.dy * 1e3),
        "width_z_mm": _width(pz, q, level, grid.dz * 1e3),
        "pslr_y_db": _pslr_db(py, j),
    }
