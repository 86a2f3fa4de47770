"""Seeded synthetic MIMO-SAR scans shaped like the paper's workloads.

This module is the one input source shared by the FP64 oracle and the CUDA
path.  It holds no arithmetic of the imaging method (no phase compensation,
no spectral transform): it builds radar layouts, scan trajectories and point
scenes, and evaluates the forward echo model of Sec. II-C, Eq. 9 (with P(f)=1
and, by default, no 1/(R_T R_R) amplitude) in a small C helper.

Workloads (all seeded with numpy's PCG64):

* ``tiny``      -- 1 Tx / 2 Rx, 16x16 jittered positions, Nk=32, 3 points,
                   30 dB SNR, 32x32x16 voxels (1 mm x 1 mm x 5 mm).
* ``realistic`` -- 2 Tx / 4 Rx (AWR1443-like, Sec. IV), 128x128 serpentine
                   random-walk scan, Nk=256, 200 points on a bar chart at
                   z in [0.25, 0.35] m, 256x256x64 voxels.
* ``large``     -- 3 Tx / 4 Rx, 256x256 positions, Nk=512, 2000 points in
                   z in [0.2, 0.5] m, 512x512x128 voxels.
* ``batch_mix`` -- uneven scans of the batched mix (32x32 .. 128x160
                   positions, Nk in {64,128,256}).
* ``custom``    -- any of the above knobs, for parity cases and edge cases.

Frequencies follow f_k = f0 + k*B/Nk (77-81 GHz, Sec. IV) and the carrier
wavelength is lambda_c = c / 79 GHz (Sec. V-A).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import tempfile
import threading

import numpy as np

C0 = 299792458.0
F0 = 77e9
BANDWIDTH = 4e9
F_CENTER = F0 + BANDWIDTH / 2
LAMBDA_C = C0 / F_CENTER

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the echo helper (gcc, OpenMP) next to its source; return the path."""
    src = os.path.join(_HERE, "echo.c")
    so = os.path.join(_HERE, "_echo.so")
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", src, "-o", tmp, "-lm"])
    os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.synth_echo.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                                           ctypes.c_int, dp, ctypes.c_int,
                                                           ctypes.POINTER(ctypes.c_float)]
            lib.synth_echo.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclasses.dataclass
class Grid:
    """Voxel grid: centres x0 + i*dx (i < nx), likewise y and z."""
    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    nx: int
    ny: int
    nz: int

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    def centre_index(self, x: float, y: float, z: float):
        return (int(round((x - self.x0) / self.dx)), int(round((y - self.y0) / self.dy)),
                int(round((z - self.z0) / self.dz)))


@dataclasses.dataclass
class Scan:
    """One synthetic scan: echo s[t][r][p][k] (complex64) plus its geometry."""
    echo: np.ndarray          # complex64 [T, R, P, Nk]
    pos: np.ndarray           # float64 [P, 3] radar reference point per position (m)
    tx: np.ndarray            # float64 [T, 3] Tx offsets from the reference point (m)
    rx: np.ndarray            # float64 [R, 3] Rx offsets (m)
    f0: float                 # first frequency (Hz)
    df: float                 # frequency step (Hz)
    grid: Grid
    scatterers: np.ndarray    # float64 [S, 4] (x, y, z, sigma), the truth
    name: str = "custom"
    seed: int = 0

    @property
    def shape(self):
        return self.echo.shape

    @property
    def n_k(self) -> int:
        return self.echo.shape[3]

    @property
    def freqs(self) -> np.ndarray:
        return self.f0 + self.df * np.arange(self.n_k)


def echo(pos, tx, rx, f0, df, n_k, scatterers, amplitude=False) -> np.ndarray:
    """Evaluate the Eq. 9 forward model; returns complex64 [T, R, P, Nk]."""
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
    tx = np.ascontiguousarray(tx, np.float64).reshape(-1, 3)
    rx = np.ascontiguousarray(rx, np.float64).reshape(-1, 3)
    sc = np.ascontiguousarray(scatterers, np.float64).reshape(-1, 4)
    T, R, P = tx.shape[0], rx.shape[0], pos.shape[0]
    out = np.zeros((T, R, P, n_k, 2), np.float32)
    if T * R * P == 0:
        return out.view(np.complex64)[..., 0]
    rc = _lib().synth_echo(T, R, P, int(n_k), _dp(pos), _dp(tx), _dp(rx), float(f0), float(df),
                           sc.shape[0], _dp(sc), int(bool(amplitude)),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if rc != 0:
        raise ValueError("synth_echo rejected its arguments")
    return out.view(np.complex64)[..., 0]


def add_noise(s: np.ndarray, snr_db: float, rng: np.random.Generator) -> np.ndarray:
    """Complex Gaussian noise with variance mean|s|^2 / 10^(SNR/10), split over re/im."""
    p = float(np.mean(np.abs(s.astype(np.complex128)) ** 2))
    var = p / 10 ** (snr_db / 10)
    sd = np.sqrt(var / 2)
    n = rng.normal(0, sd, s.shape) + 1j * rng.normal(0, sd, s.shape)
    return (s + n).astype(np.complex64)


# ----------------------------------------------------------------------------- layouts
def layout_tiny():
    lam = LAMBDA_C
    tx = np.array([[0.0, -lam, 0.0]])
    rx = np.array([[0.0, 0.0, 0.0], [0.0, lam / 2, 0.0]])
    return tx, rx


def layout_awr1443():
    """2 Tx / 4 Rx: Rx at y = {0, .5, 1, 1.5} lambda, Tx at y = {-2.5, -0.5} lambda."""
    lam = LAMBDA_C
    tx = np.array([[0.0, -2.5 * lam, 0.0], [0.0, -0.5 * lam, 0.0]])
    rx = np.array([[0.0, a * lam, 0.0] for a in (0.0, 0.5, 1.0, 1.5)])
    return tx, rx


def layout_3x4():
    lam = LAMBDA_C
    tx = np.array([[0.0, a * lam, 0.0] for a in (-4.0, -2.0, 0.0)])
    rx = np.array([[0.0, a * lam, 0.0] for a in (0.0, 0.5, 1.0, 1.5)])
    return tx, rx


# ----------------------------------------------------------------------------- trajectories
def jittered_grid(nx, ny, pitch, jit_xy, jit_z, rng):
    """Regular nx*ny grid centred at 0 with independent uniform jitter."""
    xs = (np.arange(nx) - (nx - 1) / 2) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2) * pitch
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    P = nx * ny
    pos = np.stack([X.ravel(), Y.ravel(), np.zeros(P)], 1)
    pos[:, 0] += rng.uniform(-jit_xy, jit_xy, P)
    pos[:, 1] += rng.uniform(-jit_xy, jit_xy, P)
    pos[:, 2] += rng.uniform(-jit_z, jit_z, P)
    return pos


def _smooth_walk(n, rng, bound, corr=24):
    """Gaussian random walk, low-pass filtered, rescaled to max |.| = bound."""
    if n == 0 or bound == 0:
        return np.zeros(n)
    inc = rng.normal(size=n + 4 * corr)
    walk = np.cumsum(inc)
    ker = np.exp(-0.5 * (np.arange(-2 * corr, 2 * corr + 1) / corr) ** 2)
    ker /= ker.sum()
    sm = np.convolve(walk, ker, mode="same")[2 * corr:2 * corr + n]
    sm = sm - sm.mean()
    m = np.max(np.abs(sm))
    return sm * (bound / m) if m > 0 else sm


def serpentine(nx, ny, pitch, wander_xy, wander_z, rng):
    """Serpentine raster (rows along x alternate direction, rows step in y)
    with a smooth random-walk wander: a stand-in for the paper's
    'semi-smooth random curve' freehand trajectories (Sec. V-A)."""
    xs = (np.arange(nx) - (nx - 1) / 2) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2) * pitch
    pts = []
    for j, y in enumerate(ys):
        row = xs if j % 2 == 0 else xs[::-1]
        pts.extend((x, y) for x in row)
    pos = np.zeros((nx * ny, 3))
    pos[:, :2] = np.array(pts)
    P = nx * ny
    pos[:, 0] += _smooth_walk(P, rng, wander_xy)
    pos[:, 1] += _smooth_walk(P, rng, wander_xy)
    pos[:, 2] += _smooth_walk(P, rng, wander_z)
    return pos


# ----------------------------------------------------------------------------- scenes
def bar_chart(n_points, grid: Grid, z_lo, z_hi, half_width, rng):
    """Point scatterers on bar groups of decreasing spacing (a generic
    resolution chart), each group on one voxel-centre z plane."""
    pts = []
    spacings = [8, 6, 5, 4, 3, 2]
    qlo = int(np.ceil((z_lo - grid.z0) / grid.dz))
    qhi = int(np.floor((z_hi - grid.z0) / grid.dz))
    ci, cj = grid.nx // 2, grid.ny // 2
    hw = int(half_width / grid.dx)
    g = 0
    while len(pts) < n_points:
        sp = spacings[g % len(spacings)]
        q = int(rng.integers(qlo, qhi + 1))
        i0 = int(rng.integers(ci - hw, ci + hw - 4 * sp + 1))
        j0 = int(rng.integers(cj - hw, cj + hw - 8 + 1))
        horizontal = g % 2 == 0
        for b in range(4):          # 4 bars
            for s in range(8):      # 8 points per bar
                if len(pts) >= n_points:
                    break
                i, j = (i0 + b * sp, j0 + s) if horizontal else (i0 + s, j0 + b * sp)
                if not (0 <= i < grid.nx and 0 <= j < grid.ny):
                    continue
                pts.append((grid.x0 + i * grid.dx, grid.y0 + j * grid.dy, grid.z0 + q * grid.dz,
                            rng.uniform(0.5, 1.0)))
        g += 1
    return np.array(pts[:n_points])


def random_points(n_points, grid: Grid, z_lo, z_hi, half_width, rng):
    ci, cj = grid.nx // 2, grid.ny // 2
    hw = int(half_width / grid.dx)
    i = rng.integers(ci - hw, ci + hw + 1, n_points)
    j = rng.integers(cj - hw, cj + hw + 1, n_points)
    qlo = int(np.ceil((z_lo - grid.z0) / grid.dz))
    qhi = int(np.floor((z_hi - grid.z0) / grid.dz))
    q = rng.integers(qlo, qhi + 1, n_points)
    return np.stack([grid.x0 + i * grid.dx, grid.y0 + j * grid.dy, grid.z0 + q * grid.dz,
                     rng.uniform(0.5, 1.0, n_points)], 1)


def centred_grid(nx, ny, nz, dx, dz, z0) -> Grid:
    """Voxel grid whose x/y centre voxel (index n//2) sits at 0."""
    return Grid(-(nx // 2) * dx, -(ny // 2) * dx, z0, dx, dx, dz, nx, ny, nz)


# ----------------------------------------------------------------------------- workloads
def tiny(seed: int = 0) -> Scan:
    rng = np.random.default_rng(seed)
    tx, rx = layout_tiny()
    nk = 32
    pos = jittered_grid(16, 16, 1e-3, 0.5e-3, 1e-3, rng)
    grid = centred_grid(32, 32, 16, 1e-3, 5e-3, 0.260)
    sc = np.array([[-5e-3, -5e-3, 0.300, 1.0], [0.0, 0.0, 0.300, 1.0], [5e-3, 5e-3, 0.300, 1.0]])
    s = echo(pos, tx, rx, F0, BANDWIDTH / nk, nk, sc)
    s = add_noise(s, 30.0, rng)
    return Scan(s, pos, tx, rx, F0, BANDWIDTH / nk, grid, sc, "tiny", seed)


def realistic(seed: int = 2000, n_points: int = 200) -> Scan:
    rng = np.random.default_rng(seed)
    tx, rx = layout_awr1443()
    nk = 256
    pos = serpentine(128, 128, 1e-3, 2e-3, 3e-3, rng)
    grid = centred_grid(256, 256, 64, 1e-3, 3.125e-3, 0.200)
    sc = bar_chart(n_points, grid, 0.25, 0.35, 0.055, rng)
    s = echo(pos, tx, rx, F0, BANDWIDTH / nk, nk, sc)
    return Scan(s, pos, tx, rx, F0, BANDWIDTH / nk, grid, sc, "realistic", seed)


def large(seed: int = 5000, n_points: int = 2000) -> Scan:
    rng = np.random.default_rng(seed)
    tx, rx = layout_3x4()
    nk = 512
    pos = serpentine(256, 256, 1e-3, 2e-3, 3e-3, rng)
    grid = centred_grid(512, 512, 128, 1e-3, 3.125e-3, 0.150)
    sc = random_points(n_points, grid, 0.2, 0.5, 0.12, rng)
    s = echo(pos, tx, rx, F0, BANDWIDTH / nk, nk, sc)
    return Scan(s, pos, tx, rx, F0, BANDWIDTH / nk, grid, sc, "large", seed)


def psf_track(dz_max: float, seed: int = 4000, n_pos: int = 256, nk: int = 64) -> Scan:
    """The point-spread study of Sec. V-A: a linear MIMO array (2 Tx x 4 Rx
    along y) moved along y over y' in [-12.5, 12.5] cm at x = 0 in n_pos
    steps, on a semi-smooth random z track around the plane Z_0 = 0 whose
    largest deviation |d^z| is dz_max; one unit point target at (0, 0, 0.5 m).
    Image: the y-z plane x = 0, 256 x 64 voxels at 1 x 2.5 mm centred on the
    target.  The single x column has a coarse x pitch (0.5 m), so the spectral
    x grid collapses to k_x ~ 0 and the 3-D transform reduces to the 2-D (y, z)
    one of a linear aperture (a finer x grid would add near-evanescent k_x
    columns that the linear aperture does not resolve)."""
    rng = np.random.default_rng(seed)
    tx, rx = layout_awr1443()
    pos = np.zeros((n_pos, 3))
    pos[:, 1] = np.linspace(-0.125, 0.125, n_pos)
    pos[:, 2] = _smooth_walk(n_pos, rng, dz_max)
    grid = Grid(0.0, -0.128, 0.5 - 32 * 2.5e-3, 0.5, 1e-3, 2.5e-3, 1, 256, 64)
    sc = np.array([[0.0, 0.0, 0.5, 1.0]])
    s = echo(pos, tx, rx, F0, BANDWIDTH / nk, nk, sc)
    return Scan(s, pos, tx, rx, F0, BANDWIDTH / nk, grid, sc, f"psf dz_max={dz_max:g}", seed)


def custom(nx_pos=16, ny_pos=16, nk=32, layout="tiny", nx=32, ny=32, nz=16, dx=1e-3, dz=5e-3,
           z0=0.26, scatterers=None, n_points=3, jitter=(0.5e-3, 1e-3), serp=False,
           snr_db=None, seed=0, amplitude=False) -> Scan:
    """Free-form scan for parity and edge cases (ragged sizes, odd Nk ...)."""
    rng = np.random.default_rng(seed)
    tx, rx = {"tiny": layout_tiny, "awr1443": layout_awr1443, "3x4": layout_3x4}[layout]()
    if serp:
        pos = serpentine(nx_pos, ny_pos, 1e-3, jitter[0], jitter[1], rng)
    else:
        pos = jittered_grid(nx_pos, ny_pos, 1e-3, jitter[0], jitter[1], rng)
    grid = centred_grid(nx, ny, nz, dx, dz, z0)
    if scatterers is None:
        hw = min(nx_pos, ny_pos) * 1e-3 / 2
        mz = min(2, (nz - 1) // 2)
        scatterers = random_points(n_points, grid, z0 + mz * dz, z0 + (nz - 1 - mz) * dz, hw, rng)
    scatterers = np.asarray(scatterers, np.float64).reshape(-1, 4)
    s = echo(pos, tx, rx, F0, BANDWIDTH / nk, nk, scatterers, amplitude)
    if snr_db is not None:
        s = add_noise(s, snr_db, rng)
    return Scan(s, pos, tx, rx, F0, BANDWIDTH / nk, grid, scatterers, "custom", seed)


def batch_mix(n_scans: int = 64, seed0: int = 3000):
    """The uneven batched mix: positions 32x32..128x160, Nk in {64,128,256},
    2Tx x 4Rx, random-walk trajectories, 20-200 points.  Output grids are
    2*n_pos per axis (rounded to a power of two here), Nz = 64."""
    scans = []
    for i in range(n_scans):
        rng = np.random.default_rng(seed0 + i)
        npx = int(rng.choice(np.arange(32, 129, 16)))
        npy = int(rng.choice(np.arange(32, 161, 16)))
        nk = int(rng.choice([64, 128, 256]))
        tx, rx = layout_awr1443()
        pos = serpentine(npx, npy, 1e-3, 2e-3, 3e-3, rng)
        nx = 1 << int(np.ceil(np.log2(2 * npx)))
        ny = 1 << int(np.ceil(np.log2(2 * npy)))
        grid = Grid(-(nx // 2) * 1e-3, -(ny // 2) * 1e-3, 0.2, 1e-3, 1e-3, 3.125e-3, nx, ny, 64)
        npts = int(rng.integers(20, 201))
        sc = random_points(npts, grid, 0.22, 0.38, min(npx, npy) * 0.4e-3, rng)
        s = echo(pos, tx, rx, F0, BANDWIDTH / nk, nk, sc)
        scans.append(Scan(s, pos, tx, rx, F0, BANDWIDTH / nk, grid, sc, "batch_mix", seed0 + i))
    return scans
