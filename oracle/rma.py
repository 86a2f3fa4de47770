"""FP64 CPU oracle for multi-planar multistatic compensation + planar RMA.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA library and imports nothing from it.

Two oracles of the same operator (Sec. II-C and Sec. III of the paper):

``rma_exact``  -- the paper's pipeline with every resampling replaced by its
                  exact definition: compensation (Eq. 11-12), the 2-D Fourier
                  transform of the non-uniform virtual-array samples written as
                  a direct sum (FT_2D of Eq. 16), the k_z weight and phase of
                  Eq. 15, the Stolt step plus inverse transform over k_z written
                  as the exact sum over the non-uniform k_z samples, and the
                  inverse 2-D transform over (k_x, k_y).  Cost ~ M^2 L Nk.
``rma_fast``   -- the same steps in the order the paper gives, with the two
                  non-uniform transforms done by fast Gaussian gridding
                  (Greengard-Lee FGG NUFFT, named in Sec. III for "the Fourier
                  transforms and Stolt interpolation") at a high-accuracy
                  kernel width (default w = 16: relative error ~1e-8 per
                  transform) and library FFTs.

Conventions (the paper leaves these open; the readings are fixed here and
used identically by the CUDA path, which implements them independently):

* Virtual element (Eq. 3-4): x' = (x_T + x_R)/2, y' = (y_T + y_R)/2,
  d^x = x_R - x_T, d^y = y_R - y_T, z_l = (z_T + z_R)/2, d^z = z_l - z_ref.
* +z points from the scan plane toward the scene, so the scene lies at
  z > z_ref and Z_c = z_scene - z_ref > 0.  Then the Eq. 5 expansion on axis
  reads R^RT ~ 2 R_0 - 2 d^z + (d^x^2 + d^y^2)/(4 Z_c), and the residual of
  Eq. 12 is beta = -2 d^z + (d^x^2 + d^y^2) / (4 Z_c).  (Eq. 7 as printed has
  +2 d^z because it puts the plane at z = +Z_0 above a target at the origin.)
* Compensation (Eq. 11): s_hat = s * exp(+j k beta), k = 2 pi f / c (Eq. 9).
* Spectral grid: m in [-Mx/2, Mx/2), k_x = 2 pi m / (Mx dx); likewise y.
  Positions are taken relative to the grid centre x_c = x0 + (nx//2) dx.
  Forward kernel exp(-j(k_x x' + k_y y')), inverse kernel exp(+j ...).
* k_z = sqrt(4k^2 - k_x^2 - k_y^2) (Eq. 14); evanescent terms
  (4k^2 <= k_x^2 + k_y^2) are dropped.
* Eq. 15 with P(f) = 1 and the phase taken against the scan plane:
  weight k_z * exp(+j k_z (z_q - z_ref)).  No Stolt Jacobian.
* Normalisation 1/(T R P Nk); no density compensation.
* Defaults: z_ref = mean of z_l over all samples; z_scene = z0 + (nz-1)/2 dz;
  Mx, My = next power of two >= nx, ny.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import _native

C0 = 299792458.0


def next_pow2(n: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, n)))))


@dataclasses.dataclass
class Setup:
    """Everything the operator needs, in plain numpy arrays and scalars."""
    echo: np.ndarray        # complex [T, R, P, Nk]
    pos: np.ndarray         # [P, 3]
    tx: np.ndarray          # [T, 3]
    rx: np.ndarray          # [R, 3]
    f0: float
    df: float
    x0: float
    y0: float
    z0: float
    dx: float
    dy: float
    dz: float
    nx: int
    ny: int
    nz: int
    z_ref: float
    z_scene: float
    compensate: int         # 0 none, 1 Eq. 7 residual (paper), 2 Eq. 5 at the scene centre
    Mx: int
    My: int

    @property
    def n_k(self):
        return self.echo.shape[3]

    @property
    def wavenumbers(self):
        """k = 2 pi f / c (Eq. 9) on f_k = f0 + k df."""
        return 2 * np.pi * (self.f0 + self.df * np.arange(self.n_k)) / C0

    @property
    def x_c(self):
        return self.x0 + (self.nx // 2) * self.dx

    @property
    def y_c(self):
        return self.y0 + (self.ny // 2) * self.dy

    @property
    def n_total(self):
        return int(np.prod(self.echo.shape))


def setup_from(scan, z_ref=None, z_scene=None, compensate=True, Mx=None, My=None,
               echo=None) -> Setup:
    """Build a Setup from any object with echo/pos/tx/rx/f0/df/grid attributes."""
    g = scan.grid
    e = np.asarray(scan.echo if echo is None else echo)
    pos = np.asarray(scan.pos, np.float64).reshape(-1, 3)
    tx = np.asarray(scan.tx, np.float64).reshape(-1, 3)
    rx = np.asarray(scan.rx, np.float64).reshape(-1, 3)
    if z_ref is None or (isinstance(z_ref, float) and math.isnan(z_ref)):
        z_ref = default_z_ref(pos, tx, rx)
    if z_scene is None or (isinstance(z_scene, float) and math.isnan(z_scene)):
        z_scene = g.z0 + 0.5 * (g.nz - 1) * g.dz
    return Setup(e, pos, tx, rx, float(scan.f0), float(scan.df), g.x0, g.y0, g.z0, g.dx, g.dy, g.dz,
                 g.nx, g.ny, g.nz, float(z_ref), float(z_scene), int(compensate),
                 int(Mx or next_pow2(g.nx)), int(My or next_pow2(g.ny)))


def default_z_ref(pos, tx, rx) -> float:
    """Mean of z_l over all (t, r, p) samples."""
    if pos.shape[0] == 0:
        return 0.0
    return float(pos[:, 2].mean() + 0.5 * (tx[:, 2].mean() + rx[:, 2].mean()))


# ----------------------------------------------------------------------------- Sec. II
def virtual_elements(pos, tx, rx):
    """Eq. 3-4: virtual element (x', y'), separations d^x, d^y and the sample
    plane z_l for every (t, r, p); each output has shape [T, R, P]."""
    T = pos[None, None, :, :] + tx[:, None, None, :]
    R = pos[None, None, :, :] + rx[None, :, None, :]
    T, R = np.broadcast_arrays(T, R)
    xv = 0.5 * (T[..., 0] + R[..., 0])
    yv = 0.5 * (T[..., 1] + R[..., 1])
    zl = 0.5 * (T[..., 2] + R[..., 2])
    dxl = R[..., 0] - T[..., 0]
    dyl = R[..., 1] - T[..., 1]
    return xv, yv, zl, dxl, dyl


def residual_beta(dxl, dyl, dzl, Zc):
    """Eq. 12 (sign per the +z-toward-scene reading): the near-field residual
    beta = -2 d^z + (d^x^2 + d^y^2) / (4 Z_c)."""
    return -2.0 * dzl + (dxl * dxl + dyl * dyl) / (4.0 * Zc)


def residual_beta_scene(xv, yv, dxl, dyl, dzl, x_s, y_s, Zc):
    """Eq. 5 evaluated at a scatterer at the scene centre (x_s, y_s, z_ref + Z_c)
    for a virtual element at (x', y', z_ref): the second-order round-trip
    residual R^RT - 2 R_0 with the off-axis terms that Eq. 7 drops.  With +z
    toward the scene, Z_0 - z of Eq. 5 is -Z_c:
        R_0 = sqrt((x' - x_s)^2 + (y' - y_s)^2 + Z_c^2)
        beta = -2 Z_c d^z / R_0 + (d^x^2 + d^y^2 + 4 d^z^2) / (4 R_0)
               - [((x' - x_s) d^x + (y' - y_s) d^y)^2 + 4 Z_c^2 d^z^2] / (4 R_0^3)
    On axis (x' = x_s, y' = y_s, R_0 = Z_c) it reduces to residual_beta."""
    ax, ay = xv - x_s, yv - y_s
    R0 = np.sqrt(ax * ax + ay * ay + Zc * Zc)
    cross = ax * dxl + ay * dyl
    return (-2.0 * Zc * dzl / R0 + (dxl * dxl + dyl * dyl + 4.0 * dzl * dzl) / (4.0 * R0)
            - (cross * cross + 4.0 * Zc * Zc * dzl * dzl) / (4.0 * R0 ** 3))


def compensate(su: Setup):
    """Eq. 11: s_hat(x', y', f) = s * exp(+j k beta_l).  Returns (s_hat [L, Nk],
    x' [L], y' [L]) with the samples flattened in (t, r, p) order.  beta is
    Eq. 12's residual (compensate = 1), or Eq. 5's at the scene centre
    (compensate = 2); none for 0."""
    xv, yv, zl, dxl, dyl = virtual_elements(su.pos, su.tx, su.rx)
    L = xv.size
    s = su.echo.reshape(L, su.n_k).astype(np.complex128)
    Zc = su.z_scene - su.z_ref
    if su.compensate == 1:
        beta = residual_beta(dxl, dyl, zl - su.z_ref, Zc).ravel()
    elif su.compensate == 2:
        beta = residual_beta_scene(xv, yv, dxl, dyl, zl - su.z_ref, su.x_c, su.y_c, Zc).ravel()
    else:
        beta = None
    if beta is not None:
        s = s * np.exp(1j * np.outer(beta, su.wavenumbers))
    return s, xv.ravel(), yv.ravel()


# ----------------------------------------------------------------------------- Sec. III, exact
def spectral_axes(su: Setup):
    m = np.arange(-su.Mx // 2, su.Mx // 2)
    n = np.arange(-su.My // 2, su.My // 2)
    return 2 * np.pi * m / (su.Mx * su.dx), 2 * np.pi * n / (su.My * su.dy)


def spectrum_exact(su: Setup, shat=None, xv=None, yv=None, cols=None):
    """FT_2D of Eq. 16 as the direct sum over the non-uniform samples:
    S(m, n, k) = sum_l s_hat_l(k) exp(-j (k_x,m (x'_l - x_c) + k_y,n (y'_l - y_c))).
    Returns [Mx, My, Nk], or [len(cols), Nk] for a list of (m_index, n_index)
    (indices into the centred axes, 0 <= m_index < Mx)."""
    if shat is None:
        shat, xv, yv = compensate(su)
    kx, ky = spectral_axes(su)
    if cols is not None:
        cols = np.asarray(cols).reshape(-1, 2)
        ph = np.exp(-1j * (np.outer(kx[cols[:, 0]], xv - su.x_c) + np.outer(ky[cols[:, 1]], yv - su.y_c)))
        return ph @ shat
    Ex = np.exp(-1j * np.outer(kx, xv - su.x_c))     # [Mx, L]
    Ey = np.exp(-1j * np.outer(ky, yv - su.y_c))     # [My, L]
    S = np.empty((su.Mx, su.My, su.n_k), np.complex128)
    for k in range(su.n_k):
        S[:, :, k] = (Ex * shat[:, k]) @ Ey.T
    return S


def kz_filter(su: Setup, kx, ky):
    """Eq. 14: k_z = sqrt(4k^2 - k_x^2 - k_y^2) on [len(kx), len(ky), Nk] and
    the propagating mask (evanescent terms are dropped)."""
    k = su.wavenumbers
    kz2 = 4 * k[None, None, :] ** 2 - kx[:, None, None] ** 2 - ky[None, :, None] ** 2
    valid = kz2 > 0
    return np.sqrt(np.where(valid, kz2, 0.0)), valid


def stolt_exact(su: Setup, S, kx=None, ky=None):
    """Eq. 15 (P = 1) followed by the inverse transform over the non-uniform
    k_z samples, written as its exact sum:
    Z(m, n, q) = sum_k S(m, n, k) k_z exp(+j k_z (z_q - z_ref))."""
    if kx is None:
        kx, ky = spectral_axes(su)
    kz, valid = kz_filter(su, kx, ky)
    zq = su.z0 + su.dz * np.arange(su.nz)
    W = np.where(valid, S * kz, 0.0)
    Z = np.zeros(S.shape[:2] + (su.nz,), np.complex128)
    for q in range(su.nz):
        Z[:, :, q] = np.sum(W * np.exp(1j * kz * (zq[q] - su.z_ref)), axis=2)
    return Z


def image_from_Z(su: Setup, Z):
    """IFT over (k_x, k_y) of Eq. 16 as the direct sum, then 1/(T R P Nk):
    o(i, j, q) = (1/N) sum_{m,n} Z(m, n, q) exp(+j (k_x (x_i - x_c) + k_y (y_j - y_c)))."""
    kx, ky = spectral_axes(su)
    xi = su.x0 + su.dx * np.arange(su.nx) - su.x_c
    yj = su.y0 + su.dy * np.arange(su.ny) - su.y_c
    Fx = np.exp(1j * np.outer(xi, kx))   # [nx, Mx]
    Fy = np.exp(1j * np.outer(yj, ky))   # [ny, My]
    o = np.einsum("im,mnq->inq", Fx, Z)
    o = np.einsum("jn,inq->ijq", Fy, o)
    N = su.n_total
    return o / N if N else o * 0


def rma_exact(su: Setup):
    """The whole operator with exact transforms; complex128 [nx, ny, nz]."""
    if su.n_total == 0:
        return np.zeros((su.nx, su.ny, su.nz), np.complex128)
    S = spectrum_exact(su)
    return image_from_Z(su, stolt_exact(su, S))


# ----------------------------------------------------------------------------- Sec. III, FGG
def fgg_tau(M: int, w: int, sigma: float = 2.0) -> float:
    """Greengard-Lee Gaussian variance for M modes, oversampling sigma and a
    kernel of w points per axis (half-width M_sp = w/2)."""
    return math.pi * (w / 2) / (M * M * sigma * (sigma - 0.5))


def fgg_type1_2d(c, xr, yr, Mx, My, w):
    """F(m, n, :) = sum_l c_l exp(-j (m xr_l + n yr_l)), m in [-Mx/2, Mx/2),
    by Gaussian gridding on a 2Mx x 2My periodic grid + FFT + deconvolution.
    Returns [Mx, My, Nk]."""
    Nk = c.shape[1]
    Mrx, Mry = 2 * Mx, 2 * My
    tx_, ty_ = fgg_tau(Mx, w), fgg_tau(My, w)
    G = np.zeros((Mry, Mrx, Nk), np.complex128)
    _native.spread2d(np.ascontiguousarray(xr, np.float64), np.ascontiguousarray(yr, np.float64),
                     np.ascontiguousarray(c, np.complex128), Mrx, Mry, w, tx_, ty_, G)
    import scipy.fft
    F = scipy.fft.fft2(G, axes=(0, 1), workers=-1)          # [Mry, Mrx, Nk]
    m = np.arange(-Mx // 2, Mx // 2)
    n = np.arange(-My // 2, My // 2)
    F = F[np.ix_(n % Mry, m % Mrx)]                           # [My, Mx, Nk]
    dm = math.sqrt(math.pi / tx_) / Mrx * np.exp(m * m * tx_)
    dn = math.sqrt(math.pi / ty_) / Mry * np.exp(n * n * ty_)
    return np.transpose(F, (1, 0, 2)) * dm[:, None, None] * dn[None, :, None]


def fgg_type1_1d_plus(c, t, N, w):
    """F(q', col) = sum_k c_k exp(+j q' t_k), q' in [-N/2, N/2), per column,
    by Gaussian gridding on a 2N periodic grid + inverse FFT + deconvolution.
    c, t: [ncols, Nk].  Returns [ncols, N]."""
    ncols = c.shape[0]
    Mr = 2 * N
    tau = fgg_tau(N, w)
    g = np.zeros((ncols, Mr), np.complex128)
    _native.spread1d(np.ascontiguousarray(t, np.float64), np.ascontiguousarray(c, np.complex128), Mr, w, tau, g)
    import scipy.fft
    F = Mr * scipy.fft.ifft(g, axis=1, workers=-1)
    q = np.arange(-N // 2, N // 2)
    return F[:, q % Mr] * (math.sqrt(math.pi / tau) / Mr * np.exp(q * q * tau))[None, :]


def rma_fast(su: Setup, w: int = 16, k_slice: slice | None = None):
    """Same operator, paper's step order, FGG transforms.  ``k_slice``
    restricts the frequency samples (the image is linear in them); the
    normalisation stays 1/(T R P Nk) of the full scan."""
    if su.n_total == 0:
        return np.zeros((su.nx, su.ny, su.nz), np.complex128)
    shat, xv, yv = compensate(su)
    ks = k_slice or slice(0, su.n_k)
    shat = shat[:, ks]
    k = su.wavenumbers[ks]
    # FT_2D by FGG: sample positions in radians of the Mx-periodic spectrum.
    xr = 2 * np.pi * (xv - su.x_c) / (su.Mx * su.dx)
    yr = 2 * np.pi * (yv - su.y_c) / (su.My * su.dy)
    S = fgg_type1_2d(shat, xr, yr, su.Mx, su.My, w)            # [Mx, My, Nk']
    kx, ky = spectral_axes(su)
    kz2 = 4 * k[None, None, :] ** 2 - kx[:, None, None] ** 2 - ky[None, :, None] ** 2
    valid = kz2 > 0
    kz = np.sqrt(np.where(valid, kz2, 0.0))
    # Eq. 15 weight with the phase split at the centre slice q = nz//2.
    zc = su.z0 + (su.nz // 2) * su.dz
    c = np.where(valid, S * kz * np.exp(1j * kz * (zc - su.z_ref)), 0.0)
    t = kz * su.dz
    Zq = fgg_type1_1d_plus(c.reshape(-1, c.shape[2]), t.reshape(-1, t.shape[2]), su.nz, w)
    Z = Zq.reshape(su.Mx, su.My, su.nz)                         # q' -> q = q' + nz//2
    # IFT_2D: x_i - x_c = (i - nx//2) dx, so the sum is an Mx-point inverse DFT.
    import scipy.fft
    Zs = np.zeros_like(Z)
    m = np.arange(-su.Mx // 2, su.Mx // 2)
    n = np.arange(-su.My // 2, su.My // 2)
    Zs[np.ix_(m % su.Mx, n % su.My)] = Z
    A = scipy.fft.ifft2(Zs, axes=(0, 1), workers=-1) * (su.Mx * su.My)
    i = (np.arange(su.nx) - su.nx // 2) % su.Mx
    j = (np.arange(su.ny) - su.ny // 2) % su.My
    return A[np.ix_(i, j)] / su.n_total


# ----------------------------------------------------------------------------- helpers
def peak_index(vol, rel=1e-6):
    """Lowest linear index among voxels whose |o| is within rel of the max
    (row-major [nx, ny, nz], z fastest)."""
    a = np.abs(vol).ravel()
    mx = a.max()
    return int(np.flatnonzero(a >= mx * (1 - rel))[0])


def nmse(a, ref):
    ref = np.asarray(ref)
    d = np.linalg.norm((np.asarray(a) - ref).ravel()) ** 2
    r = np.linalg.norm(ref.ravel()) ** 2
    return d / r if r > 0 else (0.0 if d == 0 else math.inf)
