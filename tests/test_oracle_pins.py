"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a Taylor
order (Eq. 5 / appendix), the ideal virtual monostatic echo (Eq. 10), a
library FFT in the on-grid special case, the Weyl plane-wave identity behind
Eq. 13-15, closed-form resolutions (Eq. 17), values printed in the paper
(tests/golden/paper_constants.json), brute-force sums and geometric
invariants.  A plausible slip in the oracle (a flipped sign of the d^z term,
a dropped MIMO term, a missing k_z weight, a transposed axis, a wrong
forward/inverse sign) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import bpa as obpa
from oracle import rma

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- constants
def test_lambda_and_prf_printed_values():
    g = _golden()
    lam = rma.C0 / g["prf_lower_bound_hz"]["f_center_hz"]
    assert round(lam * 1e3, 2) == g["lambda_c_mm_at_79GHz"]["value"]
    prf = 4 * g["prf_lower_bound_hz"]["v_max_m_s"] / lam
    assert abs(prf - g["prf_lower_bound_hz"]["value"]) / g["prf_lower_bound_hz"]["value"] < g["prf_lower_bound_hz"]["rel_tol"]
    assert g["dz_max_over_lambda"]["dz_max_m"] / lam > g["dz_max_over_lambda"]["value"]
    assert synth.LAMBDA_C == pytest.approx(lam, rel=1e-12)
    assert synth.BANDWIDTH == g["bandwidth_hz"]["value"] and synth.F0 == g["f0_hz"]["value"]


# ----------------------------------------------------------------------------- Eq. 5/7/12
def _exact_round_trip(xv, yv, z_ref, dxl, dyl, dzl, target):
    """Eq. 2 with the Eq. 3-4 substitution, computed directly."""
    T = np.array([xv - dxl / 2, yv - dyl / 2, z_ref + dzl])
    R = np.array([xv + dxl / 2, yv + dyl / 2, z_ref + dzl])
    return np.linalg.norm(T - target) + np.linalg.norm(R - target)


@pytest.mark.parametrize("seed", range(5))
def test_beta_taylor_order(seed):
    """R^RT - 2 R_0 - beta must vanish as O(d^3) on axis (Eq. 5 / appendix
    quadratic expansion).  A flipped d^z sign leaves an O(d) residual, a
    dropped or mis-scaled MIMO term an O(d^2) one."""
    rng = np.random.default_rng(seed)
    Zc, z_ref = 0.3, 0.01
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    target = np.array([0.02, -0.01, z_ref + Zc])
    res = []
    for eps in (4e-3, 2e-3, 1e-3):
        d = eps * u
        exact = _exact_round_trip(target[0], target[1], z_ref, d[0], d[1], d[2], target)
        beta = rma.residual_beta(d[0], d[1], d[2], Zc)
        res.append(abs(exact - 2 * Zc - beta))
    r1, r2 = res[0] / res[1], res[1] / res[2]
    assert 6.0 < r1 < 10.5 and 6.0 < r2 < 10.5, res
    assert res[2] < (1e-3) ** 3 / Zc ** 2


@pytest.mark.parametrize("seed", range(5))
def test_beta_scene_taylor_order_off_axis(seed):
    """Eq. 5 at the scene centre for an off-axis virtual element: the exact
    round trip minus 2 R_0 minus the refined residual vanishes as O(d^3),
    while Eq. 7's on-axis residual is off at first order there (its -2 d^z
    misses the Z_c / R_0 obliquity).  On axis the refined form equals Eq. 7's."""
    rng = np.random.default_rng(100 + seed)
    Zc, z_ref = 0.5, -0.02
    xs, ys = 0.01, -0.02
    xv, yv = xs + rng.uniform(0.05, 0.15), ys + rng.uniform(-0.12, 0.12)   # off axis
    target = np.array([xs, ys, z_ref + Zc])
    R0 = math.sqrt((xv - xs) ** 2 + (yv - ys) ** 2 + Zc ** 2)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    ref, eq7 = [], []
    for eps in (2e-3, 1e-3, 5e-4):
        d = eps * u
        exact = _exact_round_trip(xv, yv, z_ref, d[0], d[1], d[2], target) - 2 * R0
        ref.append(abs(exact - rma.residual_beta_scene(xv, yv, d[0], d[1], d[2], xs, ys, Zc)))
        eq7.append(abs(exact - rma.residual_beta(d[0], d[1], d[2], Zc)))
    assert 5.5 < ref[0] / ref[1] < 11 and 5.5 < ref[1] / ref[2] < 11, ref   # third order
    assert eq7[0] / eq7[2] < 20, eq7     # at best second order (first order off axis)
    assert all(r < 1e-2 * e for r, e in zip(ref, eq7)), (ref, eq7)
    # on axis the two residuals coincide
    d = 3e-3 * u
    on = rma.residual_beta_scene(xs, ys, d[0], d[1], d[2], xs, ys, Zc)
    assert on == pytest.approx(rma.residual_beta(d[0], d[1], d[2], Zc), rel=1e-12, abs=1e-15)


def test_beta_sign_matters():
    """The opposite sign of the 2 d^z term leaves a residual ~ 4|d^z|."""
    Zc = 0.3
    target = np.array([0.0, 0.0, Zc])
    d = np.array([1e-3, 2e-3, 3e-3])
    exact = _exact_round_trip(0.0, 0.0, 0.0, *d, target)
    good = rma.residual_beta(*d, Zc)
    bad = +2 * d[2] + (d[0] ** 2 + d[1] ** 2) / (4 * Zc)
    assert abs(exact - 2 * Zc - good) < 1e-7
    assert abs(exact - 2 * Zc - bad) == pytest.approx(4 * d[2], rel=0.01)


def test_compensation_approaches_virtual_monostatic():
    """Eq. 10-11: after compensation the echo of a scatterer at the scene
    centre approaches exp(-j 2 k R_0) of the virtual planar monostatic array;
    without compensation it does not."""
    rng = np.random.default_rng(3)
    lam = synth.LAMBDA_C
    tx = np.array([[0.0, -2.5 * lam, 0.0], [3 * lam, -0.5 * lam, 1e-3]])
    rx = np.array([[0.0, 0.0, 1e-3], [-lam, 1.5 * lam, 0.0]])
    pos = synth.jittered_grid(12, 12, 2e-3, 1e-3, 20e-3, rng)
    z_ref, z_scene = 0.0, 0.35
    sc = np.array([[0.0, 0.0, z_scene, 1.0]])
    nk = 16
    s = synth.echo(pos, tx, rx, synth.F0, synth.BANDWIDTH / nk, nk, sc)
    scan = synth.Scan(s, pos, tx, rx, synth.F0, synth.BANDWIDTH / nk,
                      synth.centred_grid(16, 16, 8, 1e-3, 5e-3, 0.3), sc)
    k = rma.setup_from(scan).wavenumbers
    errs = {}
    for comp in (True, False):
        su = rma.setup_from(scan, z_ref=z_ref, z_scene=z_scene, compensate=comp)
        shat, xv, yv = rma.compensate(su)
        R0 = np.sqrt(xv ** 2 + yv ** 2 + (z_scene - z_ref) ** 2)
        ideal = np.exp(-2j * np.outer(R0, k))
        errs[comp] = np.max(np.abs(np.angle(shat * np.conj(ideal))))
    # residual left by the Eq. 7 approximation (off-axis terms of Eq. 5) only
    assert errs[True] < 0.15, errs
    assert errs[False] > 10 * errs[True], errs


# ----------------------------------------------------------------------------- FT_2D
def _on_grid_setup(nxp, nyp, nk, M, seed, monostatic=True):
    """Monostatic elements exactly on the voxel pitch at z = z_ref: beta = 0
    and FT_2D is a plain 2-D DFT."""
    rng = np.random.default_rng(seed)
    a = rng.choice(np.arange(-M // 2, M // 2), size=nxp, replace=False)
    b = rng.choice(np.arange(-M // 2, M // 2), size=nyp, replace=False)
    A, B = np.meshgrid(a, b, indexing="ij")
    dx = 1e-3
    grid = synth.centred_grid(M, M, 4, dx, 5e-3, 0.2)
    pos = np.stack([A.ravel() * dx, B.ravel() * dx, np.zeros(A.size)], 1)
    z = np.zeros((1, 3))
    echo = (rng.normal(size=(1, 1, A.size, nk)) + 1j * rng.normal(size=(1, 1, A.size, nk))).astype(np.complex64)
    scan = synth.Scan(echo, pos, z, z, synth.F0, synth.BANDWIDTH / nk, grid, np.zeros((0, 4)))
    return scan, A.ravel(), B.ravel()


@pytest.mark.parametrize("M", [16, 32])
def test_ft2d_on_grid_equals_fft(M):
    scan, A, B = _on_grid_setup(9, 7, 5, M, seed=M)
    su = rma.setup_from(scan, z_ref=0.0)
    D = np.zeros((M, M, su.n_k), np.complex128)
    D[A % M, B % M, :] = scan.echo.reshape(-1, su.n_k)
    ref = np.fft.fft2(D, axes=(0, 1))
    m = np.arange(-M // 2, M // 2) % M
    ref = ref[np.ix_(m, m)]
    S = rma.spectrum_exact(su)
    assert np.allclose(S, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    shat, xv, yv = rma.compensate(su)
    Sf = rma.fgg_type1_2d(shat, 2 * np.pi * (xv - su.x_c) / (M * su.dx), 2 * np.pi * (yv - su.y_c) / (M * su.dy),
                          M, M, 16)
    assert np.allclose(Sf, ref, rtol=0, atol=1e-7 * np.abs(ref).max())


def test_fgg_1d_against_direct_sum():
    rng = np.random.default_rng(11)
    t = np.sort(rng.uniform(-9, 9, size=(3, 40)), axis=1)
    c = rng.normal(size=(3, 40)) + 1j * rng.normal(size=(3, 40))
    N = 24
    q = np.arange(-N // 2, N // 2)
    ref = np.stack([np.exp(1j * np.outer(q, t[i])) @ c[i] for i in range(3)])
    for w, tol in ((16, 1e-7), (8, 3e-4)):
        got = rma.fgg_type1_1d_plus(c, t, N, w)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol


# ----------------------------------------------------------------------------- Eq. 13-15
def test_weyl_identity_fixes_kz_weight_and_phase():
    """For the monostatic field exp(-j 2k R_0)/R_0 over a large planar aperture
    the 2-D spectrum is -2 pi j exp(-j k_z Z)/k_z (Weyl), so Eq. 15's weight
    k_z exp(+j k_z (z - z_ref)) makes every frequency add in phase at the
    target depth: |Z(m, n, q_t)| = Nk * 2 pi / pitch^2 for near-normal (m, n).
    A missing k_z factor or a flipped phase sign breaks the equality."""
    pitch = 1e-3
    half = 100
    xs = np.arange(-half, half + 1) * pitch
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    Zt = 0.1
    nk = 8
    f = synth.F0 + synth.BANDWIDTH / nk * np.arange(nk)
    k = 2 * np.pi * f / rma.C0
    R0 = np.sqrt(X.ravel() ** 2 + Y.ravel() ** 2 + Zt ** 2)
    echo = (np.exp(-2j * np.outer(R0, k)) / R0[:, None]).reshape(1, 1, -1, nk)
    grid = synth.Grid(-128 * pitch, -128 * pitch, Zt - 4 * 2e-3, pitch, pitch, 2e-3, 256, 256, 9)
    z = np.zeros((1, 3))
    pos = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    scan = synth.Scan(echo, pos, z, z, synth.F0, synth.BANDWIDTH / nk, grid, np.zeros((0, 4)))
    su = rma.setup_from(scan, z_ref=0.0, compensate=False)
    shat, xv, yv = rma.compensate(su)
    kx, ky = rma.spectral_axes(su)
    for (mi, ni) in [(128, 128), (130, 127), (125, 131)]:
        S = rma.spectrum_exact(su, shat, xv, yv, cols=[(mi, ni)])[0]
        Z = rma.stolt_exact(su, S[None, None, :], kx=kx[mi:mi + 1], ky=ky[ni:ni + 1])[0, 0]
        q_t = 4
        assert abs(Z[q_t]) * pitch ** 2 / (2 * np.pi * nk) == pytest.approx(1.0, abs=0.03)
        assert abs(Z[q_t]) >= 0.98 * np.abs(Z).max()


# ----------------------------------------------------------------------------- Eq. 17
def _profile_width(p, step):
    """-3 dB width of |p| around its maximum by linear interpolation."""
    a = np.abs(p) / np.abs(p).max()
    i = int(np.argmax(a))
    lvl = 1 / np.sqrt(2)
    lo = i
    while lo > 0 and a[lo - 1] >= lvl:
        lo -= 1
    hi = i
    while hi < len(a) - 1 and a[hi + 1] >= lvl:
        hi += 1
    left = lo - (a[lo] - lvl) / (a[lo] - a[lo - 1])
    right = hi + (a[hi] - lvl) / (a[hi] - a[hi + 1])
    return (right - left) * step


def _monostatic_planar(nxp, nk, grid, target, seed=0):
    rng = np.random.default_rng(seed)
    pos = synth.jittered_grid(nxp, nxp, 1e-3, 0.0, 0.0, rng)
    z = np.zeros((1, 3))
    sc = np.array([[*target, 1.0]])
    s = synth.echo(pos, z, z, synth.F0, synth.BANDWIDTH / nk, nk, sc)
    return synth.Scan(s, pos, z, z, synth.F0, synth.BANDWIDTH / nk, grid, sc)


def test_range_resolution_closed_form():
    """Eq. 17: delta_z = c / 2B; a point target focuses at its depth with a
    -3 dB width of 0.886 c/(2B) (uniform spectrum), here within 15 %.  The
    lateral window (128 mm) is many cross-range PSF widths (9 mm) and the
    aperture spans several Fresnel zones, so stationary phase holds; the
    amplitude-free echo model leaves at most a one-voxel (2 mm) range bias."""
    dz = 2e-3
    grid = synth.centred_grid(128, 128, 48, 1e-3, dz, 0.300 - 24 * dz)
    scan = _monostatic_planar(64, 64, grid, (0.0, 0.0, 0.300))
    o = rma.rma_fast(rma.setup_from(scan, z_ref=0.0), w=12)
    i, j, q = np.unravel_index(rma.peak_index(o), o.shape)
    assert (i, j) == (64, 64) and abs(q - 24) <= 1
    width = _profile_width(o[i, j, :], dz)
    assert width == pytest.approx(0.886 * rma.C0 / (2 * synth.BANDWIDTH), rel=0.15)


def test_cross_range_resolution_closed_form():
    """Eq. 17: delta_x = lambda_c Z / (2 D); -3 dB width 0.886 delta_x, 25 %."""
    D_pos = 64
    Zt = 0.3
    grid = synth.centred_grid(128, 128, 8, 1e-3, 5e-3, Zt - 4 * 5e-3)
    scan = _monostatic_planar(D_pos, 32, grid, (0.0, 0.0, Zt))
    o = rma.rma_fast(rma.setup_from(scan, z_ref=0.0), w=12)
    i, j, q = np.unravel_index(rma.peak_index(o), o.shape)
    assert (i, j) == (64, 64) and abs(q - 4) <= 1
    D = D_pos * 1e-3
    expect = 0.886 * synth.LAMBDA_C * Zt / (2 * D)
    assert _profile_width(o[:, j, q], 1e-3) == pytest.approx(expect, rel=0.25)
    assert _profile_width(o[i, :, q], 1e-3) == pytest.approx(expect, rel=0.25)


# ----------------------------------------------------------------------------- whole operator
def test_tiny_peaks_land_on_the_scatterer(tiny_scan):
    """On the tiny scan the cross-range PSF (~35 mm) is wider than the 32 mm
    lateral window, so only the range peak is well posed for the RMA; the
    back-projection (not periodic) must hit the scatterer voxel exactly."""
    su = rma.setup_from(tiny_scan)
    o = rma.rma_exact(su)
    pk = np.array(np.unravel_index(rma.peak_index(o), o.shape))
    truth = np.array(tiny_scan.grid.centre_index(0.0, 0.0, 0.3))
    assert abs(pk[2] - truth[2]) <= 1, (pk, truth)
    ob = obpa.bpa(tiny_scan)
    pb = np.array(np.unravel_index(rma.peak_index(ob), ob.shape))
    assert np.all(pb == truth)


def test_bpa_closed_form_single_point():
    """Noiseless unit scatterer: every term of the back-projection sum is 1
    at the scatterer, so o_BP = T R P Nk there and smaller elsewhere."""
    scan = synth.custom(nx_pos=6, ny_pos=5, nk=12, layout="awr1443", nx=8, ny=8, nz=6,
                        scatterers=[[0.0, 0.0, 0.26 + 3 * 5e-3, 1.0]], seed=4)
    o = obpa.bpa(scan)
    N = np.prod(scan.echo.shape)
    c = scan.grid.centre_index(0.0, 0.0, 0.26 + 3 * 5e-3)
    assert o[c] == pytest.approx(N, rel=1e-6)
    assert np.abs(o).max() == pytest.approx(N, rel=1e-6)


def test_shift_equivariance():
    """Moving positions and scene by whole pitches moves the image by the same
    number of voxels (periodic in the Mx x My field; here nx = Mx)."""
    base = synth.custom(nx_pos=10, ny_pos=10, nk=16, layout="tiny", nx=32, ny=32, nz=8, seed=5,
                        scatterers=[[1e-3, -2e-3, 0.29, 1.0], [-3e-3, 4e-3, 0.28, 0.7]])
    a, b = 3, -2
    sh = np.array([a * 1e-3, b * 1e-3, 0.0])
    sc2 = base.scatterers.copy()
    sc2[:, :3] += sh
    s2 = synth.echo(base.pos + sh, base.tx, base.rx, base.f0, base.df, base.n_k, sc2)
    moved = synth.Scan(s2, base.pos + sh, base.tx, base.rx, base.f0, base.df, base.grid, sc2)
    z_ref = 0.0
    o1 = rma.rma_exact(rma.setup_from(base, z_ref=z_ref))
    o2 = rma.rma_exact(rma.setup_from(moved, z_ref=z_ref))
    assert rma.nmse(o2, np.roll(o1, (a, b), axis=(0, 1))) < 1e-10


def test_evanescent_columns_are_zero():
    """Columns with k_x^2 + k_y^2 >= 4 k_max^2 carry no energy (dropped terms)."""
    scan = synth.custom(nx_pos=6, ny_pos=6, nk=8, nx=64, ny=64, nz=4, dx=0.4e-3, seed=6)
    su = rma.setup_from(scan)
    S = rma.spectrum_exact(su)
    Z = rma.stolt_exact(su, S)
    kx, ky = rma.spectral_axes(su)
    kmax = su.wavenumbers.max()
    ev = (kx[:, None] ** 2 + ky[None, :] ** 2) >= 4 * kmax ** 2
    assert ev.any() and (~ev).any()
    assert np.all(Z[ev] == 0)
    assert np.abs(Z[~ev]).max() > 0


@pytest.mark.parametrize("case", ["tiny", "ragged", "ragged_nocomp", "empty"])
def test_fast_oracle_matches_exact(case, tiny_scan):
    if case == "tiny":
        su = rma.setup_from(tiny_scan)
    elif case == "empty":
        sc = synth.custom(nx_pos=0, ny_pos=0, nk=8, nx=8, ny=8, nz=4, seed=1)
        su = rma.setup_from(sc)
        assert np.all(rma.rma_fast(su) == 0) and np.all(rma.rma_exact(su) == 0)
        return
    else:
        sc = synth.custom(nx_pos=7, ny_pos=5, nk=20, layout="awr1443", nx=24, ny=12, nz=10, seed=9,
                          jitter=(0.7e-3, 4e-3), snr_db=20)
        su = rma.setup_from(sc, compensate=(case == "ragged"))
        assert (su.Mx, su.My) == (32, 16)
    e = rma.rma_exact(su)
    f = rma.rma_fast(su, w=16)
    assert rma.nmse(f, e) < 1e-12
    assert rma.peak_index(f) == rma.peak_index(e)


def test_fast_oracle_k_slices_add_up(tiny_scan):
    su = rma.setup_from(tiny_scan)
    full = rma.rma_fast(su)
    parts = rma.rma_fast(su, k_slice=slice(0, 11)) + rma.rma_fast(su, k_slice=slice(11, 32))
    assert rma.nmse(parts, full) < 1e-24


@pytest.mark.parametrize("fast", [False, True])
def test_oracle_is_linear_in_the_echo(fast):
    """The image is linear in the echo (Eq. 11-16 are all linear in s): the
    image of a*s1 + b*s2 is a*image(s1) + b*image(s2), for complex a, b and
    two scenes on the same jittered multi-planar scan."""
    base = synth.custom(nx_pos=8, ny_pos=7, nk=16, layout="awr1443", nx=16, ny=16, nz=8, seed=12,
                        jitter=(0.7e-3, 3e-3), scatterers=[[1e-3, -2e-3, 0.29, 1.0]])
    s2 = synth.echo(base.pos, base.tx, base.rx, base.f0, base.df, base.n_k,
                    np.array([[-3e-3, 2e-3, 0.28, 0.6], [0.0, 4e-3, 0.30, 0.9]]))
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    e1, e2 = base.echo.astype(np.complex128), s2.astype(np.complex128)   # combine without complex64 rounding
    img = (lambda e: rma.rma_fast(rma.setup_from(base, echo=e))) if fast else \
          (lambda e: rma.rma_exact(rma.setup_from(base, echo=e)))
    lhs = img(a * e1 + b * e2)
    rhs = a * img(e1) + b * img(e2)
    assert rma.nmse(lhs, rhs) < 1e-24
    assert np.linalg.norm(img(e2)) > 0.1 * np.linalg.norm(img(e1))   # the second scene is not negligible


def test_compensation_sharpens_jittered_scan():
    """Sec. V: without compensation the multi-planar data defocus (lower peak);
    with it the peak is restored near the back-projection peak."""
    scan = synth.custom(nx_pos=32, ny_pos=32, nk=32, layout="awr1443", nx=64, ny=64, nz=16, seed=12,
                        jitter=(0.3e-3, 6e-3), scatterers=[[0.0, 0.0, 0.3, 1.0]])
    on = rma.rma_fast(rma.setup_from(scan, compensate=True), w=12)
    off = rma.rma_fast(rma.setup_from(scan, compensate=False), w=12)
    assert np.abs(on).max() > 1.5 * np.abs(off).max()
    truth = np.array(scan.grid.centre_index(0.0, 0.0, 0.3))
    pk = np.array(np.unravel_index(rma.peak_index(on), on.shape))
    assert np.all(np.abs(pk - truth) <= 1)


def test_normalisation_is_per_total_sample_count(tiny_scan):
    """1/(T R P Nk) normalisation: repeating every position (same echo) leaves
    the image unchanged, while the raw sums double."""
    su = rma.setup_from(tiny_scan)
    pos2 = np.concatenate([tiny_scan.pos, tiny_scan.pos])
    echo2 = np.concatenate([tiny_scan.echo, tiny_scan.echo], axis=2)
    twice = synth.Scan(echo2, pos2, tiny_scan.tx, tiny_scan.rx, tiny_scan.f0, tiny_scan.df, tiny_scan.grid,
                       tiny_scan.scatterers)
    su2 = rma.setup_from(twice, z_ref=su.z_ref)
    assert rma.nmse(rma.rma_exact(su2), rma.rma_exact(su)) < 1e-24
    s1 = rma.spectrum_exact(su)
    s2 = rma.spectrum_exact(su2)
    assert np.allclose(s2, 2 * s1)


def test_peak_index_tie_break():
    v = np.zeros((2, 3, 4), np.complex64)
    v[1, 2, 3] = 1.0
    v[0, 1, 2] = 1.0 - 1e-8
    assert rma.peak_index(v) == np.ravel_multi_index((0, 1, 2), v.shape)
    v[0, 1, 2] = 0.9
    assert rma.peak_index(v) == np.ravel_multi_index((1, 2, 3), v.shape)


# ----------------------------------------------------------------------------- Sec. V-A PSF study
def test_psf_study_compensation_modes():
    """The point-spread study of Sec. V-A on the oracle: with the samples
    spread +-5 cm off the reference plane, the uncompensated RMA loses the
    target (peak far below the planar case, misplaced), Eq. 7's residual
    recovers most of it, and Eq. 5 at the scene centre recovers the planar
    PSF (same peak, position and main lobe); the planar case has the
    closed-form cross-range width 0.886 lambda z / (2 D)."""
    from paper_2305_02064_gb300 import quality
    ref = None
    for dz, mode in ((0.0, 1), (0.05, 0), (0.05, 1), (0.05, 2)):
        sc = synth.psf_track(dz)
        su = rma.setup_from(sc, z_ref=0.0, compensate=mode, Mx=16)
        m = quality.psf_metrics(rma.rma_fast(su), sc.grid, sc.scatterers[0])
        if ref is None:
            ref = m
            lam = synth.LAMBDA_C
            assert m["width_y_mm"] == pytest.approx(0.886 * lam * 0.5 / (2 * 0.25) * 1e3, rel=0.05)
            assert m["peak_offset_y_mm"] == 0 and m["peak_offset_z_mm"] == 0
        elif mode == 0:
            assert m["peak"] < 0.3 * ref["peak"]
        elif mode == 1:
            assert 0.6 * ref["peak"] < m["peak"] < 0.97 * ref["peak"]
            assert m["width_y_mm"] > ref["width_y_mm"]
        else:
            assert m["peak"] == pytest.approx(ref["peak"], rel=0.01)
            assert m["width_y_mm"] == pytest.approx(ref["width_y_mm"], rel=0.02)
            assert abs(m["peak_offset_y_mm"]) < 1.5 and abs(m["peak_offset_z_mm"]) < 3


def test_psf_metrics_gaussian():
    """-3 dB widths of a separable Gaussian: 2 sigma sqrt(ln 2) per axis."""
    from paper_2305_02064_gb300 import quality

    class G:
        x0, y0, z0, dx, dy, dz = 0.0, -0.128, 0.42, 1e-3, 1e-3, 2.5e-3

    y = G.y0 + np.arange(256) * G.dy
    z = G.z0 + np.arange(64) * G.dz
    sy, sz = 3e-3, 10e-3
    vol = np.exp(-0.5 * (y[None, :, None] / sy) ** 2 - 0.5 * ((z[None, None, :] - 0.5) / sz) ** 2) * np.ones((2, 1, 1))
    m = quality.psf_metrics(vol, G, (0.0, 0.0, 0.5))
    assert m["width_y_mm"] == pytest.approx(2 * sy * math.sqrt(math.log(2)) * 1e3, rel=0.02)
    assert m["width_z_mm"] == pytest.approx(2 * sz * math.sqrt(math.log(2)) * 1e3, rel=0.02)
    assert m["peak_offset_y_mm"] == 0 and m["peak_offset_z_mm"] == 0 and m["pslr_y_db"] == -np.inf
