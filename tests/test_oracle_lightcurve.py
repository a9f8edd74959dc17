"""Pins of the FP64 convolution / light-curve oracle (oracle/lightcurve.py), each
against something other than the oracle itself: closed forms, special cases, a
library routine, and the finite-source magnification of a point lens."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import lightcurve as LC


def _rand_counts(rng, ny, nx, lam=20.0):
    return rng.poisson(lam, (ny, nx)).astype(np.uint32)


@pytest.mark.parametrize("profile,size", [(LC.GAUSSIAN, 0.3), (LC.DISK, 0.45)])
def test_constant_map_stays_constant_away_from_edges(profile, size):
    src = W.Grid(-2.0, 2.0, -1.0, 1.0, 80, 50)  # anisotropic pixels: 0.05 x 0.04
    c = np.full((src.ny, src.nx), 7, dtype=np.uint32)
    out = LC.convolve(c, src, profile, size, scale=0.5)
    k = 25
    assert np.allclose(out[k:-k, k:-k], 3.5, rtol=1e-13, atol=0)
    assert np.all(out <= 3.5 * (1 + 1e-13)) and out[0, 0] < 3.5  # zero padding at the edges


def test_delta_map_returns_the_profile():
    src = W.Grid(0.0, 3.0, 0.0, 2.0, 60, 50)  # dx = 0.05, dy = 0.04
    c = np.zeros((src.ny, src.nx), dtype=np.uint32)
    c[25, 30] = 1000
    sigma = 0.2
    g = LC.convolve(c, src, LC.GAUSSIAN, sigma)
    # closed form of the normalised, truncated, separable Gaussian
    kx, ky = math.ceil(4 * sigma / 0.05), math.ceil(4 * sigma / 0.04)
    nx_ = sum(math.exp(-(k * 0.05) ** 2 / (2 * sigma * sigma)) for k in range(-kx, kx + 1))
    ny_ = sum(math.exp(-(k * 0.04) ** 2 / (2 * sigma * sigma)) for k in range(-ky, ky + 1))
    for a, b in [(0, 0), (3, 0), (0, 5), (-4, 7), (ky, kx), (ky + 1, 0)]:
        want = 0.0
        if abs(a) <= ky and abs(b) <= kx:
            want = 1000 * math.exp(-((b * 0.05) ** 2 + (a * 0.04) ** 2) / (2 * sigma * sigma)) / (nx_ * ny_)
        assert g[25 + a, 30 + b] == pytest.approx(want, rel=1e-12, abs=1e-300), (a, b)
    R = 0.21
    d = LC.convolve(c, src, LC.DISK, R)
    inside = [(a, b) for a in range(-6, 7) for b in range(-6, 7)
              if (b * 0.05) ** 2 + (a * 0.04) ** 2 <= R * R]
    for a in range(-7, 8):
        for b in range(-7, 8):
            want = 1000 / len(inside) if (a, b) in inside else 0.0
            assert d[25 + a, 30 + b] == pytest.approx(want, rel=1e-14), (a, b)
    assert g.sum() == pytest.approx(1000, rel=1e-12) and d.sum() == pytest.approx(1000, rel=1e-12)


def test_matches_a_library_correlation_on_random_maps():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    src = W.Grid(-1.0, 1.0, -1.5, 1.5, 41, 73)  # dx = 0.0488, dy = 0.0411
    c = _rand_counts(rng, src.ny, src.nx)
    dx, dy = 2.0 / 41, 3.0 / 73
    sigma = 0.17
    kx, ky = math.ceil(4 * sigma / dx), math.ceil(4 * sigma / dy)
    X, Y = np.meshgrid(np.arange(-kx, kx + 1) * dx, np.arange(-ky, ky + 1) * dy)
    ker = np.exp(-(X * X + Y * Y) / (2 * sigma * sigma))
    ker /= ker.sum()
    want = ndimage.correlate(c.astype(np.float64), ker, mode="constant", cval=0.0)
    assert np.allclose(LC.convolve(c, src, LC.GAUSSIAN, sigma, scale=1.0), want, rtol=1e-12, atol=1e-12)
    R = 0.2
    hx, hy = int(R / dx) + 1, int(R / dy) + 1
    X, Y = np.meshgrid(np.arange(-hx, hx + 1) * dx, np.arange(-hy, hy + 1) * dy)
    disk = (X * X + Y * Y <= R * R).astype(np.float64)
    want = ndimage.correlate(c.astype(np.float64), disk / disk.sum(), mode="constant", cval=0.0)
    assert np.allclose(LC.convolve(c, src, LC.DISK, R), want, rtol=1e-12, atol=1e-12)


def test_disk_support_area():
    offs = LC.disk_offsets(10.0, 0.1, 0.1)
    assert abs(len(offs) * 0.01 - math.pi * 100.0) < 2 * math.pi * 10.0 * 0.1  # within a perimeter's width
    assert (0, 0) in offs and (100, 0) in offs and (101, 0) not in offs and (71, 71) not in offs


def test_unlensed_sheet_has_unit_magnification():
    """No stars, no shear: rays aligned with 0.1 x 0.2 pixels, 50 per pixel; scale * counts = 1."""
    f = W.Field(xy=np.zeros((0, 2)), m=np.zeros(0), kappa_c=0.0, gamma1=0.0, gamma2=0.0)
    rays = W.Grid(-10.0, 10.0, -10.0, 10.0, 1000, 1000)
    src = W.Grid(-5.0, 5.0, -4.0, 4.0, 100, 40)
    c, _ = oracle.shoot(rays, src, f)
    mu = c * LC.magnification_scale(rays, src)
    assert np.all(c == 50) and np.allclose(mu, 1.0, rtol=1e-14)


def test_point_lens_disk_source_magnification():
    """A uniform disk source of radius rho centred on a point lens: its images fill the
    annulus rho_-(rho) <= |theta| <= rho_+(rho), area pi rho sqrt(rho^2 + 4), so
    mu = sqrt(1 + 4 / rho^2) (Witt & Mao 1994 at zero impact parameter)."""
    f = W.Field(xy=np.zeros((1, 2)), m=np.ones(1), kappa_c=0.0, gamma1=0.0, gamma2=0.0)
    rays = W.Grid(-3.0, 3.0, -3.0, 3.0, 3000, 3000)
    src = W.Grid(-1.0, 1.0, -1.0, 1.0, 101, 101)  # the lens sits on the centre of pixel (50, 50)
    c, _ = oracle.shoot(rays, src, f)
    scale = LC.magnification_scale(rays, src)
    for rho in (0.3, 0.5, 0.8):
        mu = LC.convolve(c, src, LC.DISK, rho, scale)[50, 50]
        assert mu == pytest.approx(math.sqrt(1 + 4 / rho ** 2), rel=0.01), rho


def test_light_curve_is_exact_on_affine_maps_and_hits_pixel_centres():
    src = W.Grid(-2.0, 2.0, -1.0, 3.0, 40, 20)  # dx = 0.1, dy = 0.2
    j, i = np.mgrid[0:20, 0:40]
    m = 1.5 + 0.25 * i - 0.75 * j  # affine in the pixel indices
    b0, b1 = (-1.23, -0.4), (1.71, 2.52)
    lc = LC.light_curve(m, src, b0, b1, 57)
    t = np.arange(57) / 56
    u = (b0[0] + t * (b1[0] - b0[0]) + 2.0) / 0.1 - 0.5
    v = (b0[1] + t * (b1[1] - b0[1]) + 1.0) / 0.2 - 0.5
    assert np.allclose(lc, 1.5 + 0.25 * u - 0.75 * v, rtol=1e-13)
    # at a pixel centre the curve takes the pixel's value; beyond the outer centres it is flat
    c = LC.light_curve(m, src, (-2.0 + 0.05 * 7, -1.0 + 0.2 * 3.5), (10.0, -1.0 + 0.2 * 3.5), 2)
    assert c[0] == pytest.approx(m[3, 3]) and c[1] == pytest.approx(m[3, 39])
    assert LC.light_curve(m, src, (5.0, 5.0), (5.0, 5.0), 1)[0] == m[19, 39]


@pytest.mark.parametrize("profile,size", [(LC.GAUSSIAN, 0.12), (LC.DISK, 0.2)])
def test_pointwise_form_equals_the_whole_map_form(profile, size):
    rng = np.random.default_rng(8)
    src = W.Grid(-1.0, 1.0, -0.6, 0.6, 37, 29)
    c = _rand_counts(rng, src.ny, src.nx)
    full = LC.convolve(c, src, profile, size, 0.7)
    js, is_ = rng.integers(0, src.ny, 60), rng.integers(0, src.nx, 60)
    assert np.allclose(LC.convolve_at(c, src, profile, size, 0.7, js, is_), full[js, is_], rtol=1e-13, atol=0)
