"""FP64 oracle for the map's source-profile convolution and light curves.

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the bench's
CPU-baseline leg; it shares no code with the CUDA library.

Section 1 of the paper: given a model of the background source's size and
intensity profile, the magnification pattern yields simulated light curves.
Here that is written out as
  * convolution: O[j, i] = scale * sum_{(di, dj) in K} w(di, dj) C[j + dj, i + di],
    C = 0 outside the map, with the source profile's weights w normalised to
    sum 1 over its support K (offsets measured in theta_E with the map's pixel
    widths dx, dy):
      Gaussian of width sigma: w proportional to exp(-d^2 / (2 sigma^2)) over
        |di| <= ceil(4 sigma / dx), |dj| <= ceil(4 sigma / dy); it factorises
        into normalised 1-D weights wx(di) wy(dj);
      uniform disk of radius R: w = 1 / |K| on K = {(di dx)^2 + (dj dy)^2 <= R^2};
  * magnification scale: a pixel holding its mean share of rays has
    N_rays * A_pix / A_lens of them, so mu = counts * A_lens / (N_rays * A_pix);
  * light curve: the convolved map sampled at n points evenly spaced on the
    segment b0 -> b1 of the source plane, by bilinear interpolation between pixel
    centres (x0 + (i + 1/2) dx, ...), constant beyond the outermost centres.
Plain loops over the kernel's offsets (vectorised over pixels); no FFT, no
separable shortcut in the direct form.
"""
from __future__ import annotations

import math

import numpy as np

GAUSSIAN = 0
DISK = 1


def _pix(src):
    return (src.x1 - src.x0) / src.nx, (src.y1 - src.y0) / src.ny


def magnification_scale(rays, src) -> float:
    """A_lens / (N_rays * A_pix): counts -> magnification."""
    a_lens = (rays.x1 - rays.x0) * (rays.y1 - rays.y0)
    dx, dy = _pix(src)
    return a_lens / (rays.nx * rays.ny * dx * dy)


def gaussian_weights(sigma: float, d: float) -> np.ndarray:
    """Normalised 1-D weights exp(-(k d)^2 / (2 sigma^2)), |k| <= ceil(4 sigma / d)."""
    k = int(math.ceil(4.0 * sigma / d))
    off = np.arange(-k, k + 1, dtype=np.float64) * d
    w = np.exp(-(off * off) / (2.0 * sigma * sigma))
    return w / w.sum()


def disk_offsets(radius: float, dx: float, dy: float):
    """All (di, dj) with (di dx)^2 + (dj dy)^2 <= R^2, evaluated in FP64."""
    kx, ky = int(math.floor(radius / dx)) + 1, int(math.floor(radius / dy)) + 1
    out = []
    for dj in range(-ky, ky + 1):
        for di in range(-kx, kx + 1):
            if (di * dx) * (di * dx) + (dj * dy) * (dj * dy) <= radius * radius:
                out.append((di, dj))
    return out


def _shifted(c: np.ndarray, di: int, dj: int) -> np.ndarray:
    """S[j, i] = c[j + dj, i + di], zero outside the map."""
    ny, nx = c.shape
    s = np.zeros_like(c)
    j0, j1 = max(0, -dj), min(ny, ny - dj)
    i0, i1 = max(0, -di), min(nx, nx - di)
    if j1 > j0 and i1 > i0:
        s[j0:j1, i0:i1] = c[j0 + dj:j1 + dj, i0 + di:i1 + di]
    return s


def convolve(counts: np.ndarray, src, profile: int, size: float, scale: float = 1.0) -> np.ndarray:
    """The direct convolution defined above, in FP64 (float32 output rounding is the
    caller's).  counts: [ny, nx] uint32."""
    c = np.asarray(counts, dtype=np.float64)
    dx, dy = _pix(src)
    out = np.zeros_like(c)
    if profile == GAUSSIAN:
        wx, wy = gaussian_weights(size, dx), gaussian_weights(size, dy)
        kx, ky = len(wx) // 2, len(wy) // 2
        for dj in range(-ky, ky + 1):
            for di in range(-kx, kx + 1):
                out += (wx[di + kx] * wy[dj + ky]) * _shifted(c, di, dj)
        return scale * out
    if profile == DISK:
        offs = disk_offsets(size, dx, dy)
        tot = np.zeros(c.shape, dtype=np.int64)
        ci = np.asarray(counts, dtype=np.int64)
        for di, dj in offs:
            tot += _shifted(ci, di, dj)
        f = scale / len(offs)
        return tot.astype(np.float64) * f
    raise ValueError("unknown profile")


def convolve_at(counts: np.ndarray, src, profile: int, size: float, scale: float, js, is_) -> np.ndarray:
    """The same sum evaluated only at pixels (js[k], is_[k]) -- for maps too large to
    convolve whole on the host."""
    c = np.asarray(counts)
    ny, nx = c.shape
    dx, dy = _pix(src)
    out = np.empty(len(js))
    if profile == GAUSSIAN:
        wx, wy = gaussian_weights(size, dx), gaussian_weights(size, dy)
        kx, ky = len(wx) // 2, len(wy) // 2
        for k, (j, i) in enumerate(zip(js, is_)):
            acc = 0.0
            for dj in range(-ky, ky + 1):
                if 0 <= j + dj < ny:
                    for di in range(-kx, kx + 1):
                        if 0 <= i + di < nx:
                            acc += (wx[di + kx] * wy[dj + ky]) * float(c[j + dj, i + di])
            out[k] = scale * acc
        return out
    if profile == DISK:
        offs = disk_offsets(size, dx, dy)
        f = scale / len(offs)
        for k, (j, i) in enumerate(zip(js, is_)):
            tot = 0
            for di, dj in offs:
                if 0 <= j + dj < ny and 0 <= i + di < nx:
                    tot += int(c[j + dj, i + di])
            out[k] = float(tot) * f
        return out
    raise ValueError("unknown profile")


def light_curve(mp: np.ndarray, src, b0, b1, npts: int) -> np.ndarray:
    """Bilinear samples of map mp[ny, nx] at npts points from b0 to b1 (theta_E)."""
    m = np.asarray(mp, dtype=np.float64)
    ny, nx = m.shape
    dx, dy = _pix(src)
    t = np.arange(npts, dtype=np.float64) / (npts - 1) if npts > 1 else np.zeros(1)
    bx = b0[0] + t * (b1[0] - b0[0])
    by = b0[1] + t * (b1[1] - b0[1])
    u = (bx - src.x0) / dx - 0.5
    v = (by - src.y0) / dy - 0.5
    out = np.empty(npts)
    for k in range(npts):
        i0, j0 = math.floor(u[k]), math.floor(v[k])
        fx, fy = u[k] - i0, v[k] - j0
        ia, ib = min(max(i0, 0), nx - 1), min(max(i0 + 1, 0), nx - 1)
        ja, jb = min(max(j0, 0), ny - 1), min(max(j0 + 1, 0), ny - 1)
        out[k] = ((1 - fy) * ((1 - fx) * m[ja, ia] + fx * m[ja, ib]) +
                  fy * ((1 - fx) * m[jb, ia] + fx * m[jb, ib]))
    return out
