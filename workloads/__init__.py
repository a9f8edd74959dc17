"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *draws* inputs: star positions, masses, lens parameters, ray-grid and
source-map boxes, ray subsamples.  It holds none of the method's arithmetic (no
deflection, no source position, no binning), so importing it couples neither side to
the other.

Workloads follow the paper's random star field (Section 3: uniformly random positions,
a mass spectrum, smooth convergence kappa_c and external shear gamma) with the sizes of
the five benchmark configurations:

  tiny      100 unit masses, 1000^2 rays over [-10,10]^2, 256^2 map over [-4,4]^2
  paper     1e4 stars, 8192^2 rays, 1024^2 map over [-10,10]^2
  precision 1e5 stars, 16384^2 rays, 2048^2 map over [-10,10]^2
  learned   1e6 stars, 32768^2 rays, 4096^2 map over [-10,10]^2
  batched   256 fields with N in [1e2,1e4] log-uniform, 2048^2 rays, 512^2 maps
  large_n   1e7 stars (the learned field's parameters), 512^2 rays, 256^2 map over
            [-2,2]^2: few ray tiles for many stars (the split star sum's regime)

Units follow Eq. (4): angles in Einstein radii of a 1 M_sun lens, masses in M_sun.
With the deflection of Eq. (3), a uniform sheet of surface mass density rho (M_sun per
theta_E^2) deflects by pi*rho*theta, so a disk of N stars of mean mass <m> and radius R
has kappa_* = N <m> / R^2.

Star coordinates and masses are drawn in float64 and rounded to float32, so the same
numbers are exactly representable on both sides (the oracle promotes them to float64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field
from typing import List, Optional

import numpy as np

SEED_BASE = 170309707

# Salpeter-like mass function dN/dm ~ m^-2.35 on [0.1, 1] M_sun (configs paper..batched).
MF_SLOPE = 2.35
MF_LO = 0.1
MF_HI = 1.0


@dataclass
class Grid:
    """An axis-aligned box [x0,x1) x [y0,y1) cut into nx x ny cells (rays or pixels)."""
    x0: float
    x1: float
    y0: float
    y1: float
    nx: int
    ny: int

    @property
    def n(self) -> int:
        return int(self.nx) * int(self.ny)

    def astuple(self):
        return (float(self.x0), float(self.x1), float(self.y0), float(self.y1), int(self.nx), int(self.ny))


@dataclass
class Field:
    """One random star field plus the smooth part of the lens (Eq. 1)."""
    xy: np.ndarray          # (N,2) float64, float32-representable
    m: np.ndarray           # (N,)  float64, float32-representable
    kappa_c: float
    gamma1: float
    gamma2: float
    kappa_star: float = 0.0
    radius: float = 0.0

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


@dataclass
class Workload:
    name: str
    fields: List[Field]
    rays: List[Grid]
    srcs: List[Grid]
    note: str = ""
    cells: Optional[int] = None
    extra: dict = dc_field(default_factory=dict)


def mean_mass(slope: float = MF_SLOPE, lo: float = MF_LO, hi: float = MF_HI) -> float:
    """<m> of dN/dm ~ m^-slope on [lo, hi] (closed form of the two power-law integrals)."""
    a = 2.0 - slope
    b = 1.0 - slope
    return ((hi ** a - lo ** a) / a) / ((hi ** b - lo ** b) / b)


def draw_masses(rng: np.random.Generator, n: int, slope=MF_SLOPE, lo=MF_LO, hi=MF_HI) -> np.ndarray:
    """Inverse-CDF draw from dN/dm ~ m^-slope on [lo, hi]."""
    u = rng.random(n)
    e = 1.0 - slope
    m = (lo ** e + u * (hi ** e - lo ** e)) ** (1.0 / e)
    return m


def draw_disk(rng: np.random.Generator, n: int, radius: float) -> np.ndarray:
    """Uniform positions in a disk of the given radius (r = R sqrt(u), phi = 2 pi v)."""
    u = rng.random(n)
    v = rng.random(n)
    r = radius * np.sqrt(u)
    phi = 2.0 * np.pi * v
    return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)


def to_f32_exact(a: np.ndarray) -> np.ndarray:
    """Round to the nearest float32 and return as float64 (exactly representable in both)."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def random_field(seed: int, n: int, kappa_star: float, kappa_c: float, gamma1: float, gamma2: float,
                 unit_masses: bool = False, radius: Optional[float] = None) -> Field:
    rng = np.random.default_rng(seed)
    if unit_masses:
        m = np.ones(n)
        mm = 1.0
    else:
        m = draw_masses(rng, n)
        mm = mean_mass()
    if radius is None:
        radius = math.sqrt(n * mm / kappa_star) if n > 0 else 0.0
    xy = draw_disk(rng, n, radius)
    return Field(xy=to_f32_exact(xy), m=to_f32_exact(m), kappa_c=float(kappa_c), gamma1=float(gamma1),
                 gamma2=float(gamma2), kappa_star=float(kappa_star), radius=float(radius))


def lens_box(kappa: float, gamma1: float, gamma2: float, src_half: float, factor: float = 1.5):
    """Ray box = bounding box of the macro-model preimage of the source box enlarged by `factor`.

    The macro model is the linear part of Eq. (1) with the stars smeared into a sheet:
    beta = [[1-k-g1, -g2], [-g2, 1-k+g1]] theta with k = kappa_c + kappa_*.
    """
    a = np.array([[1.0 - kappa - gamma1, -gamma2], [-gamma2, 1.0 - kappa + gamma1]])
    ainv = np.linalg.inv(a)
    h = factor * src_half
    corners = np.array([[h, h], [h, -h], [-h, h], [-h, -h]]).T
    pre = ainv @ corners
    hx = float(np.max(np.abs(pre[0])))
    hy = float(np.max(np.abs(pre[1])))
    return hx, hy


def _round_box(h: float) -> float:
    # keep boxes on a 1/64 theta_E lattice so that they print and compare cleanly
    return math.ceil(h * 64.0 - 1e-9) / 64.0


def config(name: str, rays_scale: float = 1.0, src_scale: float = 1.0) -> Workload:
    """Return a workload by name.  `rays_scale` / `src_scale` shrink the ray grid / map
    resolution (same boxes, same stars) to make oracle-sized parity cases."""
    if name == "tiny":
        n = 100
        f = random_field(SEED_BASE + 1, n, kappa_star=0.45, kappa_c=0.0, gamma1=0.0, gamma2=0.0,
                         unit_masses=True, radius=math.sqrt(100.0 / 0.45))
        rays = Grid(-10.0, 10.0, -10.0, 10.0, 1000, 1000)
        src = Grid(-4.0, 4.0, -4.0, 4.0, 256, 256)
        wl = Workload("tiny", [f], [rays], [src], note="100 unit masses, disk R=sqrt(100/0.45)")
    elif name in ("paper", "precision", "learned"):
        p = {
            "paper": dict(idx=2, n=10_000, ks=0.3, kc=0.2, g=(0.3, 0.0), nr=8192, ns=1024),
            "precision": dict(idx=3, n=100_000, ks=0.4, kc=0.1, g=(0.2, 0.1), nr=16384, ns=2048),
            "learned": dict(idx=4, n=1_000_000, ks=0.45, kc=0.05, g=(0.25, 0.0), nr=32768, ns=4096),
        }[name]
        f = random_field(SEED_BASE + p["idx"], p["n"], p["ks"], p["kc"], p["g"][0], p["g"][1])
        hx, hy = lens_box(p["kc"] + p["ks"], p["g"][0], p["g"][1], 10.0)
        hx, hy = _round_box(hx), _round_box(hy)
        rays = Grid(-hx, hx, -hy, hy, p["nr"], p["nr"])
        src = Grid(-10.0, 10.0, -10.0, 10.0, p["ns"], p["ns"])
        wl = Workload(name, [f], [rays], [src], cells=256 if name == "learned" else None)
    elif name == "large_n":
        f = random_field(SEED_BASE + 6, 10_000_000, 0.45, 0.05, 0.25, 0.0)
        hx, hy = lens_box(0.5, 0.25, 0.0, 2.0)
        hx, hy = _round_box(hx), _round_box(hy)
        rays = Grid(-hx, hx, -hy, hy, 512, 512)
        src = Grid(-2.0, 2.0, -2.0, 2.0, 256, 256)
        wl = Workload(name, [f], [rays], [src])
    elif name == "batched":
        wl = batched_config()
    else:
        raise ValueError(f"unknown workload {name!r}")
    if rays_scale != 1.0 or src_scale != 1.0:
        wl.rays = [Grid(g.x0, g.x1, g.y0, g.y1, max(1, int(round(g.nx * rays_scale))),
                        max(1, int(round(g.ny * rays_scale)))) for g in wl.rays]
        wl.srcs = [Grid(g.x0, g.x1, g.y0, g.y1, max(1, int(round(g.nx * src_scale))),
                        max(1, int(round(g.ny * src_scale)))) for g in wl.srcs]
    return wl


def batched_config(nfields: int = 256, nrays: int = 2048, nsrc: int = 512, seed: int = SEED_BASE + 5,
                   n_lo: float = 1e2, n_hi: float = 1e4, min_eig: float = 0.1) -> Workload:
    """Many independent fields with uneven N_* (parameter-grid use case of Section 2.2).

    N_* log-uniform on [n_lo, n_hi], kappa_* ~ U[0.1,0.8], kappa_c ~ U[0,0.3],
    |gamma| ~ U[0,0.6] at a uniform random angle.  Fields whose macro model has an
    eigenvalue of magnitude < min_eig (near-critical, exploding lens box) are redrawn.
    The source box of each field is sized so that its ray box stays inside the star disk.
    """
    rng = np.random.default_rng(seed)
    fields, rays, srcs = [], [], []
    mm = mean_mass()
    while len(fields) < nfields:
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        ks = rng.uniform(0.1, 0.8)
        kc = rng.uniform(0.0, 0.3)
        gm = rng.uniform(0.0, 0.6)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        g1, g2 = gm * math.cos(ang), gm * math.sin(ang)
        k = ks + kc
        lam = (1.0 - k - gm, 1.0 - k + gm)
        fseed = int(rng.integers(0, 2**31 - 1))
        if min(abs(lam[0]), abs(lam[1])) < min_eig:
            continue
        radius = math.sqrt(n * mm / ks)
        lmin = min(abs(lam[0]), abs(lam[1]))
        half = 0.9 * radius * lmin / (1.5 * math.sqrt(2.0))
        half = math.floor(half * 64.0) / 64.0
        if half <= 0.0:
            continue
        f = random_field(fseed, n, ks, kc, g1, g2)
        hx, hy = lens_box(k, g1, g2, half)
        hx, hy = _round_box(hx), _round_box(hy)
        fields.append(f)
        rays.append(Grid(-hx, hx, -hy, hy, nrays, nrays))
        srcs.append(Grid(-half, half, -half, half, nsrc, nsrc))
    return Workload("batched", fields, rays, srcs, note=f"{nfields} fields")


def ray_sample(grid: Grid, k: int, seed: int) -> np.ndarray:
    """k distinct linear ray indices (j*nx + i) drawn uniformly from the grid, sorted."""
    rng = np.random.default_rng(seed)
    n = grid.n
    k = min(k, n)
    idx = rng.choice(n, size=k, replace=False)
    return np.sort(idx.astype(np.int64))


def flat_source_pixels(grid: Grid):
    """Pixel areas etc. for turning counts into magnification (no method arithmetic)."""
    return (grid.x1 - grid.x0) / grid.nx * (grid.y1 - grid.y0) / grid.ny
