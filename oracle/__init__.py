"""FP64 CPU oracle for backward microlensing ray-shooting (arXiv:1703.09707).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the bench's CPU-baseline
leg import this package.  It shares no code with the CUDA library and never
imports it.

The C part (mlens_oracle.c) restates Eq. (1)-(3) and Algorithm 1 in plain double
precision; this module compiles it with gcc on first use and exposes numpy-level
wrappers.  See the C file's header for the readings of points the paper leaves
open.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlens_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmlens_oracle.so")
_lock = threading.Lock()
_lib = None


class OrcCells(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("w", C.c_double), ("nx", C.c_int32), ("ny", C.c_int32)]


class OrcGrid(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libmlens_oracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load(path: str):
    """Open a compiled oracle and declare its C signatures."""
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    fp = C.POINTER(C.c_float)
    ip = C.POINTER(C.c_int64)
    up = C.POINTER(C.c_uint32)
    u64p = C.POINTER(C.c_uint64)
    gp = C.POINTER(OrcGrid)
    L.orc_alpha.argtypes = [dp, C.c_int64, dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp, C.c_int]
    L.orc_alpha_scale.argtypes = [dp, C.c_int64, dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp,
                                  C.c_int]
    L.orc_alpha_jacobian.argtypes = [dp, C.c_int64, dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp,
                                     C.c_int]
    cp = C.POINTER(OrcCells)
    L.orc_cell_index.argtypes = [dp, C.c_int64, cp, ip]
    L.orc_split_alpha.argtypes = [dp, ip, C.c_int64, dp, dp, C.c_int64, cp, dp, dp, C.c_int]
    L.orc_local_coeffs.argtypes = [ip, C.c_int64, C.c_int32, C.c_double, dp, dp, C.c_int64, cp, dp, C.c_int]
    L.orc_pixels.argtypes = [dp, C.c_int64, gp, ip]
    L.orc_ray_theta.argtypes = [gp, ip, C.c_int64, dp]
    L.orc_shoot.argtypes = [gp, gp, dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, up, u64p, C.c_int]
    L.orc_beta_rays.argtypes = [gp, ip, C.c_int64, dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double,
                                dp, C.c_int]
    L.orc_rebin_pair.argtypes = [fp, C.c_int64, gp, up, u64p]
    L.orc_pair_pixels.argtypes = [fp, C.c_int64, gp, ip]
    L.orc_max_threads.restype = C.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _load(_LIB)
    return _lib


class using:
    """Context manager: route every oracle call through another compiled copy of the
    oracle (the mutation tests use it to check that the pins catch planted mistakes)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self._old = _lib
        _lib = _load(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._old
        return False


def build_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source (used only by the mutation tests)."""
    tmp_c = out_path + ".c"
    with open(tmp_c, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", tmp_c, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _grid(g) -> OrcGrid:
    if isinstance(g, OrcGrid):
        return g
    if hasattr(g, "astuple"):
        g = g.astuple()
    x0, x1, y0, y1, nx, ny = g
    return OrcGrid(float(x0), float(x1), float(y0), float(y1), int(nx), int(ny))


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _stars(field):
    xy, pxy = _d(field.xy.reshape(-1, 2) if field.n else np.zeros((0, 2)))
    m, pm = _d(field.m if field.n else np.zeros(0))
    return xy, pxy, m, pm


def max_threads() -> int:
    return int(lib().orc_max_threads())


def alpha(theta: np.ndarray, field, nthreads: int = 0) -> np.ndarray:
    """Eq. (3) at arbitrary image positions theta (k,2)."""
    th, pth = _d(np.asarray(theta).reshape(-1, 2))
    xy, pxy, m, pm = _stars(field)
    out = np.empty_like(th)
    lib().orc_alpha(pth, th.shape[0], pxy, pm, field.n, field.kappa_c, field.gamma1, field.gamma2,
                    out.ctypes.data_as(C.POINTER(C.c_double)), int(nthreads))
    return out


def alpha_scale(theta: np.ndarray, field, nthreads: int = 0) -> np.ndarray:
    """|alpha_0| + sum_k m_k/|theta-theta_k|: the magnitude scale of the terms of Eq. (3)."""
    th, pth = _d(np.asarray(theta).reshape(-1, 2))
    xy, pxy, m, pm = _stars(field)
    out = np.empty(th.shape[0])
    lib().orc_alpha_scale(pth, th.shape[0], pxy, pm, field.n, field.kappa_c, field.gamma1, field.gamma2,
                          out.ctypes.data_as(C.POINTER(C.c_double)), int(nthreads))
    return out


def alpha_jacobian(theta: np.ndarray, field, nthreads: int = 0) -> np.ndarray:
    """d alpha / d theta of Eq. (3) as (k,3) = {J11, J12, J22}."""
    th, pth = _d(np.asarray(theta).reshape(-1, 2))
    xy, pxy, m, pm = _stars(field)
    out = np.empty((th.shape[0], 3))
    lib().orc_alpha_jacobian(pth, th.shape[0], pxy, pm, field.n, field.kappa_c, field.gamma1, field.gamma2,
                             out.ctypes.data_as(C.POINTER(C.c_double)), int(nthreads))
    return out


def beta(theta: np.ndarray, field, nthreads: int = 0) -> np.ndarray:
    """Eq. (2): beta = theta - alpha."""
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 2)
    return th - alpha(th, field, nthreads)


def ray_theta(rays, idx: np.ndarray) -> np.ndarray:
    """Image positions of grid rays given by linear index j*nx+i (cell centres)."""
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty((ix.shape[0], 2))
    g = _grid(rays)
    lib().orc_ray_theta(C.byref(g), ix.ctypes.data_as(C.POINTER(C.c_int64)), ix.shape[0],
                        out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def beta_rays(rays, idx: np.ndarray, field, nthreads: int = 0) -> np.ndarray:
    """beta of selected grid rays (linear indices), FP64."""
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    xy, pxy, m, pm = _stars(field)
    out = np.empty((ix.shape[0], 2))
    g = _grid(rays)
    lib().orc_beta_rays(C.byref(g), ix.ctypes.data_as(C.POINTER(C.c_int64)), ix.shape[0], pxy, pm, field.n,
                        field.kappa_c, field.gamma1, field.gamma2, out.ctypes.data_as(C.POINTER(C.c_double)),
                        int(nthreads))
    return out


def pixels(beta_xy: np.ndarray, src) -> np.ndarray:
    """Source pixel (j*nx+i) of each FP64 beta; -1 outside the window, -2 non-finite."""
    b, pb = _d(np.asarray(beta_xy).reshape(-1, 2))
    out = np.empty(b.shape[0], dtype=np.int64)
    g = _grid(src)
    lib().orc_pixels(pb, b.shape[0], C.byref(g), out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


def shoot(rays, src, field, nthreads: int = 0):
    """Algorithm 1 over the whole ray grid.  Returns (counts[ny,nx] uint32, stats dict)."""
    g, s = _grid(rays), _grid(src)
    xy, pxy, m, pm = _stars(field)
    counts = np.empty((s.ny, s.nx), dtype=np.uint32)
    st = np.zeros(4, dtype=np.uint64)
    lib().orc_shoot(C.byref(g), C.byref(s), pxy, pm, field.n, field.kappa_c, field.gamma1, field.gamma2,
                    counts.ctypes.data_as(C.POINTER(C.c_uint32)), st.ctypes.data_as(C.POINTER(C.c_uint64)),
                    int(nthreads))
    return counts, dict(rays_total=int(st[0]), rays_binned=int(st[1]), rays_out=int(st[2]), rays_nan=int(st[3]))


def rebin_pair(beta4: np.ndarray, src):
    """Re-bin float-pair betas {x_hi, y_hi, x_lo, y_lo} with the GPU's float32 rule."""
    b = np.ascontiguousarray(beta4, dtype=np.float32).reshape(-1, 4)
    s = _grid(src)
    counts = np.empty((s.ny, s.nx), dtype=np.uint32)
    st = np.zeros(4, dtype=np.uint64)
    lib().orc_rebin_pair(b.ctypes.data_as(C.POINTER(C.c_float)), b.shape[0], C.byref(s),
                         counts.ctypes.data_as(C.POINTER(C.c_uint32)), st.ctypes.data_as(C.POINTER(C.c_uint64)))
    return counts, dict(rays_total=int(st[0]), rays_binned=int(st[1]), rays_out=int(st[2]), rays_nan=int(st[3]))


def pair_pixels(beta4: np.ndarray, src) -> np.ndarray:
    b = np.ascontiguousarray(beta4, dtype=np.float32).reshape(-1, 4)
    out = np.empty(b.shape[0], dtype=np.int64)
    s = _grid(src)
    lib().orc_pair_pixels(b.ctypes.data_as(C.POINTER(C.c_float)), b.shape[0], C.byref(s),
                          out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


# ----------------------------------------------------------------- cells
def cells(x0: float, y0: float, w: float, nx: int, ny: int = None) -> OrcCells:
    """Square cells of width w: nx x ny of them from (x0, y0); index iy*nx + ix."""
    return OrcCells(float(x0), float(y0), float(w), int(nx), int(nx if ny is None else ny))


def cell_index(xy: np.ndarray, c: OrcCells) -> np.ndarray:
    a, pa = _d(np.asarray(xy).reshape(-1, 2))
    out = np.empty(a.shape[0], dtype=np.int64)
    lib().orc_cell_index(pa, a.shape[0], C.byref(c), out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


def split_alpha(theta: np.ndarray, ray_cell: np.ndarray, field, c: OrcCells, nthreads: int = 0):
    """(near, far) star terms of Eq. (3) at theta for rays in the given cells."""
    th, pth = _d(np.asarray(theta).reshape(-1, 2))
    rc = np.ascontiguousarray(ray_cell, dtype=np.int64)
    xy, pxy, m, pm = _stars(field)
    near = np.empty_like(th)
    far = np.empty_like(th)
    lib().orc_split_alpha(pth, rc.ctypes.data_as(C.POINTER(C.c_int64)), th.shape[0], pxy, pm, field.n, C.byref(c),
                          near.ctypes.data_as(C.POINTER(C.c_double)), far.ctypes.data_as(C.POINTER(C.c_double)),
                          int(nthreads))
    return near, far


def local_coeffs(cell_ids: np.ndarray, P: int, scale: float, field, c: OrcCells, nthreads: int = 0) -> np.ndarray:
    """Complex coefficients (ncell, P+1) of the far field's local expansion in (z - z_c)/scale."""
    ids = np.ascontiguousarray(cell_ids, dtype=np.int64)
    xy, pxy, m, pm = _stars(field)
    out = np.empty((ids.shape[0], P + 1, 2))
    lib().orc_local_coeffs(ids.ctypes.data_as(C.POINTER(C.c_int64)), ids.shape[0], int(P), float(scale), pxy, pm,
                           field.n, C.byref(c), out.ctypes.data_as(C.POINTER(C.c_double)), int(nthreads))
    return out[..., 0] + 1j * out[..., 1]
