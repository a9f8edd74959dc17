"""Thin ctypes binding of libmlens (include/mlens.h).

Argument marshalling only: every function here forwards to the C entry point of the
same name; all computation runs in the library's CUDA kernels.  Device buffers are
torch CUDA tensors (their data pointers are passed through); the stream defaults to
torch's current stream so CUDA events recorded by torch bracket the kernels.

The binding fails loudly when the library has not been built: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from .build import LIB

MLENS_OK = 0
MLENS_ERR_ARG = -1
MLENS_ERR_CUDA = -2
MLENS_ERR_NOMEM = -3
MLENS_ERR_STATE = -4
MLENS_ERR_UNSUPPORTED = -5

MLENS_PREC_FP32 = 0
MLENS_PREC_FP32_NAIVE = 1
MLENS_PREC_FP64 = 2

MLENS_ACCUMULATE = 1

MLENS_PROFILE_GAUSSIAN = 0
MLENS_PROFILE_DISK = 1

PRECISIONS = {"fp32": MLENS_PREC_FP32, "fp32_naive": MLENS_PREC_FP32_NAIVE, "fp64": MLENS_PREC_FP64}


class MlensError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmlens error {code}: {msg}")
        self.code = code


class mlens_grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


class mlens_stats(C.Structure):
    _fields_ = [("rays_total", C.c_uint64), ("rays_binned", C.c_uint64), ("rays_out", C.c_uint64),
                ("rays_nan", C.c_uint64)]

    def asdict(self):
        return dict(rays_total=int(self.rays_total), rays_binned=int(self.rays_binned),
                    rays_out=int(self.rays_out), rays_nan=int(self.rays_nan))


class mlens_fit_params(C.Structure):
    _fields_ = [("cells_x", C.c_int32), ("order", C.c_int32), ("target_order", C.c_int32),
                ("use_network", C.c_int32), ("train_samples", C.c_int64), ("epochs", C.c_int32),
                ("batch", C.c_int32), ("lr_weights", C.c_float), ("lr_latents", C.c_float),
                ("val_samples_per_cell", C.c_int32), ("tolerance", C.c_double), ("seed", C.c_uint64)]


class mlens_fit_report(C.Structure):
    _fields_ = [("cells", C.c_int32), ("cells_fallback", C.c_int32), ("tiles", C.c_int64),
                ("tiles_fallback", C.c_int64), ("train_steps", C.c_int64), ("final_loss", C.c_double),
                ("val_max_err_net", C.c_double), ("val_mean_err_net", C.c_double),
                ("val_max_err_series", C.c_double), ("val_mean_err_series", C.c_double),
                ("seconds_coefficients", C.c_double), ("seconds_train", C.c_double),
                ("seconds_validate", C.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mlens_far_field_info(C.Structure):
    _fields_ = [("cells_x", C.c_int32), ("cells_y", C.c_int32), ("grid_x0", C.c_double), ("grid_y0", C.c_double),
                ("cell_width", C.c_double), ("grid_nx", C.c_int32), ("grid_ny", C.c_int32), ("order", C.c_int32),
                ("target_order", C.c_int32), ("use_network", C.c_int32), ("n_params", C.c_int32),
                ("latent_dim", C.c_int32), ("report", mlens_fit_report)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); mirrors include/mlens.h
_vp = C.c_void_p
_gp = C.POINTER(mlens_grid)
_sp = C.POINTER(mlens_stats)
_dp = C.POINTER(C.c_double)
SIGNATURES = {
    "mlens_create": (C.c_int, [C.POINTER(_vp), _dp, _dp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int32]),
    "mlens_set_precision": (C.c_int, [_vp, C.c_int32]),
    "mlens_set_tuning": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32]),
    "mlens_set_star_split": (C.c_int, [_vp, C.c_int32]),
    "mlens_star_split_for": (C.c_int, [_vp, _gp, C.POINTER(C.c_int32)]),
    "mlens_shoot": (C.c_int, [_vp, _gp, _gp, _vp, C.c_uint32, _sp, _vp]),
    "mlens_shoot_beta": (C.c_int, [_vp, _gp, _gp, _vp, _vp, C.c_uint32, _sp, _vp]),
    "mlens_shoot_rows": (C.c_int, [_vp, _gp, C.c_int32, C.c_int32, _gp, _vp, _vp, C.c_uint32, _sp, _vp]),
    "mlens_trace": (C.c_int, [_vp, _dp, C.c_int64, _dp, _vp]),
    "mlens_bin": (C.c_int, [_vp, C.c_int64, _gp, _vp, C.c_uint32, _sp, _vp]),
    "mlens_bin_grid": (C.c_int, [_vp, _gp, _gp, _vp, C.c_uint32, _sp, _vp]),
    "mlens_convolve": (C.c_int, [_vp, _gp, C.c_int32, C.c_double, C.c_double, _vp, _vp, C.c_uint64, _vp]),
    "mlens_convolve_workspace": (C.c_int, [_gp, C.c_int32, C.c_double, C.POINTER(C.c_uint64)]),
    "mlens_light_curve": (C.c_int, [_vp, _gp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32, _vp, _vp]),
    "mlens_magnification_scale": (C.c_int, [_gp, _gp, _dp]),
    "mlens_shoot_noalloc": (C.c_int, [_vp, C.c_int64, C.c_double, C.c_double, C.c_double, _gp, _gp, _vp, C.c_uint32,
                                      _sp, _vp]),
    "mlens_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int32, _gp, _gp, C.POINTER(_vp),
                                     C.c_uint32]),
    "mlens_batch_set_tuning": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32]),
    "mlens_batch_tune": (C.c_int, [_vp, _vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_double)]),
    "mlens_batch_run": (C.c_int, [_vp, _sp, _vp]),
    "mlens_batch_destroy": (None, [_vp]),
    "mlens_shoot_batch": (C.c_int, [C.POINTER(_vp), C.c_int32, _gp, _gp, C.POINTER(_vp), C.c_uint32, _sp, _vp]),
    "mlens_fit_params_default": (None, [C.POINTER(mlens_fit_params)]),
    "mlens_fit_far_field": (C.c_int, [_vp, _gp, C.POINTER(mlens_fit_params), C.POINTER(mlens_fit_report), _vp]),
    "mlens_shoot_learned": (C.c_int, [_vp, _gp, _gp, _vp, _vp, C.c_int32, C.c_int32, C.c_uint32, _sp, _vp]),
    "mlens_far_field_get_info": (C.c_int, [_vp, C.POINTER(mlens_far_field_info)]),
    "mlens_far_field_export": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mlens_save_far_field": (C.c_int, [_vp, C.c_char_p]),
    "mlens_load_far_field": (C.c_int, [_vp, C.c_char_p, _vp]),
    "mlens_ff_eval": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, _vp, _vp, _vp, C.POINTER(C.c_float), _vp]),
    "mlens_destroy": (None, [_vp]),
    "mlens_last_error": (C.c_char_p, []),
    "mlens_set_device_memory_limit": (C.c_int, [C.c_uint64]),
    "mlens_debug_wait_probe": (C.c_int, [C.c_int32]),
    "mlens_device_memory_in_use": (C.c_uint64, []),
    "mlens_version": (C.c_int, []),
}


def load(path: Optional[str] = None):
    """Open libmlens.so (built by build.py) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libmlens.so not found at {p}: build it first (python -m paper_1703_09707_gb300.build "
                               "or __graft_entry__.build()); there is no fallback")
        L = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = L
        return L


def _check(rc: int):
    if rc != MLENS_OK:
        raise MlensError(rc, mlens_last_error())


def mlens_last_error() -> str:
    return load().mlens_last_error().decode()


def mlens_set_device_memory_limit(nbytes: int):
    _check(load().mlens_set_device_memory_limit(int(nbytes)))


def mlens_debug_wait_probe(on: bool):
    """Test aid: tensor-core completion waits poll an mbarrier nothing arrives on
    (their bounded-wait failure path runs; calls report MLENS_ERR_CUDA)."""
    _check(load().mlens_debug_wait_probe(1 if on else 0))


def mlens_device_memory_in_use() -> int:
    return int(load().mlens_device_memory_in_use())


def mlens_version() -> int:
    return load().mlens_version()


def grid(g) -> mlens_grid:
    if isinstance(g, mlens_grid):
        return g
    if hasattr(g, "astuple"):
        g = g.astuple()
    x0, x1, y0, y1, nx, ny = g
    return mlens_grid(float(x0), float(x1), float(y0), float(y1), int(nx), int(ny))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dev_ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    if hasattr(t, "data_ptr"):
        if not t.is_cuda:
            raise ValueError("device buffer must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError("device buffer must be contiguous")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


def _check_tensor(t, what: str, min_elems: int, dtypes):
    """Check what the C side cannot see in a torch tensor: its element type,
    contiguity and that it holds at least `min_elems` elements (ValueError).
    Anything that is not a tensor (an integer address) is not checked."""
    if not hasattr(t, "data_ptr"):
        return
    names = {str(d).replace("torch.", "") for d in dtypes}
    if str(t.dtype).replace("torch.", "") not in names:
        raise ValueError(f"{what} must have dtype {' or '.join(sorted(names))}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() < min_elems:
        raise ValueError(f"{what} holds {t.numel()} elements, needs at least {min_elems}")


def _counts_buf(counts, src: mlens_grid) -> C.c_void_p:
    """A source map: int32 or uint32, src.nx * src.ny elements at least, on the device."""
    _check_tensor(counts, "counts", int(src.nx) * int(src.ny), ("int32", "uint32"))
    return _dev_ptr(counts)


class Ctx:
    """Owns one mlens_ctx*."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle and self.handle.value:
            load().mlens_destroy(self.handle)
            self.handle = C.c_void_p(0)


def mlens_create(xy: np.ndarray, m: np.ndarray, kappa_c: float, gamma1: float, gamma2: float,
                 precision=MLENS_PREC_FP32) -> Ctx:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1)
    if xy.shape[0] != m.shape[0]:
        raise ValueError("xy and m disagree on the number of stars")
    h = C.c_void_p(0)
    _check(load().mlens_create(C.byref(h), xy.ctypes.data_as(_dp), m.ctypes.data_as(_dp), m.shape[0],
                               float(kappa_c), float(gamma1), float(gamma2), int(precision)))
    return Ctx(h.value)


def mlens_set_precision(ctx: Ctx, precision):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    _check(load().mlens_set_precision(ctx.handle, int(precision)))


def mlens_set_tuning(ctx: Ctx, rays_per_thread: int, star_stage: int = 0, fma_pairs: int = 1):
    _check(load().mlens_set_tuning(ctx.handle, int(rays_per_thread), int(star_stage), int(fma_pairs)))


def mlens_set_star_split(ctx: Ctx, split: int):
    """0 = automatic, 1 = never, 2 .. 8 CTAs per tile in a cluster, 9 .. 4096 through global memory."""
    _check(load().mlens_set_star_split(ctx.handle, int(split)))


def mlens_star_split_for(ctx: Ctx, rays) -> int:
    out = C.c_int32(0)
    g = grid(rays)
    _check(load().mlens_star_split_for(ctx.handle, C.byref(g), C.byref(out)))
    return int(out.value)


def mlens_shoot(ctx: Ctx, rays, src, counts, flags: int = 0, stats: bool = False, stream=None):
    st = mlens_stats()
    g, s = grid(rays), grid(src)
    _check(load().mlens_shoot(ctx.handle, C.byref(g), C.byref(s), _counts_buf(counts, s), int(flags),
                              C.byref(st) if stats else None, _stream_ptr(stream)))
    return st.asdict() if stats else None


def mlens_shoot_beta(ctx: Ctx, rays, src, counts, beta, flags: int = 0, stats: bool = False, stream=None):
    st = mlens_stats()
    g, s = grid(rays), grid(src)
    _check(load().mlens_shoot_beta(ctx.handle, C.byref(g), C.byref(s), _counts_buf(counts, s), _dev_ptr(beta),
                                   int(flags), C.byref(st) if stats else None, _stream_ptr(stream)))
    return st.asdict() if stats else None


MLENS_ROW_ALIGN = 32


def mlens_shoot_rows(ctx: Ctx, rays, rows, src, counts, beta=None, flags: int = 0, stats: bool = False,
                     stream=None):
    """Ray rows [rows[0], rows[1]) of the grid (multiples of MLENS_ROW_ALIGN, or the
    end at rays.ny); beta (optional) holds the whole grid's records."""
    st = mlens_stats()
    g, s = grid(rays), grid(src)
    _check(load().mlens_shoot_rows(ctx.handle, C.byref(g), int(rows[0]), int(rows[1]), C.byref(s),
                                   _counts_buf(counts, s), _dev_ptr(beta), int(flags),
                                   C.byref(st) if stats else None, _stream_ptr(stream)))
    return st.asdict() if stats else None


def mlens_trace(ctx: Ctx, theta: np.ndarray, stream=None) -> np.ndarray:
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 2)
    out = np.empty_like(th)
    _check(load().mlens_trace(ctx.handle, th.ctypes.data_as(_dp), th.shape[0], out.ctypes.data_as(_dp),
                              _stream_ptr(stream)))
    return out


def mlens_bin(beta, n: int, src, counts, flags: int = 0, stats: bool = False, stream=None):
    st = mlens_stats()
    s = grid(src)
    _check(load().mlens_bin(_dev_ptr(beta), int(n), C.byref(s), _dev_ptr(counts), int(flags),
                            C.byref(st) if stats else None, _stream_ptr(stream)))
    return st.asdict() if stats else None


def mlens_bin_grid(beta, rays, src, counts, flags: int = 0, stats: bool = False, stream=None):
    """beta: rays.nx * rays.ny float-pair records in ray-grid row order."""
    st = mlens_stats()
    g, s = grid(rays), grid(src)
    _check(load().mlens_bin_grid(_dev_ptr(beta), C.byref(g), C.byref(s), _dev_ptr(counts), int(flags),
                                 C.byref(st) if stats else None, _stream_ptr(stream)))
    return st.asdict() if stats else None


def mlens_convolve_workspace(src, profile: int, size: float) -> int:
    s = grid(src)
    out = C.c_uint64(0)
    _check(load().mlens_convolve_workspace(C.byref(s), int(profile), float(size), C.byref(out)))
    return int(out.value)


def mlens_convolve(counts, src, profile: int, size: float, out, scale: float = 1.0, work=None, stream=None):
    """counts: CUDA int32/uint32 tensor of src.ny*src.nx; out: CUDA float32 tensor of the
    same size; work: optional CUDA byte tensor of mlens_convolve_workspace bytes (the
    call is then asynchronous)."""
    s = grid(src)
    nb = 0 if work is None else int(work.numel() * work.element_size())
    _check(load().mlens_convolve(_dev_ptr(counts), C.byref(s), int(profile), float(size), float(scale),
                                 _dev_ptr(out), _dev_ptr(work), nb, _stream_ptr(stream)))


def mlens_light_curve(map_, src, b0, b1, npts: int, out, stream=None):
    s = grid(src)
    _check(load().mlens_light_curve(_dev_ptr(map_), C.byref(s), float(b0[0]), float(b0[1]), float(b1[0]),
                                    float(b1[1]), int(npts), _dev_ptr(out), _stream_ptr(stream)))


def mlens_magnification_scale(rays, src) -> float:
    g, s = grid(rays), grid(src)
    out = C.c_double(0.0)
    _check(load().mlens_magnification_scale(C.byref(g), C.byref(s), C.byref(out)))
    return float(out.value)


def mlens_shoot_noalloc(stars, n: int, kappa_c: float, gamma1: float, gamma2: float, rays, src, counts,
                        flags: int = 0, stats: bool = False, stream=None):
    """stars: contiguous CUDA float32 tensor holding n records (x, y, m, unused),
    shape (n, 4) or flat; it is read on the device, so its type and length are
    checked here before the call (ValueError)."""
    st = mlens_stats()
    g, s = grid(rays), grid(src)
    n = int(n)
    if n < 0:
        raise ValueError("n must be >= 0")
    if hasattr(stars, "data_ptr") and stars.dim() > 1 and stars.shape[-1] != 4:
        raise ValueError(f"stars must be (n, 4) records or flat, got shape {tuple(stars.shape)}")
    _check_tensor(stars, "stars", 4 * n, ("float32",))
    _check_tensor(counts, "counts", int(s.nx) * int(s.ny), ("int32", "uint32"))
    sp, cp = _dev_ptr(stars), _dev_ptr(counts)
    _check(load().mlens_shoot_noalloc(sp, n, float(kappa_c), float(gamma1), float(gamma2),
                                      C.byref(g), C.byref(s), cp, int(flags),
                                      C.byref(st) if stats else None, _stream_ptr(stream)))
    return st.asdict() if stats else None


class Batch:
    """Owns one mlens_batch* (and keeps its contexts and maps referenced)."""

    def __init__(self, handle: int, keep):
        self.handle = C.c_void_p(handle)
        self._keep = keep

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle and self.handle.value:
            load().mlens_batch_destroy(self.handle)
            self.handle = C.c_void_p(0)


def _batch_arrays(ctxs, rays, srcs, counts):
    nf = len(ctxs)
    if not (len(rays) == len(srcs) == len(counts) == nf):
        raise ValueError("ctxs, rays, srcs and counts must have one entry per field")
    cx = (_vp * nf)(*[c.handle.value for c in ctxs])
    ga = (mlens_grid * nf)(*[grid(g) for g in rays])
    sa = (mlens_grid * nf)(*[grid(g) for g in srcs])
    pa = (_vp * nf)(*[_dev_ptr(t).value for t in counts])
    return nf, cx, ga, sa, pa


def mlens_batch_create(ctxs, rays, srcs, counts, flags: int = 0) -> Batch:
    nf, cx, ga, sa, pa = _batch_arrays(ctxs, rays, srcs, counts)
    h = C.c_void_p(0)
    _check(load().mlens_batch_create(C.byref(h), cx, nf, ga, sa, pa, int(flags)))
    return Batch(h.value, (list(ctxs), list(counts)))


def mlens_batch_set_tuning(b: Batch, rays_per_thread: int, star_stage: int = 0, fma_pairs: int = 1):
    _check(load().mlens_batch_set_tuning(b.handle, int(rays_per_thread), int(star_stage), int(fma_pairs)))


def mlens_batch_tune(b: Batch, stream=None):
    """Returns (rays_per_thread, star_stage, fma_pairs, best_ms)."""
    r, s, f, ms = C.c_int32(0), C.c_int32(0), C.c_int32(0), C.c_double(0.0)
    _check(load().mlens_batch_tune(b.handle, _stream_ptr(stream), C.byref(r), C.byref(s), C.byref(f), C.byref(ms)))
    return int(r.value), int(s.value), int(f.value), float(ms.value)


def mlens_batch_run(b: Batch, stats: bool = False, stream=None):
    nf = len(b._keep[0])
    st = (mlens_stats * nf)()
    _check(load().mlens_batch_run(b.handle, st if stats else None, _stream_ptr(stream)))
    return [x.asdict() for x in st] if stats else None


def mlens_batch_destroy(b: Batch):
    b.close()


def mlens_shoot_batch(ctxs, rays, srcs, counts, flags: int = 0, stats: bool = False, stream=None):
    nf, cx, ga, sa, pa = _batch_arrays(ctxs, rays, srcs, counts)
    st = (mlens_stats * nf)()
    _check(load().mlens_shoot_batch(cx, nf, ga, sa, pa, int(flags), st if stats else None, _stream_ptr(stream)))
    return [x.asdict() for x in st] if stats else None


def fit_params(**kw) -> mlens_fit_params:
    """Defaults of mlens_fit_params_default, with keyword overrides."""
    p = mlens_fit_params()
    load().mlens_fit_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def mlens_fit_far_field(ctx: Ctx, rays, params: mlens_fit_params = None, stream=None) -> dict:
    g = grid(rays)
    rep = mlens_fit_report()
    _check(load().mlens_fit_far_field(ctx.handle, C.byref(g), C.byref(params) if params is not None else None,
                                      C.byref(rep), _stream_ptr(stream)))
    return rep.asdict()


def mlens_shoot_learned(ctx: Ctx, rays, src, counts, beta=None, rows=(0, 0), flags: int = 0, stats: bool = False,
                        stream=None):
    st = mlens_stats()
    g, s = grid(rays), grid(src)
    _check(load().mlens_shoot_learned(ctx.handle, C.byref(g), C.byref(s), _dev_ptr(counts), _dev_ptr(beta),
                                      int(rows[0]), int(rows[1]), int(flags), C.byref(st) if stats else None,
                                      _stream_ptr(stream)))
    return st.asdict() if stats else None


def mlens_far_field_get_info(ctx: Ctx) -> mlens_far_field_info:
    info = mlens_far_field_info()
    _check(load().mlens_far_field_get_info(ctx.handle, C.byref(info)))
    return info


def mlens_far_field_export(ctx: Ctx) -> dict:
    """All exportable far-field state as numpy arrays."""
    info = mlens_far_field_get_info(ctx)
    nrc = info.cells_x * info.cells_y
    out = dict(params=np.empty(info.n_params, np.float32), latents=np.empty((nrc, info.latent_dim), np.float32),
               flags=np.empty(nrc, np.int32), coef=np.empty((nrc, info.target_order + 1, 2), np.float64),
               cell_start=np.empty(info.grid_nx * info.grid_ny + 1, np.int32),
               val_max_net=np.empty(nrc, np.float32), val_max_series=np.empty(nrc, np.float32))
    ptr = {k: v.ctypes.data_as(_vp) for k, v in out.items()}
    _check(load().mlens_far_field_export(ctx.handle, ptr["params"], ptr["latents"], ptr["flags"], ptr["coef"],
                                         ptr["cell_start"], ptr["val_max_net"], ptr["val_max_series"]))
    out["info"] = info
    return out


def mlens_save_far_field(ctx: Ctx, path: str):
    _check(load().mlens_save_far_field(ctx.handle, path.encode()))


def mlens_load_far_field(ctx: Ctx, path: str, stream=None):
    _check(load().mlens_load_far_field(ctx.handle, path.encode(), _stream_ptr(stream)))


def mlens_ff_eval(params, z, u, t=None, y=None, grads=None, dz=None, stream=None) -> float:
    """Network kernel on explicit CUDA tensors (float32); returns the loss."""
    loss = C.c_float(0.0)
    n = int(z.shape[0])
    _check(load().mlens_ff_eval(_dev_ptr(params), _dev_ptr(z), _dev_ptr(u), _dev_ptr(t), n, _dev_ptr(y),
                                _dev_ptr(grads), _dev_ptr(dz), C.byref(loss), _stream_ptr(stream)))
    return float(loss.value)


def mlens_destroy(ctx: Ctx):
    ctx.close()
