"""CPU-side checks of the C ABI: libmlens.so builds, loads without a GPU, exports
every function include/mlens.h declares with the binding's names, and rejects bad
arguments with MLENS_ERR_ARG before touching a device.  No compute call runs here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from paper_1703_09707_gb300 import build as B
from paper_1703_09707_gb300 import mlens as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mlens_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_functions()
    assert {"mlens_create", "mlens_shoot", "mlens_destroy", "mlens_last_error"} <= names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
        assert n in M.SIGNATURES, f"{n} has no binding"
    assert set(M.SIGNATURES) <= names


def test_version(lib):
    assert M.mlens_version() >= 10000


def test_bad_arguments_are_rejected_before_any_device_call(lib):
    dp = C.POINTER(C.c_double)
    xy = np.zeros((2, 2))
    m = np.ones(2)
    h = C.c_void_p(0)
    assert lib.mlens_create(None, xy.ctypes.data_as(dp), m.ctypes.data_as(dp), 2, 0.0, 0.0, 0.0, 0) == M.MLENS_ERR_ARG
    assert lib.mlens_create(C.byref(h), xy.ctypes.data_as(dp), m.ctypes.data_as(dp), -1, 0, 0, 0, 0) == M.MLENS_ERR_ARG
    assert lib.mlens_create(C.byref(h), None, None, 2, 0.0, 0.0, 0.0, 0) == M.MLENS_ERR_ARG
    assert lib.mlens_create(C.byref(h), xy.ctypes.data_as(dp), m.ctypes.data_as(dp), 2, float("nan"), 0, 0,
                            0) == M.MLENS_ERR_ARG
    assert lib.mlens_create(C.byref(h), xy.ctypes.data_as(dp), m.ctypes.data_as(dp), 2, 0.0, 0.0, 0.0,
                            7) == M.MLENS_ERR_ARG
    bad = np.array([[0.0, np.inf], [1.0, 1.0]])
    assert lib.mlens_create(C.byref(h), bad.ctypes.data_as(dp), m.ctypes.data_as(dp), 2, 0, 0, 0, 0) == M.MLENS_ERR_ARG
    assert "star 0" in M.mlens_last_error()
    negm = np.array([1.0, -1.0])
    assert lib.mlens_create(C.byref(h), xy.ctypes.data_as(dp), negm.ctypes.data_as(dp), 2, 0, 0, 0,
                            0) == M.MLENS_ERR_ARG
    assert h.value is None
    g = M.mlens_grid(-1.0, 1.0, -1.0, 1.0, 4, 4)
    assert lib.mlens_shoot(None, C.byref(g), C.byref(g), C.c_void_p(16), 0, None, None) == M.MLENS_ERR_ARG
    assert "context" in M.mlens_last_error()
    assert lib.mlens_set_tuning(None, 8, 0, 0) == M.MLENS_ERR_ARG
    assert lib.mlens_set_star_split(None, 2) == M.MLENS_ERR_ARG
    out = C.c_int32(-7)
    assert lib.mlens_star_split_for(None, C.byref(g), C.byref(out)) == M.MLENS_ERR_ARG and out.value == -7
    assert lib.mlens_set_precision(None, 0) == M.MLENS_ERR_ARG
    badg = M.mlens_grid(1.0, -1.0, -1.0, 1.0, 4, 4)
    assert lib.mlens_bin(C.c_void_p(16), 4, C.byref(badg), C.c_void_p(16), 0, None, None) == M.MLENS_ERR_ARG
    zg = M.mlens_grid(-1.0, 1.0, -1.0, 1.0, 0, 4)
    assert lib.mlens_bin(C.c_void_p(16), 4, C.byref(zg), C.c_void_p(16), 0, None, None) == M.MLENS_ERR_ARG
    assert lib.mlens_bin(C.c_void_p(16), 4, C.byref(g), C.c_void_p(18), 0, None, None) == M.MLENS_ERR_ARG
    assert lib.mlens_bin(C.c_void_p(16), 4, C.byref(g), C.c_void_p(16), 8, None, None) == M.MLENS_ERR_ARG
    bigr = M.mlens_grid(-1.0, 1.0, -1.0, 1.0, 1 << 21, 4)
    assert lib.mlens_bin_grid(C.c_void_p(16), C.byref(bigr), C.byref(g), C.c_void_p(16), 0, None,
                              None) == M.MLENS_ERR_ARG
    assert lib.mlens_bin_grid(C.c_void_p(16), None, C.byref(g), C.c_void_p(16), 0, None, None) == M.MLENS_ERR_ARG
    assert lib.mlens_bin_grid(C.c_void_p(24), C.byref(g), C.byref(g), C.c_void_p(16), 0, None,
                              None) == M.MLENS_ERR_ARG
    assert lib.mlens_bin_grid(None, C.byref(g), C.byref(g), C.c_void_p(16), 0, None, None) == M.MLENS_ERR_ARG
    # convolution and light curves: argument checks come before any device call
    assert lib.mlens_convolve(C.c_void_p(16), C.byref(badg), 1, 0.1, 1.0, C.c_void_p(1 << 20), None, 0, None) == M.MLENS_ERR_ARG
    assert lib.mlens_convolve(None, C.byref(g), 1, 0.1, 1.0, C.c_void_p(1 << 20), None, 0, None) == M.MLENS_ERR_ARG
    assert lib.mlens_convolve(C.c_void_p(16), C.byref(g), 1, -0.1, 1.0, C.c_void_p(1 << 20), None, 0, None) == M.MLENS_ERR_ARG
    assert lib.mlens_convolve(C.c_void_p(16), C.byref(g), 1, 0.1, float("inf"), C.c_void_p(1 << 20),
                              None, 0, None) == M.MLENS_ERR_ARG
    assert lib.mlens_convolve(C.c_void_p(16), C.byref(g), 1, 0.1, 1.0, C.c_void_p(32), None, 0, None) == M.MLENS_ERR_ARG
    assert "overlap" in M.mlens_last_error()
    # a workspace that is too small or misaligned is refused before any device call
    assert lib.mlens_convolve(C.c_void_p(16), C.byref(g), 1, 0.1, 1.0, C.c_void_p(1 << 20), C.c_void_p(1 << 24), 16,
                              None) == M.MLENS_ERR_ARG
    assert lib.mlens_convolve(C.c_void_p(16), C.byref(g), 1, 0.1, 1.0, C.c_void_p(1 << 20), C.c_void_p((1 << 24) + 8),
                              1 << 20, None) == M.MLENS_ERR_ARG
    wb = C.c_uint64(0)
    mapg = M.mlens_grid(-2.0, 2.0, -1.0, 1.0, 100, 40)  # 0.04 x 0.05 pixels
    assert lib.mlens_convolve_workspace(C.byref(mapg), 0, 0.1, C.byref(wb)) == M.MLENS_OK
    kx, ky = 10, 8  # ceil(0.4 / 0.04), ceil(0.4 / 0.05)
    r256 = lambda b: (b + 255) // 256 * 256  # noqa: E731
    assert wb.value == r256(4 * (2 * kx + 1 + 2 * ky + 1)) + r256(4 * 4000)
    assert lib.mlens_convolve_workspace(C.byref(mapg), 1, 0.1, C.byref(wb)) == M.MLENS_OK
    assert wb.value == r256(4 * (2 * 2 + 1)) + r256(8 * 4000)  # support rows |dj| <= 2
    assert lib.mlens_convolve_workspace(C.byref(mapg), 0, 0.0, C.byref(wb)) == M.MLENS_ERR_ARG
    assert lib.mlens_light_curve(C.c_void_p(16), C.byref(g), 0.0, 0.0, 1.0, 1.0, 0, C.c_void_p(16),
                                 None) == M.MLENS_ERR_ARG
    assert lib.mlens_light_curve(C.c_void_p(16), C.byref(g), 0.0, float("nan"), 1.0, 1.0, 5, C.c_void_p(16),
                                 None) == M.MLENS_ERR_ARG
    sc = C.c_double(0.0)
    rays = M.mlens_grid(-10.0, 10.0, -10.0, 10.0, 1000, 1000)
    srcg = M.mlens_grid(-5.0, 5.0, -4.0, 4.0, 100, 40)
    assert lib.mlens_magnification_scale(C.byref(rays), C.byref(srcg), C.byref(sc)) == M.MLENS_OK
    assert abs(sc.value - 0.02) < 1e-16
    assert lib.mlens_magnification_scale(C.byref(badg), C.byref(srcg), C.byref(sc)) == M.MLENS_ERR_ARG
    lib.mlens_destroy(None)  # must be a no-op


def test_batch_arguments_rejected_without_a_device(lib):
    g = (M.mlens_grid * 1)(M.mlens_grid(-1.0, 1.0, -1.0, 1.0, 4, 4))
    ctxs = (C.c_void_p * 1)(None)
    cnt = (C.c_void_p * 1)(16)
    h = C.c_void_p(0)
    assert lib.mlens_batch_create(C.byref(h), ctxs, 1, g, g, cnt, 0) == M.MLENS_ERR_ARG
    assert "field 0" in M.mlens_last_error()
    assert lib.mlens_batch_create(C.byref(h), ctxs, 0, g, g, cnt, 0) == M.MLENS_ERR_ARG
    assert lib.mlens_batch_run(None, None, None) == M.MLENS_ERR_ARG
    assert lib.mlens_batch_set_tuning(None, 8, 0, 0) == M.MLENS_ERR_ARG
    lib.mlens_batch_destroy(None)


def test_noalloc_size_limit_rejected_without_a_device(lib):
    g = M.mlens_grid(-1.0, 1.0, -1.0, 1.0, 4, 4)
    rc = lib.mlens_shoot_noalloc(C.c_void_p(16), 65537, 0.0, 0.0, 0.0, C.byref(g), C.byref(g), C.c_void_p(16), 0,
                                 None, None)
    assert rc == M.MLENS_ERR_ARG and "65536" in M.mlens_last_error()


def test_noalloc_binding_refuses_mismatched_buffers_before_any_call():
    """mlens_shoot_noalloc reads the caller's star records on the device, so the
    binding checks a tensor's type, shape and length against n (and the map's length
    against the source grid) before it reaches the library; CPU tensors show the
    checks without a GPU."""
    torch = pytest.importorskip("torch")
    g = W.Grid(-1.0, 1.0, -1.0, 1.0, 8, 8)
    counts = torch.zeros(64, dtype=torch.int32)
    cases = [
        (torch.zeros((10, 4), dtype=torch.float64), 10, counts, "dtype"),       # float64 records
        (torch.zeros((9, 4), dtype=torch.float32), 10, counts, "at least 40"),  # too few records for n
        (torch.zeros(39, dtype=torch.float32), 10, counts, "at least 40"),      # flat, too short
        (torch.zeros((10, 3), dtype=torch.float32), 10, counts, "shape"),       # not 4-wide
        (torch.zeros((10, 4), dtype=torch.float32), 10, torch.zeros(63, dtype=torch.int32), "at least 64"),
        (torch.zeros((10, 4), dtype=torch.float32), 10, torch.zeros(64, dtype=torch.float32), "dtype"),
        (torch.zeros((10, 4), dtype=torch.float32), 10, counts, "CUDA tensor"),  # right shape, host memory
        (torch.zeros((10, 4), dtype=torch.float32), -1, counts, "n must"),
    ]
    for stars, n, cnt, msg in cases:
        with pytest.raises(ValueError, match=msg):
            M.mlens_shoot_noalloc(stars, n, 0.0, 0.0, 0.0, g, g, cnt)
