"""CPU pin of the binning kernels' quick test (mlens_dev.cuh, pair_axis_quick).

The kernels decide a record's pixel from its hi part alone when no pixel edge lies
within del of u = fl(fl(bh - x0h) sh), with del = 2^-21 |u| + 2 |bl| |sh| + t_q
(t_q = 2 |x0l| |sh| + 2^-100 rounded up); otherwise the exact float-pair rule runs.
Here the quick test is evaluated with IEEE float32 arithmetic (numpy; the FMAs
through float64, where the products are exact) on records placed on, next to and
across pixel edges, for maps whose origin is and is not a float32.  Wherever the
quick test decides, its pixel must equal the oracle's exact float-pair rule, so the
error bound the decision rests on is checked without a GPU."""
import numpy as np
import pytest

import oracle
import workloads as W

f32 = np.float32


def axis_constants(x0: float, x1: float, n: int):
    """The per-axis constants the library builds for the rule and the quick test."""
    s = n / (x1 - x0)
    x0h = f32(x0)
    x0l = f32(x0 - float(x0h))
    sh = f32(s)
    sl = f32(s - float(sh))
    sh2 = f32(2.0 * abs(float(sh)))
    tq_exact = 2.0 * abs(float(x0l)) * abs(float(sh)) + 2.0 ** -100
    tq = f32(tq_exact)
    if float(tq) < tq_exact:
        tq = np.nextafter(tq, f32(np.inf))
    return x0h, x0l, sh, sl, sh2, tq


def fma32(a, b, c):
    """fma(a, b, c) rounded to float32 (the float32 product is exact in float64)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def quick_axis(bh, bl, x0, x1, n):
    """(decided, pixel) per record: pixel in [0, n) or -1, valid where decided."""
    x0h, x0l, sh, sl, sh2, tq = axis_constants(x0, x1, n)
    with np.errstate(over="ignore", invalid="ignore"):
        d = (bh - x0h).astype(f32)
        u = (d * sh).astype(f32)
        inner = fma32(np.abs(bl), np.full_like(bl, sh2), np.full_like(bl, tq))
        dl = fma32(np.abs(u), np.full_like(u, f32(2.0 ** -21)), inner)
        lo = np.floor((u - dl).astype(f32))
        hi = (u + dl).astype(f32)
        decided = hi < (lo + f32(1.0)).astype(f32)
    pix = np.where((lo >= 0) & (lo < n), lo, -1).astype(np.int64)
    return decided, pix


def edge_records(rng, k, x0, w, n):
    """hi/lo pairs on pixel edges, hi parts a few ulps off an edge, lo parts that
    straddle an edge, and uniform positions in and around the map."""
    i = rng.integers(-2, n + 2, k)
    edge = x0 + i * (w / n)
    bh = edge.astype(f32)
    mode = rng.integers(0, 4, k)
    ulp = np.spacing(np.abs(bh)).astype(f32)
    bh = np.where(mode == 1, bh + rng.integers(-3, 4, k).astype(f32) * ulp, bh).astype(f32)
    bl = np.where(mode == 0, (edge - bh.astype(np.float64)).astype(f32), f32(0))
    bl = np.where(mode == 2, (rng.uniform(-0.5, 0.5, k) * ulp).astype(f32), bl).astype(f32)
    bh = np.where(mode == 3, rng.uniform(x0 - 0.1 * w, x0 + 1.1 * w, k).astype(f32), bh).astype(f32)
    return bh, bl


@pytest.mark.parametrize("x0,w,n", [(-10.0, 20.0, 1024), (3.25 + 1e-9, 0.1, 4096), (-120.5, 300.0, 37),
                                    (-4.0, 8.0, 32768), (-2.0 / 3.0, 4.0 / 3.0, 999), (1e3 + 0.3, 1e-3, 64)])
def test_quick_test_decisions_equal_the_exact_rule(x0, w, n):
    rng = np.random.default_rng(n + 7)
    k = 400_000
    bh, bl = edge_records(rng, k, x0, w, n)
    decided, px = quick_axis(bh, bl, x0, x0 + w, n)
    # the oracle's exact rule on the x axis; y is a fixed record in pixel 0
    src = W.Grid(x0, x0 + w, 0.0, 1.0, n, 1)
    b4 = np.stack([bh, np.full(k, f32(0.5)), bl, np.zeros(k, f32)], 1).astype(f32)
    pix = oracle.pair_pixels(b4, src)
    exact = np.where(pix >= 0, pix % n, -1)
    bad = decided & (px != exact)
    assert not bad.any(), (int(bad.sum()), bh[bad][:3], bl[bad][:3], px[bad][:3], exact[bad][:3])
    # three in four of these records sit on or across an edge and must go to the exact
    # rule; where a float32 hi part is coarser than a pixel (the last map) all do
    assert decided.mean() < 0.6


@pytest.mark.parametrize("x0,w,n", [(-10.0, 20.0, 1024), (-75.0, 150.0, 8192), (3.25 + 1e-9, 0.1, 4096)])
def test_quick_test_decides_almost_every_ordinary_record(x0, w, n):
    """Records spread over the map with float-pair lo parts of a typical size: the
    quick test decides all but a fraction ~2 del of them (del ~1e-2 pixel on the
    0.1-wide map, whose pixels are ~100 float32 ulps of beta), each as the exact
    rule does."""
    rng = np.random.default_rng(n)
    k = 400_000
    b = rng.uniform(x0, x0 + w, k)
    bh = b.astype(f32)
    bl = (b - bh.astype(np.float64)).astype(f32)
    decided, px = quick_axis(bh, bl, x0, x0 + w, n)
    src = W.Grid(x0, x0 + w, 0.0, 1.0, n, 1)
    b4 = np.stack([bh, np.full(k, f32(0.5)), bl, np.zeros(k, f32)], 1).astype(f32)
    pix = oracle.pair_pixels(b4, src)
    exact = np.where(pix >= 0, pix % n, -1)
    assert decided.mean() > 0.95
    assert np.array_equal(px[decided], exact[decided])


def test_quick_test_defers_non_finite_components():
    """A non-finite hi or lo part makes u or del inf or NaN: the quick test never
    decides such a record (the kernels then run the exact rule, which reports it)."""
    x0, x1, n = -10.0, 10.0, 1024
    bh = np.array([np.nan, np.inf, -np.inf, 1.0, 1.0, 1.0], dtype=f32)
    bl = np.array([0.0, 0.0, 0.0, np.nan, np.inf, -np.inf], dtype=f32)
    decided, _ = quick_axis(bh, bl, x0, x1, n)
    assert not decided.any()


def test_quick_test_on_far_out_of_map_values():
    """Values far outside the map: where decided, the pixel is -1 (out), as the exact
    rule says."""
    x0, x1, n = -10.0, 10.0, 1024
    bh = np.array([3e38, -3e38, 1e30, -1e30, 1e6, -1e6, 20.0, -20.0], dtype=f32)
    bl = np.zeros_like(bh)
    decided, px = quick_axis(bh, bl, x0, x1, n)
    assert (px[decided] == -1).all()
