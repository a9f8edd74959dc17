"""CPU pin of the double-float arithmetic the far-field coefficient kernel uses for the
order-0 term (farfield.cu: df_two_sum, df_add, df_mul, df_mulf, df_rcp): the same
float32 operation sequences, evaluated with IEEE float32 arithmetic in numpy, against
float64 results.  The FMAs are the device's: a*b + c rounded once to float32 (the
product is exact in float64; the sum is carried exactly as a float64 pair and rounded
once, checked against exact rational arithmetic).  Pins the accuracy the design relies
on: TwoSum exact, a product to ~2^-44, the reciprocal below 2^-45 (one Newton step on
the correctly rounded float reciprocal)."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def fma32(a, b, c):
    """float32 fused multiply-add with a single rounding (round to nearest even).
    p = a*b is exact in float64 (two 24-bit significands); s + e = p + c exactly
    (Knuth's TwoSum in float64).  Rounding s to float32 equals rounding the exact sum
    unless s sits exactly on the midpoint of two float32 neighbours and e != 0; the
    exact sum then lies on e's side of the midpoint."""
    a, b, c = (np.asarray(v, dtype=np.float64) for v in (a, b, c))
    p = a * b
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    r = s.astype(f32)
    lo = np.where(r.astype(np.float64) <= s, r, np.nextafter(r, f32(-np.inf))).astype(np.float64)
    hi = np.nextafter(lo.astype(f32), f32(np.inf)).astype(np.float64)
    mid = (s - lo == (hi - lo) / 2) & (e != 0)
    out = np.where(mid, np.where(e > 0, hi, lo), r.astype(np.float64))
    return out.astype(f32)


def two_sum(a, b):
    s = (a + b).astype(f32)
    bb = (s - a).astype(f32)
    return s, ((a - (s - bb).astype(f32)).astype(f32) + (b - bb).astype(f32)).astype(f32)


def df_norm(a, b):
    s = (a + b).astype(f32)
    return s, (b - (s - a).astype(f32)).astype(f32)


def df_add(a, b):
    sh, sl = two_sum(a[0], b[0])
    return df_norm(sh, (sl + (a[1] + b[1]).astype(f32)).astype(f32))


def df_mul(a, b):
    p = (a[0] * b[0]).astype(f32)
    e = fma32(a[0], b[0], -p)
    return df_norm(p, fma32(a[0], b[1], fma32(a[1], b[0], e)))


def df_mulf(a, b):
    p = (a[0] * b).astype(f32)
    e = fma32(a[0], b, -p)
    return df_norm(p, fma32(a[1], b, e))


def df_rcp(a):
    y = (1.0 / a[0].astype(np.float64)).astype(f32)  # the correctly rounded float reciprocal
    ay = df_mulf(a, y)
    r = df_add((np.ones_like(y), np.zeros_like(y)), (-ay[0], -ay[1]))
    return df_norm(y, (y * r[0]).astype(f32))


def value(a):
    return a[0].astype(np.float64) + a[1].astype(np.float64)


def pairs(rng, k):
    x = rng.uniform(0.5, 2.0, k) * 10.0 ** rng.integers(-6, 7, k) * rng.choice([-1.0, 1.0], k)
    h = x.astype(f32)
    return h, (x - h.astype(np.float64)).astype(f32)


def test_two_sum_is_exact():
    rng = np.random.default_rng(1)
    a = (rng.normal(0, 1, 200_000) * 10.0 ** rng.integers(-5, 6, 200_000)).astype(f32)
    b = (rng.normal(0, 1, 200_000) * 10.0 ** rng.integers(-5, 6, 200_000)).astype(f32)
    s, e = two_sum(a, b)
    # a + b of two floats is exact in float64, so the pair must reproduce it exactly
    assert np.array_equal(s.astype(np.float64) + e.astype(np.float64), a.astype(np.float64) + b.astype(np.float64))


def test_double_float_product_and_reciprocal_accuracy():
    rng = np.random.default_rng(2)
    a, b = pairs(rng, 200_000), pairs(rng, 200_000)
    prod = df_mul(a, b)
    rel = np.abs(value(prod) - value(a) * value(b)) / np.abs(value(a) * value(b))
    assert rel.max() < 2.0 ** -44
    rcp = df_rcp(a)
    rel = np.abs(value(rcp) - 1.0 / value(a)) * np.abs(value(a))
    assert rel.max() < 2.0 ** -45


def _fma32_exact(a, b, c):
    """a*b + c in exact rational arithmetic, rounded once to float32 (nearest even)."""
    x = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    lo = f32(float(x))  # a float32 next to x (possibly not the nearest)
    cands = {lo, np.nextafter(lo, f32(np.inf)), np.nextafter(lo, f32(-np.inf))}
    best = min(cands, key=lambda v: (abs(Fraction(float(v)) - x), int(np.array(v).view(np.uint32)) & 1))
    return best


def test_fma32_rounds_once():
    """The pin's FMA against exact rational arithmetic: random operands, and operands
    built so that a*b + c rounded to float64 lands exactly on a float32 midpoint (the
    case a float64-then-float32 evaluation gets wrong)."""
    rng = np.random.default_rng(4)
    a = (rng.normal(0, 1, 3000) * 2.0 ** rng.integers(-20, 20, 3000)).astype(f32)
    b = (rng.normal(0, 1, 3000) * 2.0 ** rng.integers(-20, 20, 3000)).astype(f32)
    c = (-(a.astype(np.float64) * b) * (1 + rng.normal(0, 1e-3, 3000))).astype(f32)
    # midpoint cases: a*b exactly on a float32 midpoint in [1, 2) (a, b = 1 + odd/4096,
    # so the product's last bit is 2^-24), and c = +-2^-60, far below a float64 ulp
    k = 2 * rng.integers(0, 600, 200) + 1
    j = 2 * rng.integers(0, 600, 200) + 1
    a2 = (1.0 + k / 4096.0).astype(f32)
    b2 = (1.0 + j / 4096.0).astype(f32)
    c2 = (rng.choice([-1.0, 1.0], 200) * 2.0 ** -60).astype(f32)
    A, B, Cc = np.concatenate([a, a2]), np.concatenate([b, b2]), np.concatenate([c, c2])
    got = fma32(A, B, Cc)
    want = np.array([_fma32_exact(x, y, z) for x, y, z in zip(A, B, Cc)], dtype=f32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # the midpoint cases do occur, and the double-rounded evaluation misses some of them
    naive = (A.astype(np.float64) * B + Cc).astype(f32)
    assert np.any(naive.view(np.uint32) != want.view(np.uint32))
