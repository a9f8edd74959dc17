"""CPU pin of the double-float arithmetic the far-field coefficient kernel uses for the
order-0 term (farfield.cu: df_two_sum, df_add, df_mul, df_mulf, df_rcp): the same
float32 operation sequences, evaluated with IEEE float32 arithmetic in numpy (FMAs
through float64, where the products are exact), against float64 results.  Pins the
accuracy the design relies on: TwoSum exact, a product to ~2^-44, the reciprocal
below 2^-45 (one Newton step on the correctly rounded float reciprocal)."""
import numpy as np

f32 = np.float32


def fma32(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(f32)


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
