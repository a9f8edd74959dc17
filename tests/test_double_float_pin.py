"""CPU pin of the double-float arithmetic the far-field coefficient kernel uses for the
order-0 term (farfield.cu: df_two_sum, df_add, df_mul, df_mulf, df_sq_sum, df_rcp,
df_acc): the same float32 operation sequences, evaluated with IEEE float32 arithmetic
in numpy, against float64 results.  The FMAs are the device's: a*b + c rounded once to float32 (the
product is exact in float64; the sum is carried exactly as a float64 pair and rounded
once, checked against exact rational arithmetic).  Pins the accuracy the design relies
on: TwoSum exact, a product to ~2^-44, the reciprocal below 2^-45 from the correctly
rounded float reciprocal and below 2^-43 from any float within one ulp of it (the
hardware approximation the kernel starts from), one Newton step either way."""
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


def df_sq_sum(x, y):
    """x^2 + y^2 as the kernel forms it (df_sq_sum)."""
    px = (x[0] * x[0]).astype(f32)
    ex = fma32(x[0], x[0], -px)
    py = (y[0] * y[0]).astype(f32)
    ey = fma32(y[0], y[0], -py)
    sh, sl = two_sum(px, py)
    lx = fma32((x[0] + x[0]).astype(f32), x[1], ex)
    ly = fma32((y[0] + y[0]).astype(f32), y[1], ey)
    return df_norm(sh, (sl + (lx + ly).astype(f32)).astype(f32))


def df_rcp_from(a, y):
    """1/a as the kernel forms it from a float approximation y of 1/a_h (df_rcp)."""
    ay = df_mulf(a, y)
    r = ((np.ones_like(y) - ay[0]).astype(f32) - ay[1]).astype(f32)
    return df_norm(y, (y * r).astype(f32))


def df_acc(s, t):
    """The kernel's compensated running sum step (df_acc)."""
    uh, ul = two_sum(s[0], t[0])
    return uh, (s[1] + (ul + t[1]).astype(f32)).astype(f32)


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
    rcp = df_rcp_from(a, (1.0 / a[0].astype(np.float64)).astype(f32))  # the correctly rounded start
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


def test_order0_steps_accuracy():
    """The order-0 term's shortened steps: x^2 + y^2 to 2^-45 (x_l^2 and y_l^2 are left
    out), the reciprocal from any float within one ulp of 1/a_h (the hardware
    approximation's bound) to 2^-43 after one Newton step, and the stage sums as the
    kernel forms them (16 double-float terms per lane and stage by the compensated
    step, normalised, then added to the running total) to 2^-44 of the sum of the
    terms' magnitudes over 64 stages."""
    rng = np.random.default_rng(3)
    x, y = pairs(rng, 200_000), pairs(rng, 200_000)
    q = df_sq_sum(x, y)
    want = value(x) ** 2 + value(y) ** 2
    assert (np.abs(value(q) - want) / want).max() < 2.0 ** -45
    a = pairs(rng, 200_000)
    a = (np.abs(a[0]), np.where(a[0] < 0, -a[1], a[1]).astype(f32))  # r^2 > 0
    y0 = (1.0 / a[0].astype(np.float64)).astype(f32)
    for y in (y0, np.nextafter(y0, f32(np.inf)), np.nextafter(y0, f32(0))):
        rcp = df_rcp_from(a, y)
        rel = np.abs(value(rcp) - 1.0 / value(a)) * value(a)
        assert rel.max() < 2.0 ** -43
    stages, per, lanes = 64, 16, 256
    terms = pairs(rng, stages * per * lanes)
    th, tl = terms[0].reshape(stages, per, lanes), terms[1].reshape(stages, per, lanes)
    total = (np.zeros(lanes, dtype=f32), np.zeros(lanes, dtype=f32))
    for g in range(stages):
        s = (np.zeros(lanes, dtype=f32), np.zeros(lanes, dtype=f32))
        for k in range(per):
            s = df_acc(s, (th[g, k], tl[g, k]))
        total = df_add(total, df_norm(s[0], s[1]))
    exact = th.astype(np.float64).sum((0, 1)) + tl.astype(np.float64).sum((0, 1))
    mag = np.abs(th.astype(np.float64)).sum((0, 1))
    got = value(total)
    assert (np.abs(got - exact) / mag).max() < 2.0 ** -44
