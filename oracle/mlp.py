"""FP64 reference of the far-field network used by the learned-far-field variant
(TEST INFRASTRUCTURE: imported only by the tests).

The network is a per-cell latent code z_c (32 numbers) plus one shared MLP
34 -> 64 -> 64 -> 2 with SiLU activations:

    x  = [z_c, u]                  u = position in the cell (2)
    h1 = W1 x + b1,  a1 = silu(h1)  (64)
    h2 = W2 a1 + b2, a2 = silu(h2)  (64)
    y  = W3 a2 + b3                (2)

silu(v) = v * sigma(v) with sigma(v) = (1 + tanh(v/2)) / 2, and
silu'(v) = sigma(v) (1 + v (1 - sigma(v))).

The GPU runs the latent block of layer 1 and layer 2 on BF16 tensor cores with
FP32 accumulation; the position block of layer 1 (W1[:, 32:34] u) and layer 3
stay in FP32 so that the position keeps full precision.  With `bf16=True` this
reference rounds exactly the operands the GPU rounds to BF16 (round to nearest
even): z, W1[:, :32], a1 and W2 in the forward pass; dh2, W2, dh1 and
W1[:, :32] in the backward pass.  Everything else stays in FP64 here.  The loss
is mean over samples of |y - t|^2 (sum over the two outputs); its gradients are
returned for every parameter and for each sample's latent.
"""
from __future__ import annotations

import numpy as np

LATENT = 32
HIDDEN = 64
NIN = LATENT + 2
NOUT = 2


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (8-bit mantissa, round to nearest even) and return float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def sigma(v):
    return 0.5 * (1.0 + np.tanh(0.5 * v))


def silu(v):
    return v * sigma(v)


def dsilu(v):
    s = sigma(v)
    return s * (1.0 + v * (1.0 - s))


def init_params(rng: np.random.Generator):
    """Glorot-style initial weights (the GPU draws its own; this is for tests)."""
    p = {
        "W1": rng.normal(0, np.sqrt(2.0 / (NIN + HIDDEN)), (HIDDEN, NIN)),
        "b1": np.zeros(HIDDEN),
        "W2": rng.normal(0, np.sqrt(2.0 / (2 * HIDDEN)), (HIDDEN, HIDDEN)),
        "b2": np.zeros(HIDDEN),
        "W3": rng.normal(0, np.sqrt(2.0 / (HIDDEN + NOUT)), (NOUT, HIDDEN)),
        "b3": np.zeros(NOUT),
    }
    return p


def forward(p, z, u, bf16: bool = True):
    """z (B,32), u (B,2) -> y (B,2) and the cache for backward."""
    R = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    zr = R(z)
    W1z = R(p["W1"][:, :LATENT])
    W1u = p["W1"][:, LATENT:]
    h1 = zr @ W1z.T + u @ W1u.T + p["b1"]
    a1 = R(silu(h1))
    W2 = R(p["W2"])
    h2 = a1 @ W2.T + p["b2"]
    a2 = silu(h2)
    y = a2 @ p["W3"].T + p["b3"]
    x = np.concatenate([zr, np.asarray(u, dtype=np.float64)], axis=1)
    return y, dict(x=x, h1=h1, a1=a1, h2=h2, a2=a2, W1z=W1z, W2=W2)


def loss_and_grads(p, z, u, t, bf16: bool = True):
    """Mean-squared loss and gradients {W1, b1, W2, b2, W3, b3, z (per sample)}."""
    R = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    B = z.shape[0]
    y, c = forward(p, z, u, bf16)
    d = y - t
    loss = float(np.sum(d * d) / B)
    dy = 2.0 * d / B
    g = {"W3": dy.T @ c["a2"], "b3": dy.sum(0)}
    da2 = dy @ p["W3"]
    dh2 = da2 * dsilu(c["h2"])
    dh2r = R(dh2)
    g["W2"] = dh2r.T @ c["a1"]
    g["b2"] = dh2.sum(0)
    da1 = dh2r @ c["W2"]
    dh1 = da1 * dsilu(c["h1"])
    dh1r = R(dh1)
    # latent block through the tensor cores (rounded dh1), position block in FP32
    g["W1"] = np.concatenate([dh1r.T @ c["x"][:, :LATENT], dh1.T @ c["x"][:, LATENT:]], axis=1)
    g["b1"] = dh1.sum(0)
    g["z"] = dh1r @ c["W1z"]
    return loss, g, y


def adam_step(p, m, v, g, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of the arrays in p, in place."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


# ---------------------------------------------------------------- error bounds
# Element-wise error bounds for an evaluation of the network above that rounds the
# same operands to BF16 (round to nearest even) but does everything else in FP32:
# products and accumulations in FP32 (tensor-core accumulation taken as one FP32
# rounding per term, in any direction) and a tanh with relative error at most
# `tanh_rel` (the hardware approximation's documented maximum is about 2^-11; the
# default rounds that up to 2^-10.9).  This is
# a running error analysis (Wilkinson's), carried element by element: for each
# intermediate quantity the FP64 value y and a bound E on |x - y|, x the other
# evaluation's value, propagated through sums and products in absolute values.
# At a BF16 rounding point R: if [y - E, y + E] stays inside the rounding interval
# of y, R(x) = R(y) and the bound drops to zero; otherwise
# |R(x) - R(y)| <= E + 2^-7 (|y| + E) (each rounding moves a value by at most
# 2^-8 of itself).  The bounds are worst-case: they hold for any tanh errors
# within tanh_rel and any rounding directions of the FP32 steps.

U32 = 2.0 ** -24   # FP32 unit roundoff
U32A = 2.0 ** -23  # FP32 accumulation step, any rounding direction


def _bf16_midpoint_distance(y):
    """Distance of each y to the nearest BF16 rounding boundary (the midpoint of two
    neighbouring BF16 values)."""
    a = np.abs(np.asarray(y, dtype=np.float64))
    ra = bf16_round(a)
    rb = ra.astype(np.float32).view(np.uint32).astype(np.int64)
    up = (rb + 0x10000).astype(np.uint32).view(np.float32).astype(np.float64)
    dn = np.where(rb >= 0x10000, rb - 0x10000, 0).astype(np.uint32).view(np.float32).astype(np.float64)
    mid_up = 0.5 * (ra + up)
    mid_dn = np.where(ra > 0, 0.5 * (ra + dn), -mid_up)  # around 0 the interval is symmetric
    return np.minimum(np.abs(mid_up - a), np.abs(a - mid_dn))


def _round(y, E):
    """BF16 rounding point: (R(y), bound on |R(x) - R(y)|)."""
    flip = E >= _bf16_midpoint_distance(y)
    return bf16_round(y), np.where(flip, E + 2.0 ** -7 * (np.abs(y) + E), 0.0)


def _matmul(a, Ea, b, Eb, k):
    """a @ b over k terms with FP32 accumulation: (value, bound)."""
    A, B = np.abs(a), np.abs(b)
    return a @ b, A @ Eb + Ea @ B + Ea @ Eb + (k + 2) * U32A * ((A + Ea) @ (B + Eb))


def _mul(a, Ea, b, Eb):
    """Element-wise product, one FP32 rounding."""
    A, B = np.abs(a), np.abs(b)
    return a * b, A * Eb + Ea * B + Ea * Eb + U32 * (A + Ea) * (B + Eb)


def _colsum(a, Ea, n):
    """Sum over samples (axis 0) in FP32 with n accumulation steps."""
    return a.sum(0), Ea.sum(0) + n * U32A * (np.abs(a) + Ea).sum(0)


def _silu(v, Ev, tanh_rel):
    """silu computed as h + h tanh~(h), h = v/2: the slope of silu over [v - Ev, v + Ev]
    (|silu''| <= 1/2, |silu'| < 1.1), the tanh error |h tanh(h)| tanh_rel, one FMA."""
    slope = np.minimum(np.abs(dsilu(v)) + 0.5 * Ev, 1.1)
    h = 0.5 * (np.abs(v) + Ev)
    own = h * np.abs(np.tanh(h)) * tanh_rel + U32 * (np.abs(silu(v)) + slope * Ev + h * tanh_rel)
    return silu(v), slope * Ev + own


def _dsilu(v, Ev, tanh_rel):
    """silu' computed as s (1 + v (1 - s)), s = 1/2 + tanh~(v/2)/2: the slope of silu' is
    at most 1/2 in size; the derivative in s is at most 1 + |v|; s carries tanh_rel/2
    and one rounding; four FP32 roundings."""
    va = np.abs(v) + Ev
    es = 0.5 * tanh_rel * np.abs(np.tanh(0.5 * va)) + U32
    return dsilu(v), 0.5 * Ev + (1.0 + va) * es + 4 * U32 * (1.0 + va) * (1.0 + es)


def error_bounds(p, z, u, t, tanh_rel: float = 2.0 ** -10.9):
    """Values and element-wise error bounds of loss_and_grads(p, z, u, t, bf16=True)
    for an evaluation in the arithmetic described above.  Returns (loss, grads, y,
    bounds) with bounds = {"loss", "y", "W1", "b1", "W2", "b2", "W3", "b3", "z"}."""
    B = z.shape[0]
    A = np.abs
    zr, W1z, W2 = bf16_round(z), bf16_round(p["W1"][:, :LATENT]), bf16_round(p["W2"])
    W1u, W3 = p["W1"][:, LATENT:], p["W3"]
    u = np.asarray(u, dtype=np.float64)
    O = np.zeros_like
    # forward
    h1, E = _matmul(zr, O(zr), W1z.T, O(W1z.T), LATENT)
    E = E + (2 + 3) * U32A * (A(u) @ A(W1u).T + A(p["b1"]) + A(h1))  # + W1u u + b1 in FP32
    h1 = h1 + u @ W1u.T + p["b1"]
    Eh1 = E
    a1, Ea1 = _round(*_silu(h1, Eh1, tanh_rel))
    h2, Eh2 = _matmul(a1, Ea1, W2.T, O(W2.T), HIDDEN)
    Eh2 = Eh2 + U32 * (A(h2) + A(p["b2"]) + Eh2)
    h2 = h2 + p["b2"]
    a2, Ea2 = _silu(h2, Eh2, tanh_rel)
    y, Ey = _matmul(a2, Ea2, W3.T, O(W3.T), HIDDEN + 1)
    Ey = Ey + U32 * (A(y) + A(p["b3"]) + Ey)
    y = y + p["b3"]
    d = y - t
    Ed = Ey + U32 * (A(d) + Ey)
    loss = float(np.sum(d * d) / B)
    Eloss = float((np.sum(2 * A(d) * Ed + Ed ** 2) + (2 * B + 4) * U32A * np.sum((A(d) + Ed) ** 2)) / B)
    # backward
    # dy = 2 (y - t) * fl(1/B): the rounded 1/B and the product, two roundings
    dy, Edy = 2.0 * d / B, 2.0 * Ed / B + 3 * U32 * A(2.0 * (A(d) + Ed) / B)
    da2, Eda2 = _matmul(dy, Edy, W3, O(W3), NOUT)
    dh2, Edh2 = _mul(da2, Eda2, *_dsilu(h2, Eh2, tanh_rel))
    dh2r, Edh2r = _round(dh2, Edh2)
    da1, Eda1 = _matmul(dh2r, Edh2r, W2, O(W2), HIDDEN)
    dh1, Edh1 = _mul(da1, Eda1, *_dsilu(h1, Eh1, tanh_rel))
    dh1r, Edh1r = _round(dh1, Edh1)
    n = B + 8  # FP32 sums over samples: per-CTA folds, then the reduction over CTAs
    g, eb = {}, {}
    g["W3"], eb["W3"] = _matmul(dy.T, Edy.T, a2, Ea2, n)
    g["b3"], eb["b3"] = _colsum(dy, Edy, n)
    g["W2"], eb["W2"] = _matmul(dh2r.T, Edh2r.T, a1, Ea1, n)
    g["b2"], eb["b2"] = _colsum(dh2, Edh2, n)
    gz, Ez = _matmul(dh1r.T, Edh1r.T, zr, O(zr), n)
    gu, Eu = _matmul(dh1.T, Edh1.T, u, O(u), n)
    g["W1"], eb["W1"] = np.concatenate([gz, gu], 1), np.concatenate([Ez, Eu], 1)
    g["b1"], eb["b1"] = _colsum(dh1, Edh1, n)
    g["z"], eb["z"] = _matmul(dh1r, Edh1r, W1z, O(W1z), HIDDEN)
    eb["y"] = Ey
    eb["loss"] = Eloss
    return loss, g, y, eb
