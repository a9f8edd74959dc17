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
