"""Pins of oracle/mlp.error_bounds, the element-wise error bounds the GPU network
tests use: an independent FP32 evaluation of the network on the CPU (BF16 operands
at the same rounding points, float32 products and sums, a tanh perturbed within the
documented 2^-11 of the hardware approximation, at random and with either sign
throughout) must stay within the bounds at every element, and plausible mistakes
planted in that evaluation (a sign, a swapped index, a transposed block, a lost
factor) must break them somewhere."""
import numpy as np
import pytest

from oracle import mlp

f32 = np.float32


def _bf(a):
    return mlp.bf16_round(a).astype(f32)


def _fp32_network(p, z, u, t, rng, tanh_mode):
    """The network's loss, gradients and outputs evaluated in float32 with BF16
    operands z, W1[:, :32], a1, W2, dh2, dh1 and a tanh off by up to 2^-11."""
    def tanh(x):
        th = np.tanh(x.astype(np.float64))
        if tanh_mode == "random":
            fac = 1 + rng.uniform(-1, 1, x.shape) * 2.0 ** -11
        else:
            fac = np.full(x.shape, 1 + (2.0 ** -11 if tanh_mode == "high" else -2.0 ** -11))
        return (th * fac).astype(f32)

    def silu(v):
        h = (f32(0.5) * v).astype(f32)
        return (h + h * tanh(h)).astype(f32)

    def dsilu(v):
        s = (f32(0.5) * tanh((f32(0.5) * v).astype(f32)) + f32(0.5)).astype(f32)
        return (s * (f32(1) + v * (f32(1) - s))).astype(f32)

    B = z.shape[0]
    P = {k: np.asarray(v, dtype=f32) for k, v in p.items()}
    zr, W1z, W1u, W2 = _bf(z), _bf(P["W1"][:, :32]), P["W1"][:, 32:], _bf(P["W2"])
    u, t = u.astype(f32), t.astype(f32)
    h1 = (zr @ W1z.T + u @ W1u.T + P["b1"]).astype(f32)
    a1 = _bf(silu(h1))
    h2 = (a1 @ W2.T + P["b2"]).astype(f32)
    a2 = silu(h2)
    y = (a2 @ P["W3"].T + P["b3"]).astype(f32)
    d = (y - t).astype(f32)
    loss = float(np.sum(d * d, dtype=f32) / f32(B))
    dy = (f32(2) * d / f32(B)).astype(f32)
    g = {"W3": dy.T @ a2, "b3": dy.sum(0)}
    dh2 = (dy @ P["W3"] * dsilu(h2)).astype(f32)
    dh2r = _bf(dh2)
    g["W2"], g["b2"] = dh2r.T @ a1, dh2.sum(0)
    dh1 = (dh2r @ W2 * dsilu(h1)).astype(f32)
    dh1r = _bf(dh1)
    g["W1"] = np.concatenate([dh1r.T @ zr, dh1.T @ u], 1)
    g["b1"], g["z"] = dh1.sum(0), dh1r @ W1z
    return loss, {k: v.astype(np.float64) for k, v in g.items()}, y.astype(np.float64)


def _case(seed, B):
    rng = np.random.default_rng(100 + seed)
    p = mlp.init_params(rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0, 0.1, p[k].shape)
    p = {k: v.astype(f32).astype(np.float64) for k, v in p.items()}
    z = rng.normal(0, 0.5, (B, 32)).astype(f32).astype(np.float64)
    u = rng.uniform(-1, 1, (B, 2)).astype(f32).astype(np.float64)
    t = rng.normal(0, 1, (B, 2)).astype(f32).astype(np.float64)
    return rng, p, z, u, t


def _worst_ratio(ref, got):
    """max over elements of |got - value| / bound, per output."""
    loss, g, y, eb = ref
    lg, gg, yg = got
    r = {"y": float(np.max(np.abs(yg - y) / eb["y"])), "loss": abs(lg - loss) / eb["loss"]}
    for k in g:
        r[k] = float(np.max(np.abs(gg[k] - g[k]) / np.maximum(eb[k], 1e-300)))
    return r


def test_values_are_the_reference_network():
    rng, p, z, u, t = _case(0, 256)
    loss, g, y, eb = mlp.error_bounds(p, z, u, t)
    l2, g2, y2 = mlp.loss_and_grads(p, z, u, t, bf16=True)
    assert loss == pytest.approx(l2, rel=1e-14) and np.array_equal(y, y2)
    for k in g2:
        assert np.allclose(g[k], g2[k], rtol=1e-13, atol=0), k
        assert eb[k].shape == g2[k].shape and np.all(eb[k] >= 0)


@pytest.mark.parametrize("B", [128, 1000])
def test_a_float32_evaluation_stays_within_the_bounds(B):
    for seed in range(4):
        for mode in ("random", "high", "low"):
            rng, p, z, u, t = _case(seed, B)
            ref = mlp.error_bounds(p, z, u, t)
            r = _worst_ratio(ref, _fp32_network(p, z, u, t, rng, mode))
            assert max(r.values()) <= 1.0, (seed, mode, r)


MISTAKES = {
    "b3 gradient sign": lambda l, g, y: (l, {**g, "b3": -g["b3"]}, y),
    "b3 gradient outputs swapped": lambda l, g, y: (l, {**g, "b3": g["b3"][::-1].copy()}, y),
    "W1u gradient sign": lambda l, g, y: (l, {**g, "W1": np.concatenate([g["W1"][:, :32], -g["W1"][:, 32:]], 1)}, y),
    "W1u gradient columns swapped": lambda l, g, y: (
        l, {**g, "W1": np.concatenate([g["W1"][:, :32], g["W1"][:, 32:][:, ::-1]], 1)}, y),
    "latent gradient columns 0 and 1 swapped": lambda l, g, y: (
        l, {**g, "z": g["z"][:, [1, 0] + list(range(2, 32))]}, y),
    "W2 gradient transposed": lambda l, g, y: (l, {**g, "W2": g["W2"].T.copy()}, y),
    "W3 gradient rows swapped": lambda l, g, y: (l, {**g, "W3": g["W3"][::-1].copy()}, y),
    "gradients halved": lambda l, g, y: (l, {k: 0.5 * v for k, v in g.items()}, y),
    "outputs swapped": lambda l, g, y: (l, g, y[:, ::-1].copy()),
    "loss halved": lambda l, g, y: (0.5 * l, g, y),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistakes_break_the_bounds(name):
    for seed, B in ((0, 128), (1, 1000)):
        rng, p, z, u, t = _case(seed, B)
        ref = mlp.error_bounds(p, z, u, t)
        r = _worst_ratio(ref, MISTAKES[name](*_fp32_network(p, z, u, t, rng, "random")))
        assert max(r.values()) > 1.0, (name, seed, r)
