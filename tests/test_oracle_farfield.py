"""Pins of the oracle pieces used by the learned-far-field variant (CPU only):
the near/far split of the star term, the far field's local (Taylor) expansion,
and the FP64 reference of the far-field network (forward, backward, Adam)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import mlp


def small_field(seed=1, n=3000, radius=12.0):
    rng = np.random.default_rng(seed)
    xy = W.to_f32_exact(W.draw_disk(rng, n, radius))
    m = W.to_f32_exact(W.draw_masses(rng, n))
    return W.Field(xy=xy, m=m, kappa_c=0.1, gamma1=0.2, gamma2=-0.05)


CELLS = oracle.cells(-8.0, -8.0, 0.5, 32, 32)


def test_near_plus_far_is_the_star_term():
    f = small_field()
    rng = np.random.default_rng(2)
    th = rng.uniform(-7.9, 7.9, (300, 2))
    rc = oracle.cell_index(th, CELLS)
    near, far = oracle.split_alpha(th, rc, f, CELLS)
    a0 = oracle.alpha(th, W.Field(xy=np.zeros((0, 2)), m=np.zeros(0), kappa_c=f.kappa_c, gamma1=f.gamma1,
                                  gamma2=f.gamma2))
    star = oracle.alpha(th, f) - a0
    assert np.allclose(near + far, star, rtol=1e-12, atol=1e-12)
    # near stars are exactly those in the 3 x 3 block: moving one star from just
    # inside the block to just outside moves its term from near to far
    assert np.all(np.isfinite(far))


def test_cell_index_edges():
    pts = np.array([[-8.0, -8.0], [-7.5, -8.0], [7.999, 7.999], [8.0, 0.0], [-8.0001, 0.0], [0.25, 0.75]])
    assert list(oracle.cell_index(pts, CELLS)) == [0, 1, 32 * 32 - 1, -1, -1, 17 * 32 + 16]


def test_local_expansion_converges_to_the_far_direct_sum():
    """The far field is holomorphic on the 3x3 block, so its Taylor series about the
    cell centre converges on the cell like (half-diagonal / 1.5 w)^p; at order 40 it
    equals the FP64 far direct sum to ~1e-11, and the error falls with the order."""
    f = small_field(n=4000)
    rng = np.random.default_rng(3)
    ids = np.array([16 * 32 + 16, 10 * 32 + 20, 25 * 32 + 7, 3 * 32 + 3])
    s = CELLS.w / math.sqrt(2)
    a = oracle.local_coeffs(ids, 40, s, f, CELLS)
    u = rng.uniform(-0.5, 0.5, (ids.shape[0], 50, 2)) * CELLS.w
    zc = np.stack([CELLS.x0 + (ids % 32 + 0.5) * CELLS.w, CELLS.y0 + (ids // 32 + 0.5) * CELLS.w], 1)
    th = (zc[:, None, :] + u).reshape(-1, 2)
    _, far = oracle.split_alpha(th, np.repeat(ids, 50), f, CELLS)
    zz = (u[..., 0] + 1j * u[..., 1]) / s
    errs = []
    for P in (4, 8, 16, 40):
        F = np.zeros_like(zz)
        for q in range(P, -1, -1):
            F = F * zz + a[:, q][:, None]
        e = np.hypot(F.real.reshape(-1) - far[:, 0], -F.imag.reshape(-1) - far[:, 1])
        errs.append(e.max())
    scale = np.abs(far).max()
    assert errs[-1] < 1e-10 * max(1.0, scale)
    assert errs[0] > errs[1] > errs[2] > errs[3]


# --------------------------------------------------------------- network
def rand_batch(rng, B=7):
    z = rng.normal(0, 0.5, (B, mlp.LATENT))
    u = rng.uniform(-1, 1, (B, 2))
    t = rng.normal(0, 1, (B, 2))
    return z, u, t


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(0, 3, 5000), [0.0, -0.0, 1.0, 1e-30, 3.0e38, 1 + 2 ** -8, 1 + 3 * 2 ** -9]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_silu_derivative():
    v = np.linspace(-8, 8, 401)
    h = 1e-6
    fd = (mlp.silu(v + h) - mlp.silu(v - h)) / (2 * h)
    assert np.allclose(mlp.dsilu(v), fd, atol=1e-8)
    assert np.allclose(mlp.silu(v), v / (1 + np.exp(-v)), rtol=1e-13, atol=1e-15)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(5)
    p = mlp.init_params(rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0, 0.1, p[k].shape)
    z, u, t = rand_batch(rng)
    loss, g, _ = mlp.loss_and_grads(p, z, u, t, bf16=False)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        idx = [tuple(rng.integers(0, s) for s in p[k].shape) for _ in range(6)]
        for ix in idx:
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][ix] += h
            lp = mlp.loss_and_grads(q, z, u, t, bf16=False)[0]
            q[k][ix] -= 2 * h
            lm = mlp.loss_and_grads(q, z, u, t, bf16=False)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][ix]) < 1e-6 * (1 + abs(fd)), (k, ix, fd, g[k][ix])
    for s in range(z.shape[0]):
        for j in (0, 7, 31):
            zp = z.copy(); zp[s, j] += h
            zm = z.copy(); zm[s, j] -= h
            fd = (mlp.loss_and_grads(p, zp, u, t, bf16=False)[0] - mlp.loss_and_grads(p, zm, u, t, bf16=False)[0]) / (2 * h)
            assert abs(fd - g["z"][s, j]) < 1e-6 * (1 + abs(fd))


def test_network_gradients_match_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    p = mlp.init_params(rng)
    z, u, t = rand_batch(rng, B=33)
    loss, g, y = mlp.loss_and_grads(p, z, u, t, bf16=False)
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    Z = torch.tensor(z, dtype=torch.float64, requires_grad=True)
    x = torch.cat([Z, torch.tensor(u, dtype=torch.float64)], 1)
    a1 = torch.nn.functional.silu(x @ P["W1"].T + P["b1"])
    a2 = torch.nn.functional.silu(a1 @ P["W2"].T + P["b2"])
    yt = a2 @ P["W3"].T + P["b3"]
    lt = ((yt - torch.tensor(t)) ** 2).sum() / z.shape[0]
    lt.backward()
    assert abs(lt.item() - loss) < 1e-12 * max(1, loss)
    assert np.allclose(yt.detach().numpy(), y, rtol=1e-12, atol=1e-14)
    for k in p:
        assert np.allclose(P[k].grad.numpy(), g[k], rtol=1e-10, atol=1e-14), k
    assert np.allclose(Z.grad.numpy(), g["z"], rtol=1e-10, atol=1e-14)


def test_adam_first_step_is_a_signed_lr_step():
    """After one step from zero moments, bias correction makes Adam move each
    parameter by lr * g / (|g| + eps): a step of ~lr against the gradient's sign."""
    p = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -1e-3, 0.0])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    mlp.adam_step(p, m, v, g, 1, lr=0.01)
    assert np.allclose(p["a"], [1.0 - 0.01 * 0.5 / (0.5 + 1e-8), -2.0 + 0.01 * 1e-3 / (1e-3 + 1e-8), 3.0])


def test_rectangular_cell_grid_rule():
    """nx != ny: index iy*nx + ix, near = within one cell in both axes, outside = far."""
    c = oracle.cells(0.0, 0.0, 1.0, 5, 3)
    pts = np.array([[0.5, 0.5], [4.5, 2.5], [4.5, 3.5], [5.0, 0.0], [2.2, 1.7]])
    assert list(oracle.cell_index(pts, c)) == [0, 14, -1, -1, 7]
    f = W.Field(xy=np.array([[2.5, 1.5], [4.5, 1.5], [0.5, 0.5]]), m=np.ones(3), kappa_c=0, gamma1=0, gamma2=0)
    th = np.array([[3.5, 1.5]])
    near, far = oracle.split_alpha(th, oracle.cell_index(th, c), f, c)
    # stars at (2.5,1.5) and (4.5,1.5) are in neighbouring cells, (0.5,0.5) is two cells away
    assert np.allclose(near[0], [1.0 / 1.0 - 1.0 / 1.0, 0.0], atol=1e-15)
    d = np.array([3.0, 1.0])
    assert np.allclose(far[0], d / (d @ d))
