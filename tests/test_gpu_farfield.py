"""The learned-far-field variant on the GPU against the FP64 oracle and against the
plain direct-sum path: cell CSR, FP64 expansion coefficients, the network's forward
and backward kernels, the shooting kernel (series only, fallback, trained network),
and save/load."""
import math
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from gpu_util import (beta_pair_to_f64, compare_to_oracle, make_ctx, oracle_reference,  # noqa: E402
                      position_rounding, shoot_gpu)
from oracle import mlp  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402

# A reduced version of the 10^6-star workload: the same star density (kappa_* = 0.45,
# 0.64 stars per theta_E^2), the same cell width (0.46875 theta_E) and 2048^2 rays.
N_STARS = 20000
RAYS = W.Grid(-7.5, 7.5, -2.5, 2.5, 2048, 2048)
SRC = W.Grid(-2.0, 2.0, -2.0, 2.0, 512, 512)
CELLS_X = 32


@pytest.fixture(scope="module")
def field():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return W.random_field(W.SEED_BASE + 40, N_STARS, 0.45, 0.05, 0.25, 0.0)


def ext_cells(info):
    return oracle.cells(info.grid_x0, info.grid_y0, info.cell_width, info.grid_nx, info.grid_ny)


def host(c, src):
    return c.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx)


def fallback_split(n):
    """The learned kernel's split of a fallback tile's star sum: the largest of 8, 4, 2
    leaving 2048 stars per slice of the padded field, else none."""
    n_pad = (n + 31) // 32 * 32
    return next((r for r in (8, 4, 2) if n_pad // r >= 2048), 1)


def plain_map(f):
    # fallback tiles run the plain tile function with the fallback split
    c, st, b4 = shoot_gpu(f, RAYS, SRC, split=fallback_split(f.n))
    return c, st, b4


def learned_map(ctx, want_beta=False):
    counts = torch.empty(SRC.n, dtype=torch.int32, device="cuda")
    beta = torch.empty(RAYS.n * 4, dtype=torch.float32, device="cuda") if want_beta else None
    st = M.mlens_shoot_learned(ctx, RAYS, SRC, counts, beta=beta, stats=True)
    torch.cuda.synchronize()
    b = beta.cpu().numpy().reshape(-1, 4) if want_beta else None
    return host(counts, SRC), st, b


def test_cell_csr_and_coefficients_match_the_oracle(field):
    ctx = make_ctx(field)
    rep = M.mlens_fit_far_field(ctx, RAYS, M.fit_params(cells_x=CELLS_X, use_network=0, order=8))
    ex = M.mlens_far_field_export(ctx)
    info = ex["info"]
    assert (info.cells_x, info.cells_y) == (32, 11) and abs(info.cell_width - 0.46875) < 1e-15
    c = ext_cells(info)
    # CSR offsets = counting sort of the oracle's cell index of every star
    idx = oracle.cell_index(field.xy, c)
    cnt = np.bincount(idx[idx >= 0], minlength=info.grid_nx * info.grid_ny)
    assert np.array_equal(ex["cell_start"], np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32))
    # FP64 coefficients of a sample of ray cells
    rng = np.random.default_rng(1)
    rcs = rng.choice(info.cells_x * info.cells_y, 12, replace=False)
    ext = (rcs // info.cells_x + 1) * info.grid_nx + rcs % info.cells_x + 1
    ref = oracle.local_coeffs(ext, info.target_order, info.cell_width / math.sqrt(2), field, c)
    got = ex["coef"][rcs, :, 0] + 1j * ex["coef"][rcs, :, 1]
    # b_0 in FP64 throughout; for p >= 1 the terms are FP32 (relative ~p 6e-8) summed in FP64
    assert np.max(np.abs(got[:, 0] - ref[:, 0]) / np.abs(ref[:, 0])) < 1e-11
    rel = np.abs(got[:, 1:] - ref[:, 1:]) / np.abs(ref[:, 1:]).max(axis=1, keepdims=True)
    assert rel.max() < 1e-5, rel.max()
    assert rep["cells"] == 352 and rep["train_steps"] == 0
    ctx.close()


def _flat(p):
    return np.concatenate([p["W1"][:, :32].ravel(), p["W1"][:, 32:].ravel(), p["b1"], p["W2"].ravel(), p["b2"],
                           p["W3"].ravel(), p["b3"]]).astype(np.float32)


def _unflat_grad(g):
    o = 0
    W1z = g[o:o + 2048].reshape(64, 32); o += 2048
    W1u = g[o:o + 128].reshape(64, 2); o += 128
    b1 = g[o:o + 64]; o += 64
    W2 = g[o:o + 4096].reshape(64, 64); o += 4096
    b2 = g[o:o + 64]; o += 64
    W3 = g[o:o + 128].reshape(2, 64); o += 128
    b3 = g[o:o + 2]
    return {"W1": np.concatenate([W1z, W1u], 1), "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


@pytest.mark.parametrize("B", [128, 1000])
def test_network_forward_and_backward_match_the_oracle(B):
    """The GPU training kernel (BF16 tensor cores, FP32 accumulation, hardware tanh)
    on explicit inputs against the FP64 reference with the same BF16 rounding points,
    element by element: every output, every parameter gradient and every latent
    gradient within the bound of oracle/mlp.error_bounds (a worst-case running error
    analysis of BF16 operands at those points, FP32 sums and a tanh within 2^-10.9,
    exact where a BF16 rounding cannot flip).  The relative (Frobenius) errors per
    block, and those against the network evaluated exactly in FP64 without BF16
    rounding, are printed."""
    rng = np.random.default_rng(10 + B)
    p = mlp.init_params(rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0, 0.1, p[k].shape)
    flat = _flat(p)
    p32 = _unflat_grad(flat.astype(np.float64))  # the float32 values the GPU sees
    z = rng.normal(0, 0.5, (B, 32)).astype(np.float32)
    u = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    t = rng.normal(0, 1, (B, 2)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    y = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    g = torch.empty(flat.shape[0], dtype=torch.float32, device="cuda")
    dz = torch.empty((B, 32), dtype=torch.float32, device="cuda")
    loss = M.mlens_ff_eval(dev(flat), dev(z), dev(u), dev(t), y=y, grads=g, dz=dz)
    z64, u64, t64 = z.astype(np.float64), u.astype(np.float64), t.astype(np.float64)
    lref, gref, yref, bound = mlp.error_bounds(p32, z64, u64, t64)
    got = _unflat_grad(g.cpu().numpy().astype(np.float64))
    got["z"] = dz.cpu().numpy().astype(np.float64)
    yg = y.cpu().numpy().astype(np.float64)
    assert abs(loss - lref) <= bound["loss"], (loss, lref, bound["loss"])
    over = np.abs(yg - yref) / bound["y"]
    assert over.max() <= 1.0, ("y", float(over.max()), np.unravel_index(over.argmax(), over.shape))
    for k in gref:
        over = np.abs(got[k] - gref[k]) / np.maximum(bound[k], 1e-300)
        assert over.max() <= 1.0, (k, float(over.max()), np.unravel_index(over.argmax(), over.shape))
    # reported: block errors against this reference and against the exact FP64 network
    _, gex, yex = mlp.loss_and_grads(p32, z64, u64, t64, bf16=False)
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))  # noqa: E731
    rep = {k: (rel(got[k], gref[k]), rel(got[k], gex[k])) for k in gref}
    rep["y"] = (rel(yg, yref), rel(yg, yex))
    print("network block errors (vs BF16-point reference, vs exact FP64):",
          {k: (f"{a:.1e}", f"{b:.1e}") for k, (a, b) in rep.items()})
    for k, (a, _) in rep.items():
        assert a < 2e-3, (k, a)


def test_series_only_far_field_matches_the_plain_path(field):
    """Order-16 exact series (truncation ~1e-9 theta_E): the learned path without a
    network must meet the same oracle bar as the plain path, and nearly equal its map."""
    ctx = make_ctx(field)
    rep = M.mlens_fit_far_field(ctx, RAYS, M.fit_params(cells_x=CELLS_X, use_network=0, order=16, tolerance=1e-6))
    assert rep["cells_fallback"] == 0, rep
    cl, st, b4 = learned_map(ctx, want_beta=True)
    c_re, st_re = oracle.rebin_pair(b4, SRC)
    assert np.array_equal(cl, c_re) and st == st_re
    cp, stp, _ = plain_map(field)
    e = compare_to_oracle(field, RAYS, SRC, b4, W.ray_sample(RAYS, 20000, 3))
    assert e["misbinned_frac"] <= 1e-4 and e["bound_ratio"] <= 1.0, e
    l1 = np.abs(cl.astype(np.int64) - cp).sum() / cp.sum()
    assert l1 < 1e-4, l1
    ctx.close()


def test_fallback_cells_reproduce_the_plain_map_bit_for_bit(field):
    ctx = make_ctx(field)
    rep = M.mlens_fit_far_field(ctx, RAYS, M.fit_params(cells_x=CELLS_X, use_network=0, order=4, tolerance=0.0))
    assert rep["cells_fallback"] == rep["cells"]
    cl, st, b4 = learned_map(ctx, want_beta=True)
    cp, stp, bp = plain_map(field)
    assert np.array_equal(cl, cp) and st == stp
    assert np.array_equal(b4.view(np.uint32), bp.view(np.uint32))
    ctx.close()


def test_trained_network_reduces_the_far_field_error(field):
    """Order-6 series + network (trained on the GPU) against order-6 series alone, on
    held-out samples; then the map of the learned path against the plain map."""
    ctx = make_ctx(field)
    prm = M.fit_params(cells_x=CELLS_X, use_network=1, order=6, train_samples=1 << 20, epochs=128, tolerance=1e-6,
                       batch=65536)
    rep = M.mlens_fit_far_field(ctx, RAYS, prm)
    print("fit", rep)
    assert rep["train_steps"] == 128 * 16
    assert rep["val_mean_err_net"] < 0.2 * rep["val_mean_err_series"], rep
    assert rep["val_max_err_net"] < rep["val_max_err_series"], rep
    cl, st, _ = learned_map(ctx)
    cp, _, _ = plain_map(field)
    l1 = np.abs(cl.astype(np.int64) - cp).sum() / cp.sum()
    print("map L1 vs plain", l1, "fallback cells", rep["cells_fallback"], "/", rep["cells"])
    assert l1 <= 1e-3
    # save / load into a fresh context of the same stars: same map without retraining
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ff.bin")
        M.mlens_save_far_field(ctx, path)
        ctx2 = make_ctx(field)
        M.mlens_load_far_field(ctx2, path)
        c2, st2, _ = learned_map(ctx2)
        assert np.array_equal(c2, cl) and st2 == st
        ctx2.close()
    ctx.close()


def test_learned_shoot_rejects_wrong_state(field):
    ctx = make_ctx(field)
    counts = torch.empty(SRC.n, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MlensError) as ei:
        M.mlens_shoot_learned(ctx, RAYS, SRC, counts)
    assert ei.value.code == M.MLENS_ERR_STATE
    with pytest.raises(M.MlensError) as ei:
        M.mlens_fit_far_field(ctx, W.Grid(-7.5, 7.5, -2.5, 2.5, 2000, 2048), M.fit_params(cells_x=32))
    assert ei.value.code == M.MLENS_ERR_ARG
    ctx.close()


def test_row_restricted_calls_add_up_to_the_full_map(field):
    ctx = make_ctx(field)
    M.mlens_fit_far_field(ctx, RAYS, M.fit_params(cells_x=CELLS_X, use_network=0, order=8, tolerance=2e-6))
    full, st, _ = learned_map(ctx)
    acc = torch.zeros(SRC.n, dtype=torch.int32, device="cuda")
    bounds = [0, 192, 1024, 1056, 2048]
    for a, b in zip(bounds[:-1], bounds[1:]):
        M.mlens_shoot_learned(ctx, RAYS, SRC, acc, rows=(a, b), flags=M.MLENS_ACCUMULATE)
    torch.cuda.synchronize()
    assert np.array_equal(host(acc, SRC), full)
    with pytest.raises(M.MlensError):
        M.mlens_shoot_learned(ctx, RAYS, SRC, acc, rows=(0, 100))
    ctx.close()


LEARNED_STRIPS = ((0, 768), (10752, 11520), (16128, 16896), (32000, 32768))


def near_scale(f, th, radius):
    """sum_k m_k / |theta - theta_k| over the stars within `radius` of each theta."""
    from scipy.spatial import cKDTree
    tree = cKDTree(f.xy)
    out = np.zeros(th.shape[0])
    for i, ks in enumerate(tree.query_ball_point(th, radius)):
        if ks:
            d = np.linalg.norm(f.xy[ks] - th[i], axis=1)
            out[i] = np.sum(f.m[ks] / d)
    return out


def test_learned_full_size_workload_against_the_oracle():
    """The bench's learned workload itself (1e6 stars, 32768^2 rays, 4096^2 map, the
    default fit) on four strips of 768 ray rows: the first and last rows of the grid
    (the cells next to the extra ring) and two interior strips.  Per strip: the map
    against the plain kernel's map of the same rays (relative L1 <= 1e-3), and 2e4
    sampled rays against the FP64 oracle: misbinned fraction <= 1e-4 and every ray's
    deflection error within
        2 tol + 1e-5 (|alpha_0| + sum_near m/r) + ||d alpha/d theta|| sqrt(2) eps_pos,
    tol the fit's validation bound on the far field (2 tol: the bound is validated on
    held-out samples, not at every position), the second term the plain path's 1e-5
    error bar applied to the exactly summed near stars (those within 2 sqrt(2) cell
    widths: a superset of the 3x3 block), the third its position rounding."""
    wl = W.config("learned")
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    tol = 5e-6
    ctx = make_ctx(f)
    rep = M.mlens_fit_far_field(ctx, rays, M.fit_params(cells_x=256, tolerance=tol))
    assert rep["cells"] == 256 * 86
    info = M.mlens_far_field_export(ctx)["info"]
    beta = torch.empty((rays.n, 4), dtype=torch.float32, device="cuda")  # rows outside the strips stay unset
    rng = np.random.default_rng(5)
    l1_num = l1_den = 0
    worst = {}
    for j0, j1 in LEARNED_STRIPS:
        cl = torch.empty(src.n, dtype=torch.int32, device="cuda")
        st = M.mlens_shoot_learned(ctx, rays, src, cl, beta=beta, rows=(j0, j1), stats=True)
        cp = torch.empty(src.n, dtype=torch.int32, device="cuda")
        stp = M.mlens_shoot_rows(ctx, rays, (j0, j1), src, cp, stats=True)
        torch.cuda.synchronize()
        assert st["rays_total"] == stp["rays_total"] == rays.nx * (j1 - j0)
        a = cl.cpu().numpy().view(np.uint32).astype(np.int64)
        b = cp.cpu().numpy().view(np.uint32).astype(np.int64)
        l1 = np.abs(a - b).sum() / b.sum()
        l1_num += np.abs(a - b).sum()
        l1_den += b.sum()
        idx = np.sort(rng.choice(rays.nx * (j1 - j0), 20000, replace=False)) + j0 * rays.nx
        b4 = beta.index_select(0, torch.from_numpy(idx).cuda()).cpu().numpy()
        ref = oracle_reference(f, rays, idx)
        e = compare_to_oracle(f, rays, src, b4, idx, presampled=True, ref=ref)
        th = ref["th"]
        dal = np.linalg.norm((th - beta_pair_to_f64(b4)) - (th - ref["b64"]), axis=1)
        ac = np.abs(np.array([[f.kappa_c + f.gamma1, f.gamma2], [f.gamma2, f.kappa_c - f.gamma1]]))
        a0 = np.linalg.norm(th @ ac.T, axis=1)
        J = ref["J"]
        jn = np.sqrt(J[:, 0] ** 2 + 2 * J[:, 1] ** 2 + J[:, 2] ** 2)
        allow = 2 * tol + 1e-5 * (a0 + near_scale(f, th, 2 * np.sqrt(2) * info.cell_width)) + \
            jn * np.sqrt(2.0) * position_rounding(rays)
        ratio = float(np.max(dal / allow))
        print(f"learned strip [{j0},{j1}): L1 {l1:.2e}, misbinned {e['misbinned_frac']:.1e}, "
              f"|d alpha| mean {dal.mean():.2e} max {dal.max():.2e} theta_E, "
              f"|d beta| mean {e['dbeta_mean_px']:.2e} max {e['dbeta_max_px']:.2e} px, bound ratio {ratio:.3f}")
        assert l1 <= 1e-3, (j0, l1)
        assert e["misbinned_frac"] <= 1e-4, (j0, e)
        assert ratio <= 1.0, (j0, ratio)
        worst[j0] = ratio
    assert l1_num / l1_den <= 1e-3
    ctx.close()


def test_fit_is_bit_reproducible(field):
    """Gradients are summed in a fixed order (per-CTA rows, per-sample latent
    gradients): two fits of the same field give the same parameters, latents, flags
    and maps bit for bit."""
    outs = []
    for _ in range(2):
        ctx = make_ctx(field)
        rep = M.mlens_fit_far_field(ctx, RAYS, M.fit_params(cells_x=CELLS_X, use_network=1, order=6,
                                                            train_samples=1 << 18, epochs=8, tolerance=1e-6))
        ex = M.mlens_far_field_export(ctx)
        cl, st, _ = learned_map(ctx)
        outs.append((rep, ex, cl, st))
        ctx.close()
    (r0, e0, c0, s0), (r1, e1, c1, s1) = outs
    for k in ("params", "latents", "flags", "val_max_net"):
        assert np.array_equal(np.asarray(e0[k]).view(np.uint32), np.asarray(e1[k]).view(np.uint32)), k
    assert r0["final_loss"] == r1["final_loss"] and r0["cells_fallback"] == r1["cells_fallback"]
    assert np.array_equal(c0, c1) and s0 == s1


def test_tensor_core_wait_that_runs_out_is_reported_and_recovered(field):
    """The bounded tensor-core waits' failure path, without a fault: with the wait
    probe on, each launch's first completion wait polls an mbarrier nothing arrives
    on and gives up; the kernel flags it, drains its MMAs (bounded), frees its tensor
    memory and returns.  The learned shoot, a fit (training and validation) and
    mlens_ff_eval must each report MLENS_ERR_CUDA; afterwards the same context
    shoots the same map bit for bit, and a fit succeeds again."""
    ctx = make_ctx(field)
    prm = M.fit_params(cells_x=CELLS_X, use_network=1, order=6, train_samples=1 << 16, epochs=1, tolerance=1.0)
    M.mlens_fit_far_field(ctx, RAYS, prm)
    ref = learned_map(ctx)
    rng = np.random.default_rng(5)
    p = mlp.init_params(rng)
    flat = torch.from_numpy(_flat(p)).cuda()
    z = torch.from_numpy(rng.normal(0, 0.5, (256, 32)).astype(np.float32)).cuda()
    u = torch.from_numpy(rng.uniform(-1, 1, (256, 2)).astype(np.float32)).cuda()
    t = torch.zeros((256, 2), dtype=torch.float32, device="cuda")
    g = torch.empty(flat.shape[0], dtype=torch.float32, device="cuda")
    M.mlens_debug_wait_probe(True)
    try:
        with pytest.raises(M.MlensError) as ei:
            learned_map(ctx)
        assert ei.value.code == M.MLENS_ERR_CUDA
        with pytest.raises(M.MlensError) as ei:
            M.mlens_ff_eval(flat, z, u, t, grads=g)
        assert ei.value.code == M.MLENS_ERR_CUDA
        ctx2 = make_ctx(field)
        with pytest.raises(M.MlensError) as ei:
            M.mlens_fit_far_field(ctx2, RAYS, prm)
        assert ei.value.code == M.MLENS_ERR_CUDA
    finally:
        M.mlens_debug_wait_probe(False)
    again = learned_map(ctx)
    assert np.array_equal(again[0], ref[0]) and again[1] == ref[1]
    M.mlens_fit_far_field(ctx2, RAYS, prm)
    learned_map(ctx2)
    ctx2.close()
    ctx.close()
