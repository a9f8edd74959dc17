"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and compare
with the FP64 oracle.  Imported only by tests marked gpu."""
import math

import numpy as np
import torch

import oracle
from paper_1703_09707_gb300 import mlens as M


def make_ctx(f, prec=M.MLENS_PREC_FP32, split=None):
    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, prec)
    if split is not None:
        M.mlens_set_star_split(ctx, split)
    return ctx


def shoot_gpu(f, rays, src, prec=M.MLENS_PREC_FP32, want_beta=True, ctx=None, flags=0, counts=None, split=None):
    """Returns (counts[ny,nx] uint32, stats, beta) with beta as (n,4) float32 pairs
    {x_hi, y_hi, x_lo, y_lo} for the FP32 variants or (n,2) float64 for FP64.
    `split` (own context only): the star split, None = the library's default."""
    own = ctx is None
    if own:
        ctx = make_ctx(f, prec, split=split)
    if counts is None:
        counts = torch.empty(src.ny * src.nx, dtype=torch.int32, device="cuda")
    beta = None
    if want_beta:
        if prec == M.MLENS_PREC_FP64:
            beta = torch.empty(rays.n * 2, dtype=torch.float64, device="cuda")
        else:
            beta = torch.empty(rays.n * 4, dtype=torch.float32, device="cuda")
        st = M.mlens_shoot_beta(ctx, rays, src, counts, beta, flags=flags, stats=True)
    else:
        st = M.mlens_shoot(ctx, rays, src, counts, flags=flags, stats=True)
    torch.cuda.synchronize()
    c = counts.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx).copy()
    b = None
    if beta is not None:
        b = beta.cpu().numpy().reshape(rays.n, -1)
    if own:
        ctx.close()
    return c, st, b


def beta_pair_to_f64(b4):
    return b4[:, :2].astype(np.float64) + b4[:, 2:].astype(np.float64)


def position_rounding(rays, rays_per_thread=8):
    """Bound on the float32 rounding of ray and star positions taken relative to a
    tile centre in the FP32 kernels: 2^-22 of the tile extent (tile = 64 x 4*rpt rays)."""
    ext = max(64 * (rays.x1 - rays.x0) / rays.nx, 4 * rays_per_thread * (rays.y1 - rays.y0) / rays.ny)
    return 2.0 ** -22 * ext


def compare_to_oracle(f, rays, src, b4, idx=None, nthreads=0, rays_per_thread=8, presampled=False):
    """Per-ray comparison of GPU float-pair beta (rows idx of the grid, or all rays)
    with the FP64 oracle.  Returns a dict of error statistics.

    `bound_ratio` is the deflection error over its allowance
        1e-5 * (|alpha_0| + sum_k m_k/r_k)  +  ||d alpha/d theta||_F * sqrt(2) * eps_pos,
    the first term a 1e-5 relative error of the summed terms, the second the effect
    of rounding the ray/star offsets from the tile centre to float32 (eps_pos)."""
    if idx is None:
        idx = np.arange(rays.n, dtype=np.int64)
        bsel = b4
    elif presampled:
        bsel = b4  # already the rows of idx
    else:
        bsel = b4[idx]
    b64 = oracle.beta_rays(rays, idx, f, nthreads)
    th = oracle.ray_theta(rays, idx)
    a64 = th - b64
    ag = th - beta_pair_to_f64(bsel)
    amag = np.linalg.norm(a64, axis=1)
    err = np.linalg.norm(ag - a64, axis=1)
    fin = np.isfinite(err)
    ok = fin & (amag >= 1e-3 * np.median(amag[fin]))
    rel = err[ok] / amag[ok]
    scale = oracle.alpha_scale(th, f, nthreads)
    cond = err[fin] / scale[fin]
    J = oracle.alpha_jacobian(th, f, nthreads)
    jn = np.sqrt(J[:, 0] ** 2 + 2 * J[:, 1] ** 2 + J[:, 2] ** 2)
    allow = 1e-5 * scale + jn * math.sqrt(2.0) * position_rounding(rays, rays_per_thread)
    ratio = err[fin] / allow[fin]
    pix_o = oracle.pixels(b64, src)
    pix_g = oracle.pair_pixels(bsel, src)
    w = min((src.x1 - src.x0) / src.nx, (src.y1 - src.y0) / src.ny)
    dbeta = np.abs(beta_pair_to_f64(bsel) - b64)
    return dict(n=int(idx.shape[0]), misbinned=int(np.sum(pix_o != pix_g)), misbinned_frac=float(np.mean(pix_o != pix_g)),
                rel_max=float(rel.max()), rel_p50=float(np.median(rel)), rel_p9999=float(np.quantile(rel, 0.9999)),
                cond_max=float(cond.max()), cond_p50=float(np.median(cond)),
                bound_ratio=float(ratio.max()),
                dbeta_mean_px=float(dbeta[np.isfinite(dbeta).all(1)].mean() / w))
