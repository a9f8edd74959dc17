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


def oracle_reference(f, rays, idx, nthreads=0):
    """The oracle's quantities for the grid rays idx: theta, FP64 beta, the term scale
    |alpha_0| + sum m/r and the Jacobian of alpha (each costs N_* per ray)."""
    th = oracle.ray_theta(rays, idx)
    return dict(idx=idx, th=th, b64=oracle.beta_rays(rays, idx, f, nthreads),
                scale=oracle.alpha_scale(th, f, nthreads), J=oracle.alpha_jacobian(th, f, nthreads))


def compare_to_oracle(f, rays, src, b4, idx=None, nthreads=0, rays_per_thread=8, presampled=False, ref=None):
    """Per-ray comparison of GPU float-pair beta (rows idx of the grid, or all rays)
    with the FP64 oracle.  Returns a dict of error statistics.  `ref` (from
    oracle_reference for the same idx) saves recomputing the oracle's side.

    `rel_max` is the literal measure |alpha_gpu - alpha_64| / |alpha_64| over the rays
    with |alpha_64| >= 1e-3 median |alpha_64|; `rel_max_conditioned` the same over
    those of them whose |alpha_64| is at least 1e-2 of the terms' magnitude
    |alpha_0| + sum m/r (`cancelled_frac` are left out: there the sum cancels its
    terms more than 100-fold, and a float32 sum's error, a fraction of the terms'
    magnitude, is no longer small against alpha).  `bound_ratio` is the deflection error
    over its allowance
        1e-5 * (|alpha_0| + sum_k m_k/r_k)  +  ||d alpha/d theta||_F * sqrt(2) * eps_pos,
    the first term a 1e-5 relative error of the summed terms, the second the effect
    of rounding the ray/star offsets from the tile centre to float32 (eps_pos)."""
    if idx is None:
        idx = np.arange(rays.n, dtype=np.int64) if ref is None else ref["idx"]
        bsel = b4
    elif presampled:
        bsel = b4  # already the rows of idx
    else:
        bsel = b4[idx]
    if ref is None:
        ref = oracle_reference(f, rays, idx, nthreads)
    b64, th, scale, J = ref["b64"], ref["th"], ref["scale"], ref["J"]
    a64 = th - b64
    ag = th - beta_pair_to_f64(bsel)
    amag = np.linalg.norm(a64, axis=1)
    err = np.linalg.norm(ag - a64, axis=1)
    fin = np.isfinite(err)
    ok = fin & (amag >= 1e-3 * np.median(amag[fin]))
    rel = err[ok] / amag[ok]
    # rays whose deflection keeps at least 1e-2 of its terms' magnitude (the sum is
    # conditioned to within 100x): the relative bar applies to them without a
    # cancellation factor
    wc = ok & (amag >= 1e-2 * scale)
    rel_wc = err[wc] / amag[wc]
    cond = err[fin] / scale[fin]
    jn = np.sqrt(J[:, 0] ** 2 + 2 * J[:, 1] ** 2 + J[:, 2] ** 2)
    allow = 1e-5 * scale + jn * math.sqrt(2.0) * position_rounding(rays, rays_per_thread)
    ratio = err[fin] / allow[fin]
    pix_o = oracle.pixels(b64, src)
    pix_g = oracle.pair_pixels(bsel, src)
    w = min((src.x1 - src.x0) / src.nx, (src.y1 - src.y0) / src.ny)
    dbeta = np.abs(beta_pair_to_f64(bsel) - b64)
    dbf = dbeta[np.isfinite(dbeta).all(1)] / w
    dbn = np.linalg.norm(dbf, axis=1)
    return dict(n=int(idx.shape[0]), misbinned=int(np.sum(pix_o != pix_g)), misbinned_frac=float(np.mean(pix_o != pix_g)),
                rel_max=float(rel.max()), rel_p50=float(np.median(rel)), rel_p9999=float(np.quantile(rel, 0.9999)),
                rel_max_conditioned=float(rel_wc.max()) if rel_wc.size else 0.0, rel_over_1e5=int(np.sum(rel > 1e-5)),
                cancelled_frac=float(1.0 - wc.sum() / max(ok.sum(), 1)),
                cond_max=float(cond.max()), cond_p50=float(np.median(cond)),
                bound_ratio=float(ratio.max()),
                dbeta_mean_px=float(dbf.mean()), dbeta_p9999_px=float(np.quantile(dbn, 0.9999)),
                dbeta_max_px=float(dbn.max()),
                # the ray with the largest relative error: its |alpha| and Jacobian norm
                rel_worst=dict(alpha=float(amag[ok][np.argmax(rel)]), jac=float(jn[ok][np.argmax(rel)]),
                               err=float(err[ok][np.argmax(rel)])))
