"""The split star sum: `split` CTAs share one ray tile, each sums a slice of the
stars.  Up to 8 they form a cluster and the first folds the others' partial sums
(read through distributed shared memory) into its own; above 8 each CTA stores its
partials in global memory and a second kernel folds them in slice order.  Every
split must meet the parity bar against the FP64 oracle, re-bin bit-exactly, and
move no more rays across pixel edges relative to the unsplit map than the error bar
allows; the automatic choice splits only grids with too few tiles for the GPU."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from gpu_util import compare_to_oracle, make_ctx, shoot_gpu  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _shoot(ctx, f, rays, src, split, rpt):
    M.mlens_set_tuning(ctx, rpt)
    M.mlens_set_star_split(ctx, split)
    assert M.mlens_star_split_for(ctx, rays) == split
    return shoot_gpu(f, rays, src, ctx=ctx)


def _moved(b4a, b4b, src):
    """Rays whose pixel differs between two float-pair beta arrays."""
    return int(np.sum(oracle.pair_pixels(b4a, src) != oracle.pair_pixels(b4b, src)))


@pytest.mark.parametrize("rpt", [8, 4])
def test_every_split_meets_the_bar(rpt):
    wl = W.config("paper", rays_scale=1 / 16, src_scale=1 / 4)  # 512^2 rays, 1e4 stars, 256^2 map
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f)
    c1, st1, b1 = _shoot(ctx, f, rays, src, 1, rpt)
    for split in (1, 2, 3, 4, 8, 12, 40):
        c, st, b4 = (c1, st1, b1) if split == 1 else _shoot(ctx, f, rays, src, split, rpt)
        c_re, st_re = oracle.rebin_pair(b4, src)
        assert np.array_equal(c, c_re) and st == st_re, split
        e = compare_to_oracle(f, rays, src, b4, rays_per_thread=rpt)
        assert e["misbinned_frac"] <= 1e-4 and e["bound_ratio"] <= 1.0, (split, e)
        assert _moved(b4, b1, src) <= max(2, 1e-4 * rays.n), split
        # the same split again: deterministic
        c2, st2, b2 = _shoot(ctx, f, rays, src, split, rpt)
        assert np.array_equal(b2.view(np.uint32), b4.view(np.uint32)) and np.array_equal(c2, c), split
    ctx.close()


def test_split_with_fewer_stars_than_slices():
    """40 stars padded to 64: with 8 slices of 32 stars six slices are empty, with 12
    (through global memory) ten, with 100 ninety-eight."""
    f = W.random_field(W.SEED_BASE + 60, 40, kappa_star=0.3, kappa_c=0.1, gamma1=0.2, gamma2=0.05)
    rays = W.Grid(-3.0, 3.0, -2.0, 2.0, 300, 200)
    src = W.Grid(-2.0, 2.0, -2.0, 2.0, 64, 64)
    ctx = make_ctx(f)
    c1, st1, b1 = _shoot(ctx, f, rays, src, 1, 8)
    for split in (8, 12, 100):
        c8, st8, b8 = _shoot(ctx, f, rays, src, split, 8)
        e = compare_to_oracle(f, rays, src, b8)
        assert e["misbinned_frac"] <= 1e-4 and e["bound_ratio"] <= 1.0, (split, e)
        assert st8 == st1 or abs(st8["rays_binned"] - st1["rays_binned"]) <= 2, split
    ctx.close()


@pytest.mark.parametrize("split", [20, 4096])
def test_global_split_passes_equal_one_pass(split):
    """The global split takes tile rows in passes whose partials fit a 256 MB
    workspace: one pass for the 512^2-ray grid at 20 slices, one tile row per pass at
    4096 slices (1 GB per tile row; most slices of the 1e4 stars are empty).  Bands of
    rows shot alone (mlens_shoot_rows) go through passes of their own and must equal
    those rows of the whole map's beta bit for bit; the whole map meets the bar."""
    wl = W.config("paper", rays_scale=1 / 16, src_scale=1 / 4)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f)
    M.mlens_set_star_split(ctx, split)
    c_all, st_all, b_all = shoot_gpu(f, rays, src, ctx=ctx)
    c_re, st_re = oracle.rebin_pair(b_all, src)
    assert np.array_equal(c_all, c_re) and st_all == st_re
    idx = W.ray_sample(rays, 4000, seed=29)
    e = compare_to_oracle(f, rays, src, b_all[idx], idx, presampled=True)
    assert e["misbinned"] == 0 and e["bound_ratio"] <= 1.0, e
    beta = torch.empty(rays.n * 4, dtype=torch.float32, device="cuda")
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    for r0, r1 in ((0, 64), (96, 224), (448, rays.ny)):
        M.mlens_shoot_rows(ctx, rays, (r0, r1), src, counts, beta=beta)
        torch.cuda.synchronize()
        b = beta.cpu().numpy().reshape(rays.ny, rays.nx, 4)[r0:r1]
        ref = b_all.reshape(rays.ny, rays.nx, 4)[r0:r1]
        assert np.array_equal(b.view(np.uint32), ref.view(np.uint32)), (split, r0, r1)
    ctx.close()


def test_large_star_field_split_against_the_oracle():
    """1e7 stars on a 128^2-ray grid (8 tiles): the automatic choice splits each tile
    over 16 CTAs per SM through global memory; 2000 sampled rays against the FP64
    oracle (2e10 interactions on the host)."""
    wl = W.config("large_n", rays_scale=0.25)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert M.mlens_star_split_for(ctx, rays) == _expected_auto(8, (f.n + 31) // 32 * 32, nsm) > 8
    c, st, b4 = shoot_gpu(f, rays, src, ctx=ctx)
    c_re, st_re = oracle.rebin_pair(b4, src)
    assert np.array_equal(c, c_re) and st == st_re
    idx = W.ray_sample(rays, 2000, seed=17)
    e = compare_to_oracle(f, rays, src, b4[idx], idx, presampled=True)
    print("large_n, automatic split", e)
    assert e["misbinned_frac"] <= 1e-3 and e["bound_ratio"] <= 1.0, e
    _, _, b1 = _shoot(ctx, f, rays, src, 1, 8)
    assert _moved(b4, b1, src) <= max(2, 1e-4 * rays.n)
    ctx.close()


def _expected_auto(tiles, nstars_padded, nsm):
    """The library's rule: the global split with at least 16 CTAs per SM (and more
    than 8 slices) if it gains 5 %, else, with too few stars for it, the best
    cluster of 2, 4 or 8."""
    def cost(r):
        c = tiles * r
        return 1.0 / r if c <= nsm else math.ceil(c / (2.0 * nsm)) * 2.0 / r
    rg = max(9, math.ceil(16 * nsm / tiles))
    if rg <= 4096 and nstars_padded // rg >= 2048:
        return rg if cost(rg) < cost(1) / 1.05 else 1
    best, bc = 1, cost(1)
    for r in (2, 4, 8):
        if nstars_padded // r < 2048:
            break
        if cost(r) < bc / 1.05:
            best, bc = r, cost(r)
    return best


def test_automatic_split_policy():
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    wl = W.config("paper")
    f, rays = wl.fields[0], wl.rays[0]
    ctx = make_ctx(f)
    assert M.mlens_star_split_for(ctx, rays) == 1  # 32768 tiles: nothing to gain
    n_pad = (f.n + 31) // 32 * 32
    for scale in (1 / 8, 1 / 16, 1 / 32, 1 / 64):
        g = W.Grid(rays.x0, rays.x1, rays.y0, rays.y1, int(rays.nx * scale), int(rays.ny * scale))
        tiles = math.ceil(g.nx / 64) * math.ceil(g.ny / 32)
        assert M.mlens_star_split_for(ctx, g) == _expected_auto(tiles, n_pad, nsm), scale
    # only the re-centred kernel with its default stage splits (with either reciprocal source)
    small = W.Grid(rays.x0, rays.x1, rays.y0, rays.y1, 256, 256)
    assert M.mlens_star_split_for(ctx, small) > 1
    M.mlens_set_tuning(ctx, 8, 512)
    assert M.mlens_star_split_for(ctx, small) == 1
    for fma in (0, 1):
        M.mlens_set_tuning(ctx, 8, 256, fma)
        assert M.mlens_star_split_for(ctx, small) > 1
    M.mlens_set_tuning(ctx, 8)
    M.mlens_set_precision(ctx, M.MLENS_PREC_FP32_NAIVE)
    assert M.mlens_star_split_for(ctx, small) == 1
    M.mlens_set_precision(ctx, M.MLENS_PREC_FP32)
    for explicit in (2, 3, 9, 4096):
        M.mlens_set_star_split(ctx, explicit)
        assert M.mlens_star_split_for(ctx, rays) == explicit  # explicit settings win
    for bad in (4097, -1):
        with pytest.raises(M.MlensError) as ei:
            M.mlens_set_star_split(ctx, bad)
        assert ei.value.code == M.MLENS_ERR_ARG
    tiny = make_ctx(W.config("tiny").fields[0])
    assert M.mlens_star_split_for(tiny, W.Grid(-1.0, 1.0, -1.0, 1.0, 64, 32)) == 1  # 100 stars: too few to slice
    tiny.close()
    ctx.close()


def test_hundred_million_stars():
    """Section 4's regime of very many microlenses: 1e8 stars (1.6 GB of float4 on the
    device) over a 256^2-ray grid; the automatic split, the bit-exact re-binning, and
    200 sampled rays against the FP64 oracle (2e10 interactions per pass on the host)."""
    f = W.random_field(W.SEED_BASE + 61, 100_000_000, 0.45, 0.05, 0.25, 0.0)
    rays = W.Grid(-12.0, 12.0, -4.0, 4.0, 256, 256)
    src = W.Grid(-2.0, 2.0, -2.0, 2.0, 256, 256)
    ctx = make_ctx(f)
    split = M.mlens_star_split_for(ctx, rays)
    assert split > 1
    c, st, b4 = shoot_gpu(f, rays, src, ctx=ctx)
    ctx.close()
    assert st["rays_total"] == rays.n
    c_re, st_re = oracle.rebin_pair(b4, src)
    assert np.array_equal(c, c_re) and st == st_re
    idx = W.ray_sample(rays, 200, seed=23)
    e = compare_to_oracle(f, rays, src, b4[idx], idx, presampled=True)
    print("1e8 stars, split", split, e)
    assert e["misbinned"] == 0 and e["bound_ratio"] <= 1.0, e
