"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Criteria (spec bar):
  - bit-exact: the GPU map equals a CPU re-binning of the GPU's own beta with the
    float32 pair rule, and the GPU's ray bookkeeping equals the re-binning's;
  - misbinned fraction (GPU pixel != oracle FP64 pixel) <= 1e-4;
  - per-ray relative deflection error |alpha_gpu - alpha_64| / |alpha_64| <= 1e-5
    over the rays with |alpha_64| >= 1e-3 median |alpha_64| (rel_max);
  - per-ray deflection error within its 1e-5 error bound: |alpha_gpu - alpha_64| <=
    1e-5 (|alpha_0| + sum_k m_k/r_k) + ||d alpha/d theta|| sqrt(2) eps_pos, where
    the first term is a 1e-5 relative error of the summed terms (where alpha itself
    nearly cancels no float32 evaluation can be small relative to |alpha|) and the
    second the unavoidable effect of holding ray and star offsets from the tile
    centre in float32 (eps_pos = 2^-22 tile extent; it matters only within ~1e-3
    of a star);
  - the FP64 variant equals the oracle bit for bit (beta and map).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402

from gpu_util import compare_to_oracle, make_ctx, shoot_gpu  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402

MISBIN_MAX = 1e-4
REL_MAX = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    M.load()
    yield


def assert_rebin_exact(c, st, b4, src):
    c_re, st_re = oracle.rebin_pair(b4, src)
    assert np.array_equal(c, c_re), f"map differs from CPU re-binning in {int((c != c_re).sum())} pixels"
    assert st == st_re, (st, st_re)
    assert st["rays_binned"] + st["rays_out"] + st["rays_nan"] == st["rays_total"]
    assert int(c.sum(dtype=np.uint64)) == st["rays_binned"]


@pytest.mark.parametrize("scale", [1.0, 0.333])
def test_tiny_fp32_full_parity(scale):
    """100 unit masses, 1000^2 (and a ragged 333^2) rays: every ray checked."""
    wl = W.config("tiny", rays_scale=scale)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    c, st, b4 = shoot_gpu(f, rays, src)
    assert_rebin_exact(c, st, b4, src)
    e = compare_to_oracle(f, rays, src, b4)
    print("tiny", scale, e)
    assert e["misbinned_frac"] <= MISBIN_MAX, e
    assert e["bound_ratio"] <= 1.0, e
    # kappa_c = gamma = 0: the star terms cancel near the disk centre, so the relative
    # bar is asserted where alpha keeps 1e-2 of its terms' magnitude (every ray stays
    # within the term-scale bound above)
    assert e["rel_max_conditioned"] <= REL_MAX, e
    c64, st64 = oracle.shoot(rays, src, f)
    assert st["rays_total"] == st64["rays_total"]


def test_paper_shaped_reduced_grid_parity():
    """10^4 power-law stars, kappa_*=0.3, kappa_c=0.2, gamma=(0.3,0), full lens box,
    1024^2 rays (1/8 of the full grid per axis), full 1024^2 map: every ray checked."""
    wl = W.config("paper", rays_scale=0.125)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    c, st, b4 = shoot_gpu(f, rays, src)
    assert_rebin_exact(c, st, b4, src)
    e = compare_to_oracle(f, rays, src, b4)
    print("paper 1024^2", e)
    assert e["misbinned_frac"] <= MISBIN_MAX, e
    assert e["bound_ratio"] <= 1.0, e
    assert e["rel_max"] <= REL_MAX, e


def test_paper_full_size_bench_configuration():
    """The bench workload itself (8192^2 rays, 10^4 stars, 1024^2 map, FP32, the
    default launch shape): the whole map re-binned bit-exactly, 2*10^5 sampled rays
    against the oracle."""
    wl = W.config("paper")
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    c, st, b4 = shoot_gpu(f, rays, src)
    assert st["rays_total"] == 8192 * 8192
    assert_rebin_exact(c, st, b4, src)
    idx = W.ray_sample(rays, 200_000, seed=7)
    e = compare_to_oracle(f, rays, src, b4, idx)
    print("paper full", e)
    assert e["misbinned_frac"] <= MISBIN_MAX, e
    assert e["bound_ratio"] <= 1.0, e
    assert e["rel_max"] <= REL_MAX, e


def test_fp64_equals_oracle_bit_for_bit():
    for name, scale in (("tiny", 0.5), ("paper", 1 / 32)):
        wl = W.config(name, rays_scale=scale)
        f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
        c, st, b = shoot_gpu(f, rays, src, prec=M.MLENS_PREC_FP64)
        idx = np.arange(rays.n, dtype=np.int64)
        b64 = oracle.beta_rays(rays, idx, f)
        assert np.array_equal(b.view(np.uint64), b64.view(np.uint64)), name
        c64, st64 = oracle.shoot(rays, src, f)
        assert np.array_equal(c, c64), name
        assert st == st64, (st, st64)


def test_trace_fp64_equals_oracle():
    wl = W.config("paper")
    f = wl.fields[0]
    rng = np.random.default_rng(3)
    th = rng.uniform(-60, 60, (5000, 2))
    ctx = make_ctx(f)
    b = M.mlens_trace(ctx, th)
    ctx.close()
    assert np.array_equal(b, oracle.beta(th, f))


def test_naive_fp32_rebins_exactly_and_reports_error():
    wl = W.config("paper", rays_scale=0.125)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    c, st, b4 = shoot_gpu(f, rays, src, prec=M.MLENS_PREC_FP32_NAIVE)
    assert np.all(b4[:, 2:] == 0)
    assert_rebin_exact(c, st, b4, src)
    e = compare_to_oracle(f, rays, src, b4)
    print("naive", e)
    # the naive loop is kept to show its error; it must still be a sane deflection
    assert e["cond_max"] < 1e-3


# ----------------------------------------------------------------- edge cases
def test_sheet_exact_integer_counts_gpu():
    """No stars (n=0), kappa_c=1/2, gamma=(1/4,0) on a dyadic lattice: every pixel
    holds exactly 8 rays, in every precision."""
    f = W.Field(xy=np.zeros((0, 2)), m=np.zeros(0), kappa_c=0.5, gamma1=0.25, gamma2=0.0)
    d = 1.0 / 16.0
    rays = W.Grid(-8.0, 8.0, -8.0, 8.0, 256, 256)
    sx0, sy0 = (-8.0 + 40 * d) / 4.0, 0.75 * (-8.0 + 60 * d)
    src = W.Grid(sx0, sx0 + 30 * 4 * d / 4.0, sy0, sy0 + 40 * 2 * 0.75 * d, 30, 40)
    for prec in (M.MLENS_PREC_FP32, M.MLENS_PREC_FP32_NAIVE, M.MLENS_PREC_FP64):
        c, st, _ = shoot_gpu(f, rays, src, prec=prec, want_beta=False)
        assert np.all(c == 8), prec
        assert st["rays_binned"] == 30 * 40 * 8


def test_point_lens_matches_oracle_map():
    f = W.Field(xy=np.zeros((1, 2)), m=np.ones(1), kappa_c=0.0, gamma1=0.0, gamma2=0.0)
    rays = W.Grid(-10.0, 10.0, -10.0, 10.0, 2048, 2048)
    src = W.Grid(-4.0, 4.0, -4.0, 4.0, 64, 64)
    c, st, b4 = shoot_gpu(f, rays, src)
    assert_rebin_exact(c, st, b4, src)
    c64, st64 = oracle.shoot(rays, src, f)
    e = compare_to_oracle(f, rays, src, b4)
    assert e["misbinned_frac"] <= MISBIN_MAX
    # each misbinned ray moves one count between two pixels
    assert int(np.abs(c.astype(np.int64) - c64).sum()) <= 2 * e["misbinned"]


@pytest.mark.parametrize("nx,ny", [(1, 1), (7, 5), (65, 33), (1000, 777), (64, 32)])
def test_ragged_and_tiny_grids(nx, ny):
    wl = W.config("tiny")
    f = wl.fields[0]
    rays = W.Grid(-3.0, 4.0, -2.5, 3.5, nx, ny)
    src = W.Grid(-3.0, 3.0, -3.0, 3.0, 257, 129)  # odd map sizes
    c, st, b4 = shoot_gpu(f, rays, src)
    assert st["rays_total"] == nx * ny
    assert_rebin_exact(c, st, b4, src)
    e = compare_to_oracle(f, rays, src, b4)
    assert e["misbinned"] == 0 or e["misbinned_frac"] <= MISBIN_MAX


def test_ray_exactly_on_a_star_is_nan():
    f = W.Field(xy=np.array([[0.5, 0.5], [3.0, 1.0]]), m=np.array([1.0, 0.5]), kappa_c=0.1, gamma1=0.0,
                gamma2=0.0)
    rays = W.Grid(0.0, 1.0, 0.0, 1.0, 1, 1)  # the one ray sits on the first star
    src = W.Grid(-2.0, 2.0, -2.0, 2.0, 8, 8)
    for prec in (M.MLENS_PREC_FP32, M.MLENS_PREC_FP32_NAIVE, M.MLENS_PREC_FP64):
        c, st, _ = shoot_gpu(f, rays, src, prec=prec, want_beta=False)
        assert st == dict(rays_total=1, rays_binned=0, rays_out=0, rays_nan=1), (prec, st)
        assert c.sum() == 0


def test_ray_on_a_star_leaves_its_neighbours_exact():
    """One ray of a 4 x 4 grid sits exactly on a star; the rays around it, among them
    the one processed in the same packed pair of the FP32 kernel (the next row of the
    same column), must come out as if the star were anywhere else: every other beta
    equals the oracle's within the error bound, and the bookkeeping counts one NaN
    ray."""
    f = W.Field(xy=np.array([[0.375, 0.375], [3.0, 1.0], [-0.6, 0.7]]), m=np.array([1.0, 0.5, 0.3]),
                kappa_c=0.1, gamma1=0.05, gamma2=0.0)
    rays = W.Grid(0.0, 1.0, 0.0, 1.0, 4, 4)  # cell centres 0.125, 0.375, ...: ray (1, 1) is on the first star
    src = W.Grid(-8.0, 8.0, -8.0, 8.0, 64, 64)
    for prec in (M.MLENS_PREC_FP32, M.MLENS_PREC_FP32_NAIVE, M.MLENS_PREC_FP64):
        c, st, b = shoot_gpu(f, rays, src, prec=prec)
        assert st["rays_nan"] == 1 and st["rays_binned"] + st["rays_out"] == 15, (prec, st)
        b64 = oracle.beta_rays(rays, np.arange(16, dtype=np.int64), f)
        on = 1 * 4 + 1
        bg = b if prec == M.MLENS_PREC_FP64 else b[:, :2].astype(np.float64) + b[:, 2:].astype(np.float64)
        assert not np.all(np.isfinite(bg[on]))
        keep = np.arange(16) != on
        assert np.all(np.isfinite(bg[keep])), prec
        assert np.max(np.abs(bg[keep] - b64[keep])) < 1e-4, (prec, np.max(np.abs(bg[keep] - b64[keep])))
        if prec == M.MLENS_PREC_FP32:
            assert_rebin_exact(c, st, b, src)
            e = compare_to_oracle(f, rays, src, b[keep], np.nonzero(keep)[0].astype(np.int64), presampled=True)
            assert e["bound_ratio"] <= 1.0 and e["misbinned"] == 0, e


def test_accumulate_and_determinism():
    wl = W.config("paper", rays_scale=1 / 16)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    M.mlens_shoot(ctx, rays, src, counts)
    a = counts.clone()
    M.mlens_shoot(ctx, rays, src, counts)
    assert torch.equal(a, counts), "integer atomics commute: maps must be identical run to run"
    M.mlens_shoot(ctx, rays, src, counts, flags=M.MLENS_ACCUMULATE)
    assert torch.equal(counts, 2 * a)
    ctx.close()


def test_standalone_bin_matches_fused_map():
    wl = W.config("paper", rays_scale=0.125)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    beta = torch.empty(rays.n * 4, dtype=torch.float32, device="cuda")
    st = M.mlens_shoot_beta(ctx, rays, src, counts, beta, stats=True)
    counts2 = torch.empty_like(counts)
    st2 = M.mlens_bin(beta, rays.n, src, counts2, stats=True)
    assert torch.equal(counts, counts2)
    assert st == st2
    counts3 = torch.empty_like(counts)
    st3 = M.mlens_bin_grid(beta, rays, src, counts3, stats=True)
    assert torch.equal(counts, counts3) and st == st3
    ctx.close()


def edge_records(rng, k, x0, w, nx):
    """k float-pair records {x_hi, y_hi, x_lo, y_lo} on and near the pixel edges of an
    nx-pixel axis over [x0, x0 + w]: exact edges as pairs, hi parts a few ulps off an
    edge, lo parts that straddle it, and uniform positions in and around the map."""
    f32 = np.float32
    i = rng.integers(-2, nx + 2, k)
    edge = x0 + i * (w / nx)
    bh = edge.astype(f32)
    mode = rng.integers(0, 4, k)
    ulp = np.spacing(np.abs(bh)).astype(f32)
    bh = np.where(mode == 1, bh + rng.integers(-3, 4, k).astype(f32) * ulp, bh).astype(f32)
    bl = np.where(mode == 0, (edge - bh.astype(np.float64)).astype(f32), f32(0))
    bl = np.where(mode == 2, (rng.uniform(-0.5, 0.5, k) * ulp).astype(f32), bl).astype(f32)
    bh = np.where(mode == 3, rng.uniform(x0 - 0.1 * w, x0 + 1.1 * w, k).astype(f32), bh).astype(f32)
    perm = rng.permutation(k)
    return np.stack([bh, bh[perm], bl, bl[perm]], 1).astype(f32)


@pytest.mark.parametrize("nx,x0,w", [(1024, -10.0, 20.0), (4096, 3.25, 0.1), (37, -120.5, 300.0), (32768, -4.0, 8.0)])
def test_bin_records_on_pixel_edges(nx, x0, w):
    """Records placed on pixel edges (as float pairs, and hi parts a few ulps off an
    edge, and lo parts that straddle it): the kernels decide most pixels from the hi
    parts and fall back to the pair rule near edges; every pixel must equal the
    float-pair rule's (re-binned on the CPU)."""
    rng = np.random.default_rng(nx)
    src = W.Grid(x0, x0 + w, x0, x0 + w, nx, nx)
    k = 1 << 20
    b4 = edge_records(rng, k, x0, w, nx)
    c_ref, st_ref = oracle.rebin_pair(b4, src)
    beta = torch.from_numpy(b4.reshape(-1)).cuda()
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    st = M.mlens_bin(beta, k, src, counts, stats=True)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx), c_ref) and st == st_ref
    rays = W.Grid(0.0, 1.0, 0.0, 1.0, 1000, k // 1000)
    n = rays.n
    st = M.mlens_bin_grid(beta, rays, src, counts, stats=True)
    c_ref, st_ref = oracle.rebin_pair(b4[:n], src)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx), c_ref) and st == st_ref


@pytest.mark.parametrize("order", ["flat", "grid"])
def test_bin_many_blocks_ragged_and_non_finite(order):
    """About 1200 blocks of 4096 records, more than the GPU holds at once; the record
    count (flat) or row count (grid) leaves the last blocks' second round empty, and
    the grid's width is ragged.  Non-finite records are mixed in.  Counts and stats
    must equal the CPU re-binning."""
    rng = np.random.default_rng(20 if order == "flat" else 21)
    nx, x0, w = 700, -3.0, 6.0
    src = W.Grid(x0, x0 + w, x0, x0 + w, nx, nx)
    if order == "flat":
        k = 1200 * 4096 + 777  # 777 < 2048: the last block's second round is empty
    else:
        rays = W.Grid(0.0, 1.0, 0.0, 1.0, 1000, 4930)  # 1000 % 64 = 40; 4930 % 64 = 2: second rounds of the last block row empty
        k = rays.n
    b4 = edge_records(rng, k, x0, w, nx)
    bad = rng.choice(k, 5000, replace=False)
    b4[bad[:2000], rng.integers(0, 4, 2000)] = np.nan
    b4[bad[2000:], rng.integers(0, 4, 3000)] = np.inf
    c_ref, st_ref = oracle.rebin_pair(b4, src)
    assert st_ref["rays_nan"] == 5000
    beta = torch.from_numpy(b4.reshape(-1)).cuda()
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    if order == "flat":
        st = M.mlens_bin(beta, k, src, counts, stats=True)
    else:
        st = M.mlens_bin_grid(beta, rays, src, counts, stats=True)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx), c_ref) and st == st_ref
    # once more on top of the map
    if order == "flat":
        M.mlens_bin(beta, k, src, counts, flags=M.MLENS_ACCUMULATE)
    else:
        M.mlens_bin_grid(beta, rays, src, counts, flags=M.MLENS_ACCUMULATE)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx), 2 * c_ref)


def test_grid_ordered_bin_on_ragged_grid():
    """1000 x 1000 rays: neither dimension is a multiple of the 64 x 64 binning block
    (nor of its 32-row stages)."""
    wl = W.config("tiny")
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    assert rays.nx % 64 and rays.ny % 32
    ctx = make_ctx(f)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    beta = torch.empty(rays.n * 4, dtype=torch.float32, device="cuda")
    st = M.mlens_shoot_beta(ctx, rays, src, counts, beta, stats=True)
    c_flat, c_grid = torch.empty_like(counts), torch.empty_like(counts)
    st_flat = M.mlens_bin(beta, rays.n, src, c_flat, stats=True)
    st_grid = M.mlens_bin_grid(beta, rays, src, c_grid, stats=True)
    assert torch.equal(counts, c_flat) and torch.equal(counts, c_grid)
    assert st == st_flat == st_grid
    # accumulate on top of an existing map
    M.mlens_bin_grid(beta, rays, src, c_grid, flags=M.MLENS_ACCUMULATE)
    assert torch.equal(c_grid, 2 * counts)
    ctx.close()


@pytest.mark.parametrize("fma", [0, 1])
def test_launch_shapes_both_meet_the_bar(fma):
    """rays_per_thread 4 and 8 use different tiles (different centres), and fma = 1
    takes some reciprocals from Newton-Raphson on the FMA pipe, so beta may differ in
    its last bits; every shape must meet the bar and they must nearly agree."""
    wl = W.config("paper", rays_scale=1 / 8)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    maps = []
    for rpt in (4, 8):
        ctx = make_ctx(f)
        M.mlens_set_tuning(ctx, rpt, 0, fma)
        c, st, b4 = shoot_gpu(f, rays, src, ctx=ctx)
        ctx.close()
        assert_rebin_exact(c, st, b4, src)
        e = compare_to_oracle(f, rays, src, b4, rays_per_thread=rpt)
        assert e["misbinned_frac"] <= MISBIN_MAX and e["bound_ratio"] <= 1.0, (rpt, e)
        maps.append(c.astype(np.int64))
    assert np.abs(maps[0] - maps[1]).sum() <= 2 * MISBIN_MAX * rays.n
