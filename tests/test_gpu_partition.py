"""mlens_shoot_rows, one process's part of a map shot by several (Section 2.2's MPI
tasks): bands of ray rows on tile boundaries give exactly the rows of the whole-grid
shot (beta bit for bit) and their maps add up to the whole map bit for bit, in every
precision, with the star sum split over clusters or through global memory, and on a
ragged grid.  The sum over
processes itself (an all-reduce of the maps) is tested with gloo ranks on the CPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from gpu_util import make_ctx  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402
from paper_1703_09707_gb300 import partition as P  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _host(c, src):
    return c.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx).copy()


CASES = [
    ("paper", 1 / 8, M.MLENS_PREC_FP32, None, 3),
    ("paper", 1 / 8, M.MLENS_PREC_FP32_NAIVE, None, 4),
    ("paper", 1 / 16, M.MLENS_PREC_FP64, None, 3),
    ("paper", 1 / 8, M.MLENS_PREC_FP32, 4, 5),      # star sum split over 4-CTA clusters
    ("paper", 1 / 8, M.MLENS_PREC_FP32, 24, 3),     # ... over 24 CTAs through global memory
    ("tiny", 0.333, M.MLENS_PREC_FP32, None, 4),     # 333 x 333: the last band is ragged
]


@pytest.mark.parametrize("name,scale,prec,split,world", CASES)
def test_bands_add_up_to_the_whole_map(name, scale, prec, split, world):
    wl = W.config(name, rays_scale=scale)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f, prec, split=split)
    rec = 2 if prec == M.MLENS_PREC_FP64 else 4
    dt = torch.float64 if prec == M.MLENS_PREC_FP64 else torch.float32
    full = torch.empty(src.n, dtype=torch.int32, device="cuda")
    beta_full = torch.empty(rays.n * rec, dtype=dt, device="cuda")
    st_full = M.mlens_shoot_beta(ctx, rays, src, full, beta_full, stats=True)
    acc = torch.zeros(src.n, dtype=torch.int32, device="cuda")
    beta = torch.full((rays.n * rec,), float("nan"), dtype=dt, device="cuda")
    tot = dict(rays_total=0, rays_binned=0, rays_out=0, rays_nan=0)
    parts = []
    for r0, r1 in P.row_bands(rays.ny, world):
        if r1 == r0:
            continue
        part = torch.empty(src.n, dtype=torch.int32, device="cuda")
        st = M.mlens_shoot_rows(ctx, rays, (r0, r1), src, part, beta=beta, stats=True)
        assert st["rays_total"] == rays.nx * (r1 - r0)
        for k in tot:
            tot[k] += st[k]
        parts.append(part)
        acc += part  # int32 addition: the all-reduce's arithmetic
    torch.cuda.synchronize()
    assert np.array_equal(_host(acc, src), _host(full, src))
    assert tot == st_full
    bits = torch.int64 if prec == M.MLENS_PREC_FP64 else torch.int32
    assert torch.equal(beta.view(bits), beta_full.view(bits)), "band beta differs from the whole-grid beta"
    # accumulating calls into one map give the same
    acc2 = torch.zeros(src.n, dtype=torch.int32, device="cuda")
    for r0, r1 in P.row_bands(rays.ny, world):
        if r1 > r0:
            M.mlens_shoot_rows(ctx, rays, (r0, r1), src, acc2, flags=M.MLENS_ACCUMULATE)
    torch.cuda.synchronize()
    assert torch.equal(acc2, full)
    ctx.close()


def test_shoot_partitioned_on_one_process_is_the_whole_map():
    wl = W.config("paper", rays_scale=1 / 8)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f)
    full = torch.empty(src.n, dtype=torch.int32, device="cuda")
    st_full = M.mlens_shoot(ctx, rays, src, full, stats=True)
    got = torch.empty(src.n, dtype=torch.int32, device="cuda")
    st = P.shoot_partitioned(ctx, rays, src, got, stats=True)
    torch.cuda.synchronize()
    assert torch.equal(got, full) and st == st_full
    ctx.close()


def test_rows_are_checked():
    wl = W.config("tiny", rays_scale=0.333)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = make_ctx(f)
    c = torch.empty(src.n, dtype=torch.int32, device="cuda")
    for rows in ((16, 64), (0, 48), (64, 32), (0, 334), (-32, 32)):
        with pytest.raises(M.MlensError) as ei:
            M.mlens_shoot_rows(ctx, rays, rows, src, c)
        assert ei.value.code == M.MLENS_ERR_ARG, rows
    M.mlens_shoot_rows(ctx, rays, (320, 333), src, c)  # the ragged end is allowed
    ctx.close()


def test_learned_bands_add_up_to_the_whole_learned_map():
    """The learned far field's map split into bands of ray rows (one per rank of a
    partitioned run) sums to the one-process learned map bit for bit, fallback
    cells included."""
    f = W.random_field(W.SEED_BASE + 40, 20000, 0.45, 0.05, 0.25, 0.0)
    rays = W.Grid(-7.5, 7.5, -2.5, 2.5, 2048, 2048)
    src = W.Grid(-2.0, 2.0, -2.0, 2.0, 512, 512)
    ctx = make_ctx(f)
    # order 6 with a strict tolerance: some cells fall back to the plain sum
    rep = M.mlens_fit_far_field(ctx, rays, M.fit_params(cells_x=32, use_network=1, order=6, train_samples=1 << 18,
                                                        epochs=8, tolerance=2e-7))
    assert rep["cells_fallback"] > 0, rep
    full = torch.empty(src.n, dtype=torch.int32, device="cuda")
    st_full = M.mlens_shoot_learned(ctx, rays, src, full, stats=True)
    acc = torch.zeros(src.n, dtype=torch.int32, device="cuda")
    tot = dict(rays_total=0, rays_binned=0, rays_out=0, rays_nan=0)
    for r0, r1 in P.row_bands(rays.ny, 3):
        part = torch.empty(src.n, dtype=torch.int32, device="cuda")
        st = M.mlens_shoot_learned(ctx, rays, src, part, rows=(r0, r1), stats=True)
        for k in tot:
            tot[k] += st[k]
        acc += part
    torch.cuda.synchronize()
    assert torch.equal(acc, full) and tot == st_full
    got = torch.empty(src.n, dtype=torch.int32, device="cuda")
    st = P.shoot_learned_partitioned(ctx, rays, src, got, stats=True)  # one process: the whole map
    torch.cuda.synchronize()
    assert torch.equal(got, full) and st == st_full
    ctx.close()
