"""mlens_shoot_noalloc is for callers that cannot allocate device memory: plugins whose
host application owns all device allocations, and real-time loops that must stay out of
the CUDA allocator.  It works out of a fixed array inside the library instead of a
context.  These tests check that it gives exactly the map of the regular entry point
(same kernel, same float32 stars), twice in a row (the array keeps the previous call's
contents, which must not leak into the next call), and that it refuses star counts
beyond its fixed capacity.

This file is collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402

pytestmark = pytest.mark.gpu


def _stars_dev(f):
    rec = np.zeros((f.n, 4), dtype=np.float32)
    rec[:, 0] = f.xy[:, 0]
    rec[:, 1] = f.xy[:, 1]
    rec[:, 2] = f.m
    return torch.from_numpy(rec).cuda()


def test_noalloc_matches_mlens_shoot_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = W.config("paper", rays_scale=1 / 8)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32)
    M.mlens_set_star_split(ctx, 1)  # the no-alloc entry never splits the star sum
    ref = torch.empty(src.n, dtype=torch.int32, device="cuda")
    st_ref = M.mlens_shoot(ctx, rays, src, ref, stats=True)
    ctx.close()

    stars = _stars_dev(f)
    # a different, smaller field in between leaves other contents in the shared array
    other = W.config("tiny").fields[0]
    other_dev = _stars_dev(other)
    for call in range(2):
        counts = torch.full((src.n,), 12345, dtype=torch.int32, device="cuda")  # must be overwritten
        st = M.mlens_shoot_noalloc(stars, f.n, f.kappa_c, f.gamma1, f.gamma2, rays, src, counts, stats=True)
        torch.cuda.synchronize()
        assert torch.equal(counts, ref), f"call {call}: map differs from mlens_shoot"
        assert st == st_ref, (call, st, st_ref)
        tmp = torch.empty(src.n, dtype=torch.int32, device="cuda")
        M.mlens_shoot_noalloc(other_dev, other.n, 0.0, 0.0, 0.0, rays, src, tmp)
    torch.cuda.synchronize()


def test_noalloc_rejects_too_many_stars():
    """The library itself refuses a star count above its fixed capacity (the binding
    passes a correctly typed buffer of that many records, so the refusal is the C
    side's)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    big = 65536 + 1
    g = W.Grid(-1.0, 1.0, -1.0, 1.0, 8, 8)
    counts = torch.empty(64, dtype=torch.int32, device="cuda")
    stars = torch.zeros((big, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(M.MlensError) as ei:
        M.mlens_shoot_noalloc(stars, big, 0.0, 0.0, 0.0, g, g, counts)
    assert ei.value.code == M.MLENS_ERR_ARG
    assert "65536" in str(ei.value)
