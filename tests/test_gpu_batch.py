"""Batched shooting (many independent fields in one persistent, graph-captured
launch) against single-field shooting and against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from gpu_util import compare_to_oracle, make_ctx, shoot_gpu  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402


@pytest.fixture(scope="module")
def small_batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = W.batched_config(nfields=12, nrays=384, nsrc=96, seed=W.SEED_BASE + 50)
    # the persistent kernel never splits a tile's star sum: compare with unsplit shots
    ctxs = [make_ctx(f, split=1) for f in wl.fields]
    counts = [torch.empty(s.n, dtype=torch.int32, device="cuda") for s in wl.srcs]
    yield wl, ctxs, counts
    for c in ctxs:
        c.close()


def host(c, s):
    return c.cpu().numpy().view(np.uint32).reshape(s.ny, s.nx)


@pytest.mark.parametrize("rpt,stage,fma", [(8, 256, 0), (4, 128, 0), (8, 512, 1), (4, 256, 1)])
def test_batch_equals_single_field_shots(small_batch, rpt, stage, fma):
    wl, ctxs, counts = small_batch
    b = M.mlens_batch_create(ctxs, wl.rays, wl.srcs, counts)
    M.mlens_batch_set_tuning(b, rpt, stage, fma)
    st = M.mlens_batch_run(b, stats=True)
    torch.cuda.synchronize()
    for f, ctx in enumerate(ctxs):
        M.mlens_set_tuning(ctx, rpt, stage, fma)
        ref = torch.empty_like(counts[f])
        st1 = M.mlens_shoot(ctx, wl.rays[f], wl.srcs[f], ref, stats=True)
        assert torch.equal(ref, counts[f]), f"field {f}"
        assert st1 == st[f], (f, st1, st[f])
        M.mlens_set_tuning(ctx, 8, 0)
    # replaying the graph gives the same maps again
    snap = [c.clone() for c in counts]
    M.mlens_batch_run(b)
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(snap, counts))
    b.close()


def test_batch_fields_match_the_oracle(small_batch):
    wl, ctxs, counts = small_batch
    b = M.mlens_batch_create(ctxs, wl.rays, wl.srcs, counts)
    st = M.mlens_batch_run(b, stats=True)
    torch.cuda.synchronize()
    # the heaviest and the lightest field, every ray, against the FP64 oracle
    ns = [f.n for f in wl.fields]
    for f in (int(np.argmax(ns)), int(np.argmin(ns))):
        fld, rays, src = wl.fields[f], wl.rays[f], wl.srcs[f]
        c64, st64 = oracle.shoot(rays, src, fld)
        c = host(counts[f], src)
        _, _, b4 = shoot_gpu(fld, rays, src)  # single-field beta (same shape as the batch)
        e = compare_to_oracle(fld, rays, src, b4)
        assert e["misbinned_frac"] <= 1e-4 and e["bound_ratio"] <= 1.0, (f, e)
        assert int(np.abs(c.astype(np.int64) - c64).sum()) <= 2 * e["misbinned"]
        assert st[f]["rays_total"] == st64["rays_total"]
    b.close()


def test_batch_accumulate_and_one_shot(small_batch):
    wl, ctxs, counts = small_batch
    M.mlens_shoot_batch(ctxs, wl.rays, wl.srcs, counts)
    first = [c.clone() for c in counts]
    M.mlens_shoot_batch(ctxs, wl.rays, wl.srcs, counts, flags=M.MLENS_ACCUMULATE)
    torch.cuda.synchronize()
    assert all(torch.equal(2 * a, c) for a, c in zip(first, counts))


def test_autotuner_picks_a_valid_shape_and_caches_it(small_batch, tmp_path, monkeypatch):
    wl, ctxs, counts = small_batch
    b = M.mlens_batch_create(ctxs, wl.rays, wl.srcs, counts)
    rpt, stage, fma, ms = M.mlens_batch_tune(b)
    assert rpt in (4, 8) and stage in (128, 256, 512) and fma in (0, 1)
    assert ms > 0 or ms == -1.0
    rpt2, stage2, fma2, ms2 = M.mlens_batch_tune(b)  # same signature: served from the cache
    assert (rpt2, stage2, fma2) == (rpt, stage, fma) and ms2 == -1.0
    st = M.mlens_batch_run(b, stats=True)
    for f, ctx in enumerate(ctxs):
        M.mlens_set_tuning(ctx, rpt, stage, fma)
        ref = torch.empty_like(counts[f])
        assert M.mlens_shoot(ctx, wl.rays[f], wl.srcs[f], ref, stats=True) == st[f]
        assert torch.equal(ref, counts[f])
        M.mlens_set_tuning(ctx, 8, 0)
    b.close()


def test_batch_rejects_bad_arguments(small_batch):
    wl, ctxs, counts = small_batch
    bad = list(wl.rays)
    bad[3] = W.Grid(1.0, -1.0, 0.0, 1.0, 8, 8)
    with pytest.raises(M.MlensError) as ei:
        M.mlens_batch_create(ctxs, bad, wl.srcs, counts)
    assert ei.value.code == M.MLENS_ERR_ARG and "field 3" in str(ei.value)
