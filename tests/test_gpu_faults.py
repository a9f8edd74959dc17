"""Failure handling without faulting the GPU: a device-memory budget makes the
library's own allocations fail on the host side (as if the device were full).
Every entry point must report MLENS_ERR_NOMEM, leave existing contexts usable and
leak nothing; lifting the budget restores normal service."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from gpu_util import make_ctx  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402

RAYS = W.Grid(-7.5, 7.5, -2.5, 2.5, 2048, 2048)
SRC = W.Grid(-2.0, 2.0, -2.0, 2.0, 256, 256)


def _shoot(ctx):
    c = torch.empty(SRC.n, dtype=torch.int32, device="cuda")
    st = M.mlens_shoot(ctx, RAYS, SRC, c, stats=True)
    return c.clone(), st


def test_memory_budget_fails_cleanly_and_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    M.mlens_set_device_memory_limit(0)
    base = M.mlens_device_memory_in_use()
    f = W.config("tiny").fields[0]
    ctx = make_ctx(f)
    assert M.mlens_device_memory_in_use() > base
    ref, st_ref = _shoot(ctx)
    try:
        M.mlens_set_device_memory_limit(M.mlens_device_memory_in_use() + 4096)
        big = W.config("paper").fields[0]
        with pytest.raises(M.MlensError) as ei:
            make_ctx(big)  # 160 KB of stars
        assert ei.value.code == M.MLENS_ERR_NOMEM
        with pytest.raises(M.MlensError) as ei:
            M.mlens_fit_far_field(ctx, RAYS, M.fit_params(cells_x=32, use_network=0))
        assert ei.value.code == M.MLENS_ERR_NOMEM
        with pytest.raises(M.MlensError) as ei:
            M.mlens_trace(ctx, np.zeros((100000, 2)))
        assert ei.value.code == M.MLENS_ERR_NOMEM
        counts = [torch.empty(SRC.n, dtype=torch.int32, device="cuda") for _ in range(300)]
        with pytest.raises(M.MlensError) as ei:
            M.mlens_batch_create([ctx] * 300, [RAYS] * 300, [SRC] * 300, counts)
        assert ei.value.code == M.MLENS_ERR_NOMEM
        with pytest.raises(M.MlensError):
            M.mlens_shoot_learned(ctx, RAYS, SRC, counts[0])  # the failed fit left no far field
        # the context still shoots, identically
        c, st = _shoot(ctx)
        assert torch.equal(c, ref) and st == st_ref
    finally:
        M.mlens_set_device_memory_limit(0)
    # service restored
    rep = M.mlens_fit_far_field(ctx, RAYS, M.fit_params(cells_x=32, use_network=0, order=12))
    assert rep["cells"] == 32 * 11
    ctx.close()
    assert M.mlens_device_memory_in_use() == base, "device memory leaked"
