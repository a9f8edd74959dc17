"""Precision study on the 10^5-star workload (kappa_* = 0.4, kappa_c = 0.1,
gamma = (0.2, 0.1); 16384^2 rays over [-60,60] x [-30,30]; 2048^2 map over
[-10,10]^2): FP32 naive, FP32 re-centred + Kahan, FP64 on the GPU and the FP64
oracle, compared on a seeded random sample of 10^6 rays (the oracle costs N_* per
ray; its side is computed once for all variants).

Each FP32 map is also re-binned bit-exactly from its own beta on the CPU.  The
study's table is written as JSON to the file named by MLENS_STUDY_OUT when it is
set."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from gpu_util import compare_to_oracle, make_ctx, oracle_reference  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402

SAMPLE = 1_000_000


def test_precision_study_full_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = W.config("precision")
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    idx = W.ray_sample(rays, SAMPLE, seed=31)
    idx_t = torch.from_numpy(idx).cuda()
    ref = oracle_reference(f, rays, idx)
    table = {}
    ctx = make_ctx(f)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    beta = torch.empty((rays.n, 4), dtype=torch.float32, device="cuda")
    for name, prec in (("fp32_recentred_kahan", M.MLENS_PREC_FP32), ("fp32_naive", M.MLENS_PREC_FP32_NAIVE)):
        M.mlens_set_precision(ctx, prec)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = M.mlens_shoot_beta(ctx, rays, src, counts, beta)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = M.mlens_shoot_beta(ctx, rays, src, counts, beta, stats=True)
        b4 = beta.index_select(0, idx_t).cpu().numpy()
        # bit-exact re-binning of the whole map from the GPU's own beta
        c_gpu = counts.cpu().numpy().view(np.uint32).reshape(src.ny, src.nx)
        c_re, st_re = oracle.rebin_pair(beta.cpu().numpy(), src)
        assert np.array_equal(c_gpu, c_re) and st == st_re, name
        e = compare_to_oracle(f, rays, src, b4, idx, presampled=True, ref=ref)
        e["ms_per_map"] = ms
        e["interactions_per_s"] = rays.n * f.n / (ms / 1e3)
        table[name] = e
    # FP64 on the GPU for the same rays (the FP64 kernel at arbitrary positions)
    th = oracle.ray_theta(rays, idx)
    M.mlens_set_precision(ctx, M.MLENS_PREC_FP64)
    b64_gpu = M.mlens_trace(ctx, th)
    b64 = ref["b64"]
    assert np.array_equal(b64_gpu.view(np.uint64), b64.view(np.uint64)), "FP64 GPU must equal the oracle bit for bit"
    table["fp64_gpu"] = dict(n=SAMPLE, misbinned=0, misbinned_frac=0.0, rel_max=0.0, bit_exact_vs_oracle=True)
    table["fp64_oracle"] = dict(n=SAMPLE, role="reference")
    ctx.close()
    print(json.dumps(table, indent=1))
    out = os.environ.get("MLENS_STUDY_OUT")
    if out:
        with open(out, "w") as fh:
            json.dump(table, fh, indent=1)
    rk = table["fp32_recentred_kahan"]
    assert rk["misbinned_frac"] <= 1e-4 and rk["bound_ratio"] <= 1.0, rk
    assert rk["rel_max"] <= 1e-5, rk
    # the naive loop is the error the re-centred + Kahan design removes
    assert table["fp32_naive"]["misbinned_frac"] > 10 * max(rk["misbinned_frac"], 1e-6)
