"""Benchmark of the backward ray-shooting hot path (direct-sum deflection, Eq. 3;
beta = theta - alpha, Eq. 2; binning into a uint32 source map, Algorithm 1) on GB300.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                  [--workload paper|tiny|precision] [--precision fp32|fp32_naive|fp64]

One step = one whole magnification map of the workload (every ray of the grid against
every star, binned).  Default workload: 10^4 power-law stars (kappa_*=0.3,
kappa_c=0.2, gamma=(0.3,0)), 8192^2 rays over the 1.5x lens box, 1024^2 map.

Prints ONE JSON line (rank 0).  `value` = ray-star interactions per second over the
timed steps (device time, CUDA events on the launch stream, max over ranks);
`e2e` = the same metric through the public C ABI from host buffers (star upload,
shoot, map download, context teardown inside the timed region).
`--impl reference` times the FP64 CPU oracle (the reference arm) on a
bounded ray sample of the same workload.

Under torchrun (N > 1), by default (--scaling strong) the ranks share one map: rank r
shoots its band of ray rows (bands on tile boundaries, paper_1703_09707_gb300.partition)
and the uint32 maps are summed with one NCCL all-reduce per step, inside the timed
region (Section 2.2's MPI tasks and map reduction).  --scaling weak gives every rank its
own independent field of the same size instead (no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "ray-star interactions/s (direct-sum deflection + binning, one map per step)"
N_SM_GB300 = 152
MUFU_RCP_PER_SM_CLK = 16  # MUFU.RCP issue rate per SM per clock (one reciprocal per interaction)
# fma_pairs = 1 takes 10 of every 128 reciprocals from Newton-Raphson on the FMA pipe
FMA_RCP_SHARE = 10.0 / 128.0


def interaction_bound(fma_pairs: int):
    """(interactions per SM per clock, basis) of the direct sum's binding pipe.  Every
    interaction needs one reciprocal: from the MUFU unit (16 per SM per clock), or for
    the share FMA_RCP_SHARE (fma_pairs = 1) from three Newton-Raphson steps on the
    FMA pipe.  The FMA pipe (128 lane-ops per SM per clock) carries ~5.5 lane-ops per
    interaction plus ~6.5 per Newton reciprocal: 21 interactions per clock at that
    share, so MUFU still binds, at 16 / (1 - share) = 17.36."""
    if fma_pairs:
        r = MUFU_RCP_PER_SM_CLK / (1.0 - FMA_RCP_SHARE)
        return r, (f"MUFU.RCP {MUFU_RCP_PER_SM_CLK}/SM/clk for the {100 * (1 - FMA_RCP_SHARE):.1f} % of interactions "
                   f"whose reciprocal it forms ({r:.2f} interactions/SM/clk; the FMA pipe allows ~21)")
    return float(MUFU_RCP_PER_SM_CLK), f"MUFU.RCP {MUFU_RCP_PER_SM_CLK}/SM/clk (one reciprocal per interaction)"
SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="paper", choices=["paper", "tiny", "precision"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_naive", "fp64"])
    ap.add_argument("--rays-per-thread", type=int, default=8, choices=[4, 8])
    ap.add_argument("--star-stage", type=int, default=256, choices=[128, 256, 512])
    ap.add_argument("--fma-pairs", type=int, default=1, choices=[0, 1],
                    help="1: a share (7.8 %%) of the reciprocals from Newton-Raphson on the FMA pipe; 0: MUFU only")
    ap.add_argument("--rays-scale", type=float, default=1.0,
                    help="shrink the ray grid per axis (same field, boxes and map) for profiling runs")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--print-kernel-hash", action="store_true", help="print the FP32 kernel source hash and exit")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-fields and learned-far-field measurements that ride along the main line")
    ap.add_argument("--extras", default="batched,binning,lightcurve,split,learned,fit",
                    help="comma list of extra sections: batched, binning, lightcurve, split, learned, fit")
    ap.add_argument("--learned-tol", type=float, default=5e-6, help="per-cell validation bound of the learned field")
    ap.add_argument("--learned-order", type=int, default=10)
    ap.add_argument("--learned-errors", type=int, default=1, choices=[0, 1],
                    help="state the learned variants' per-ray errors against FP64 (0: skip, no 17 GB beta buffer)")
    ap.add_argument("--fit-stars", type=int, default=1_000_000,
                    help="stars of the field the fit section fits (same density and cell grid as the learned one)")
    ap.add_argument("--scaling", default="strong", choices=["strong", "weak"],
                    help="strong: the ranks split one map's ray rows and sum the maps; weak: one field per rank")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def rank_field(wl, rank: int):
    """Weak scaling: rank 0 shoots the workload's own field, rank r > 0 an independent
    field of the same size and lens terms (seed offset by r); no data is exchanged."""
    f = wl.fields[0]
    if rank == 0:
        return f
    return W.random_field(W.SEED_BASE + 100 + rank, f.n, f.kappa_star, f.kappa_c, f.gamma1, f.gamma2)


def max_over_ranks(seconds: float, device=None) -> float:
    """The job's time is the slowest rank's (torch.distributed all-reduce MAX)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(name, wl, precision, note_l2):
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    return {
        "workload": f"{name}: {f.n} stars, {rays.nx}x{rays.ny} rays, {src.nx}x{src.ny} map",
        "stars": f.n, "rays": [rays.nx, rays.ny], "map": [src.nx, src.ny],
        "ray_box": [rays.x0, rays.x1, rays.y0, rays.y1], "src_box": [src.x0, src.x1, src.y0, src.y1],
        "kappa_star": f.kappa_star, "kappa_c": f.kappa_c, "gamma": [f.gamma1, f.gamma2],
        "precision": precision, "l2": note_l2,
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- profiles
KERNEL_SOURCES = ("shoot_fp32.cu", "tile.cuh", "mlens_dev.cuh", "mlens_internal.h")


def kernel_source_hash() -> str:
    """Hash of the sources the FP32 shooting kernel is compiled from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1703_09707_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        ent = d[kernel_key]
        h = kernel_source_hash()
        if ent.get("source_sha256_16") != h:
            return None, ent
        return float(ent["dram_bytes_per_launch"]), ent
    except (OSError, KeyError, ValueError):
        return None, None


# ------------------------------------------------------------ cpu baseline
def cpu_oracle_rate(field, rays, target_s: float, seed: int = 11):
    """Time the FP64 oracle (as it stands, all host cores) on a random ray sample
    sized for about target_s seconds; returns (interactions/s, cores, sample note)."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    n = max(field.n, 1)
    probe = W.ray_sample(rays, 2000, seed)
    t0 = time.perf_counter()
    oracle.beta_rays(rays, probe, field)
    dt = max(time.perf_counter() - t0, 1e-4)
    k = int(min(rays.n, max(2000, 2000 * target_s / dt)))
    idx = W.ray_sample(rays, k, seed + 1)
    t0 = time.perf_counter()
    oracle.beta_rays(rays, idx, field)
    dt = time.perf_counter() - t0
    return k * n / dt, cores, f"{k} random rays of the grid x all {field.n} stars, FP64, {dt:.1f} s"


# --------------------------------------------------------------- batched
def bench_batched(M, torch, steps: int, warmup: int, flush):
    """256 independent fields (N_* log-uniform in [1e2, 1e4], 2048^2 rays, 512^2 maps):
    one autotuned persistent launch replayed as a CUDA graph versus one mlens_shoot
    launch per field with the same launch shape.  Device time, CUDA events."""
    wl = W.batched_config()
    ctxs = [M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32) for f in wl.fields]
    counts = [torch.empty(s.n, dtype=torch.int32, device="cuda") for s in wl.srcs]
    inter = sum(r.n * f.n for r, f in zip(wl.rays, wl.fields))
    stream = torch.cuda.current_stream()
    b = M.mlens_batch_create(ctxs, wl.rays, wl.srcs, counts)
    t0 = time.perf_counter()
    rpt, stage, fma, tune_ms = M.mlens_batch_tune(b)
    tune_s = time.perf_counter() - t0

    def timed(fn):
        for _ in range(warmup):
            flush.fill_(0.0)
            fn()
        ms = []
        for i in range(steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms)

    persistent_ms = timed(lambda: M.mlens_batch_run(b))
    for c in ctxs:
        M.mlens_set_tuning(c, rpt, stage, fma)
    per_field_ms = timed(lambda: [M.mlens_shoot(c, r, s, k) for c, r, s, k in zip(ctxs, wl.rays, wl.srcs, counts)])
    b.close()
    for c in ctxs:
        c.close()
    nf = len(wl.fields)
    return {
        "workload": f"batched: {nf} fields, N_* log-uniform [1e2,1e4] (mean {inter / (nf * wl.rays[0].n):.0f}), "
                    f"{wl.rays[0].nx}^2 rays, {wl.srcs[0].nx}^2 maps",
        "maps_per_s": nf / (persistent_ms / 1e3),
        "maps_per_s_per_field_launches": nf / (per_field_ms / 1e3),
        "speedup_vs_per_field_launches": per_field_ms / persistent_ms,
        "interactions_per_s": inter / (persistent_ms / 1e3),
        "ms_per_batch": persistent_ms, "ms_per_batch_per_field_launches": per_field_ms,
        "tuned": {"rays_per_thread": rpt, "star_stage": stage, "fma_pairs": fma, "tune_s": tune_s},
        "gpu_launches_per_batch": 1,
    }


# --------------------------------------------------------------- binning
def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def bench_binning(M, torch, steps: int, warmup: int, flush):
    """The binning step alone on the paper-shaped workload: the 8192^2 float-pair beta
    records of one map (1.07 GB, above L2) binned into the 1024^2 map by the standalone
    kernel in grid order (64 x 64 ray blocks per CTA) and in flat order (4096
    consecutive records per CTA), and the fused epilogue's cost: the same grid shot
    through a star-free field (ray generation, the smooth term, beta and binning)."""
    wl = W.config("paper")
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    stream = torch.cuda.current_stream()
    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    beta = torch.empty(rays.n * 4, dtype=torch.float32, device="cuda")
    st = M.mlens_shoot_beta(ctx, rays, src, counts, beta, stats=True)
    ref = counts.clone()
    ctx.close()

    def timed(fn):
        for _ in range(warmup):
            flush.fill_(0.0)
            fn()
        ms = []
        for i in range(steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms)

    peak, basis = measured_hbm_gbs()
    algo_bytes = 16 * rays.n + 4 * src.n  # records read once, map written once
    out = {"workload": f"paper: {rays.nx}x{rays.ny} beta records (float pairs, {16 * rays.n / 1e9:.2f} GB), "
                       f"{src.nx}x{src.ny} map", "rays_binned": st["rays_binned"],
           "algorithmic_bytes": algo_bytes, "hbm_peak_gbs": peak, "hbm_peak_basis": basis}
    for name, fn in (("grid_order", lambda: M.mlens_bin_grid(beta, rays, src, counts)),
                     ("flat_order", lambda: M.mlens_bin(beta, rays.n, src, counts))):
        ms = timed(fn)
        assert torch.equal(counts, ref), name
        gbs = algo_bytes / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "records_per_s": rays.n / (ms / 1e3), "gbs": gbs, "hbm_frac": gbs / peak}
    del beta
    empty = M.mlens_create(np.zeros((0, 2)), np.zeros(0), f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32)
    ms = timed(lambda: M.mlens_shoot(empty, rays, src, counts))
    empty.close()
    out["fused_epilogue"] = {"ms": ms, "rays_per_s": rays.n / (ms / 1e3),
                             "note": "mlens_shoot over a field without stars: everything but the direct sum"}
    return out


# ------------------------------------------------------------ light curves
def bench_lightcurve(M, torch, steps: int, warmup: int, flush, peak_fp32_fma: float):
    """The paper field's 8192^2 rays binned into a 4096^2 map (the learned workload's
    map size) and convolved with a Gaussian source (sigma = 0.05 theta_E, 10 pixels)
    and a uniform disk (R = 0.1 theta_E, 20 pixels), then a 4096-point light curve
    across it; CUDA events, L2 flushed before each timed call.  The Gaussian's two
    separable passes are bound by FP32 multiply-adds (2K + 1 per pixel and pass), so
    its fraction is also stated against the FP32 FMA rate."""
    wl = W.config("paper")
    f, rays = wl.fields[0], wl.rays[0]
    src = W.Grid(-10.0, 10.0, -10.0, 10.0, 4096, 4096)
    stream = torch.cuda.current_stream()
    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    M.mlens_shoot(ctx, rays, src, counts)
    ctx.close()
    scale = M.mlens_magnification_scale(rays, src)
    conv = torch.empty(src.n, dtype=torch.float32, device="cuda")
    curve = torch.empty(4096, dtype=torch.float32, device="cuda")

    def timed(fn):
        for _ in range(warmup):
            fn()
        ms = []
        for i in range(steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms)

    peak, basis = measured_hbm_gbs()
    out = {"workload": f"paper field, {rays.nx}^2 rays into a {src.nx}^2 map over [-10,10]^2",
           "hbm_peak_gbs": peak, "hbm_peak_basis": basis}
    for key, prof, size in (("gaussian_sigma_0.05", M.MLENS_PROFILE_GAUSSIAN, 0.05),
                            ("disk_r_0.1", M.MLENS_PROFILE_DISK, 0.1)):
        work = torch.empty(M.mlens_convolve_workspace(src, prof, size), dtype=torch.uint8, device="cuda")
        ms = timed(lambda: M.mlens_convolve(counts, src, prof, size, conv, scale=scale, work=work))
        # bytes a single pass would move: the uint32 map in, the float32 map out
        gbs = 8.0 * src.n / (ms / 1e3) / 1e9
        out[key] = {"ms": ms, "pixels_per_s": src.n / (ms / 1e3), "min_bytes_gbs": gbs, "hbm_frac": gbs / peak,
                    "note": "asynchronous call with a caller workspace: setup kernel and passes"}
        if prof == M.MLENS_PROFILE_GAUSSIAN:
            # taps per axis: the library's half-width is ceil(4 sigma / pixel)
            kx = math.ceil(4.0 * size / ((src.x1 - src.x0) / src.nx))
            ky = math.ceil(4.0 * size / ((src.y1 - src.y0) / src.ny))
            fmas = src.n * ((2 * kx + 1) + (2 * ky + 1))
            out[key].update({"taps": [2 * kx + 1, 2 * ky + 1], "fma_per_s": fmas / (ms / 1e3),
                             "fma_frac": fmas / (ms / 1e3) / peak_fp32_fma,
                             "fma_peak_basis": "FP32 FMA: 128 per SM per clock x SMs x max SM clock"})
        del work
    ms = timed(lambda: M.mlens_light_curve(conv, src, (-8.0, -3.0), (8.0, 4.0), 4096, curve))
    out["light_curve_4096_points_ms"] = ms
    return out


# ----------------------------------------------------------------- split
def bench_split(M, torch, flush, peak):
    """10^7 stars on ray grids of 256^2 and 512^2 rays (32 and 128 tiles of 64 x 32
    rays, fewer than the GPU's 152 SMs): each tile's star sum split over clusters of
    1, 2, 4 and 8 CTAs and, through global memory, over the automatic choice's number
    of CTAs; one CUDA-event-timed map per setting after a warm-up map."""
    wl = W.config("large_n")
    f, rays0, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    stream = torch.cuda.current_stream()
    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    out = {"workload": f"large_n: {f.n} stars, {src.nx}x{src.ny} map; ray grids over the same box"}
    for n in (256, 512):
        rays = W.Grid(rays0.x0, rays0.x1, rays0.y0, rays0.y1, n, n)
        M.mlens_set_star_split(ctx, 0)
        auto = M.mlens_star_split_for(ctx, rays)
        inter = rays.n * f.n
        by = {}
        for split in sorted({1, 2, 4, 8, auto}):
            M.mlens_set_star_split(ctx, split)
            M.mlens_shoot(ctx, rays, src, counts)
            flush.fill_(float(split))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.mlens_shoot(ctx, rays, src, counts)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            by[str(split)] = {"ms": ms, "interactions_per_s": inter / (ms / 1e3),
                              "roofline_frac": inter / (ms / 1e3) / peak}
        out[f"rays_{n}"] = {"tiles": -(-n // 64) * -(-n // 32), "auto_split": auto, "by_split": by,
                            "speedup_auto_vs_unsplit": by["1"]["ms"] / by[str(auto)]["ms"]}
    ctx.close()
    return out


# --------------------------------------------------------------- learned
LEARNED_STRIPS = ((0, 768), (10752, 11520), (16128, 16896), (32000, 32768))


def _grid_theta(rays, idx):
    """Cell-centre image positions of grid rays (linear index j*nx + i), formed with the
    FP64 kernel's operations: x0 + (i + 1/2) ((x1 - x0) / nx)."""
    i, j = idx % rays.nx, idx // rays.nx
    tx = rays.x0 + (i + 0.5) * ((rays.x1 - rays.x0) / rays.nx)
    ty = rays.y0 + (j + 0.5) * ((rays.y1 - rays.y0) / rays.ny)
    return np.stack([tx, ty], 1)


def _pixel_f64(bx, by, src):
    """Source pixel of FP64 positions (-1 outside the map)."""
    ux = np.floor((bx - src.x0) * (src.nx / (src.x1 - src.x0)))
    uy = np.floor((by - src.y0) * (src.ny / (src.y1 - src.y0)))
    ok = np.isfinite(ux) & np.isfinite(uy) & (ux >= 0) & (ux < src.nx) & (uy >= 0) & (uy < src.ny)
    return np.where(ok, uy * src.nx + ux, -1).astype(np.int64)


def _errors_vs_fp64(b4, b64, src):
    """Per-ray error of float-pair beta against FP64 beta: |d beta| in source pixels
    (mean, p99.99, max), max |d alpha| in theta_E (= max |d beta|), misbinned fraction."""
    bg = b4[:, :2].astype(np.float64) + b4[:, 2:].astype(np.float64)
    w = min((src.x1 - src.x0) / src.nx, (src.y1 - src.y0) / src.ny)
    d = np.linalg.norm(bg - b64, axis=1)
    fin = np.isfinite(d)
    pg = _pixel_f64(bg[:, 0], bg[:, 1], src)
    p6 = _pixel_f64(b64[:, 0], b64[:, 1], src)
    return {"rays": int(d.size), "dbeta_mean_px": float(d[fin].mean() / w),
            "dbeta_p9999_px": float(np.quantile(d[fin], 0.9999) / w), "dbeta_max_px": float(d[fin].max() / w),
            "dalpha_max_theta_e": float(d[fin].max()), "misbinned_frac": float(np.mean(pg != p6))}


def bench_learned(M, torch, steps: int, flush, tol: float, order: int, errors: bool = True):
    """10^6 stars, 32768^2 rays, 4096^2 map: the learned far field (fit on the GPU,
    then one persistent launch per map) against the plain direct sum.  The plain
    map of the whole grid takes minutes, so both paths are compared on four strips of
    768 ray rows (the first and last rows of the grid and two interior strips, 1e14
    interactions for the plain path): the strips give the plain path's throughput and
    the map error of the learned path (relative L1 over the strips' maps).  Every
    variant's per-ray error is stated against FP64 on 2e4 rays sampled from the
    strips: the FP64 kernel (mlens_trace, bit-identical to the FP64 oracle) gives the
    reference, outside the timed regions.  Variants: with the network, without it at
    the same exact order, and the exact series alone at higher orders (the fastest of
    those meeting L1 <= 1e-3 is the best non-learned variant)."""
    wl = W.config("learned")
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    stream = torch.cuda.current_stream()
    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32)
    strip_rays = sum(rays.nx * (j1 - j0) for j0, j1 in LEARNED_STRIPS)
    plain_maps, plain_ms = [], 0.0
    torch.cuda.synchronize()
    for j0, j1 in LEARNED_STRIPS:
        cp = torch.empty(src.n, dtype=torch.int32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M.mlens_shoot_rows(ctx, rays, (j0, j1), src, cp)
        e1.record(stream)
        e1.synchronize()
        plain_ms += e0.elapsed_time(e1)
        plain_maps.append(cp.cpu().numpy().view(np.uint32).astype(np.int64))
    plain_rate = strip_rays * f.n / (plain_ms / 1e3)
    plain_full_s = rays.n * f.n / plain_rate
    # sampled rays and their FP64 beta
    rng = np.random.default_rng(11)
    idx = np.concatenate([np.sort(rng.choice(rays.nx * (j1 - j0), 5000, replace=False)) + j0 * rays.nx
                          for j0, j1 in LEARNED_STRIPS]).astype(np.int64)
    b64 = M.mlens_trace(ctx, _grid_theta(rays, idx)) if errors else None
    idx_t = torch.from_numpy(idx).cuda()
    # only the strips' rows are written
    beta = torch.empty((rays.n, 4), dtype=torch.float32, device="cuda") if errors else None
    out = {"workload": f"learned: {f.n} stars, {rays.nx}^2 rays, {src.nx}^2 map, 256 x 86 cells of 0.46875 theta_E",
           "plain": {"interactions_per_s": plain_rate, "map_s_estimated": plain_full_s,
                     "measured_on": f"ray rows {list(LEARNED_STRIPS)} ({strip_rays} rays)"},
           "errors_reference": "FP64 kernel (mlens_trace; bit-identical to the FP64 oracle) on 2e4 rays "
                               "sampled from the strips"}
    # the plain path's own error on the same rays, for comparison
    if errors:
        cpb = torch.empty(src.n, dtype=torch.int32, device="cuda")
        for j0, j1 in LEARNED_STRIPS:
            M.mlens_shoot_rows(ctx, rays, (j0, j1), src, cpb, beta=beta)
        out["plain"]["errors_vs_fp64"] = _errors_vs_fp64(beta.index_select(0, idx_t).cpu().numpy(), b64, src)
    # the learned path, the same series without the network (the ablation), and the
    # exact series alone at higher orders
    variants = [("with_network", 1, order), ("series_only", 0, order)]
    variants += [(f"series_only_order{o}", 0, o) for o in (12, 14, 16) if o > order]
    for key, use_net, o in variants:
        t0 = time.perf_counter()
        rep = M.mlens_fit_far_field(ctx, rays, M.fit_params(cells_x=256, order=o, use_network=use_net,
                                                            tolerance=tol))
        fit_s = time.perf_counter() - t0
        cl = torch.empty(src.n, dtype=torch.int32, device="cuda")
        strip_s = 0.0
        num = den = 0
        for (j0, j1), cp_h in zip(LEARNED_STRIPS, plain_maps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            M.mlens_shoot_learned(ctx, rays, src, cl, beta=beta, rows=(j0, j1))
            b.record(stream)
            b.synchronize()
            strip_s += a.elapsed_time(b) / 1e3
            cl_h = cl.cpu().numpy().view(np.uint32).astype(np.int64)
            num += np.abs(cl_h - cp_h).sum()
            den += cp_h.sum()
        errs = _errors_vs_fp64(beta.index_select(0, idx_t).cpu().numpy(), b64, src) if errors else None
        # whole map timed unless its fallback tiles alone would take minutes (then the
        # strips' time is scaled to the grid)
        fallback_s = rep["tiles_fallback"] * 2048 * f.n / plain_rate
        if fallback_s <= 5.0:
            counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
            M.mlens_shoot_learned(ctx, rays, src, counts)  # warm-up
            ms = []
            for i in range(steps):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                M.mlens_shoot_learned(ctx, rays, src, counts)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            learned_s = statistics.mean(ms) / 1e3
            timing = f"whole map, mean of {steps} CUDA-event-timed launches"
        else:
            learned_s = strip_s * rays.n / strip_rays
            timing = f"estimated from the strips ({strip_s:.3f} s)"
        l1 = float(num / max(den, 1))
        out[key] = {
            "map_s": learned_s, "map_s_timing": timing, "maps_per_s": 1.0 / learned_s,
            "effective_interactions_per_s": rays.n * f.n / learned_s,
            "speedup_vs_plain": plain_full_s / learned_s,
            "map_rel_l1_vs_plain": l1, "equal_error": l1 <= 1e-3,
            **({"errors_vs_fp64": errs} if errors else {}),
            "fallback_cells": rep["cells_fallback"], "cells": rep["cells"],
            "fallback_tiles": rep["tiles_fallback"], "tiles": rep["tiles"],
            "val_mean_err": rep["val_mean_err_net"] if use_net else rep["val_mean_err_series"],
            "val_max_err": rep["val_max_err_net"] if use_net else rep["val_max_err_series"],
            "fit_s": fit_s, "fit_seconds": {"coefficients": rep["seconds_coefficients"],
                                            "train": rep["seconds_train"], "validate": rep["seconds_validate"]},
            "train_steps": rep["train_steps"], "order": o, "tolerance": tol,
        }
    out["network_gain_at_equal_order"] = out["series_only"]["map_s"] / out["with_network"]["map_s"]
    series = {k: v for k, v in out.items() if k.startswith("series_only") and isinstance(v, dict) and v["equal_error"]}
    if series:
        best = min(series, key=lambda k: series[k]["map_s"])
        out["best_series_variant"] = best
        # > 1: the trained network is faster than every series-only variant at equal map error
        out["network_gain_vs_best_series"] = series[best]["map_s"] / out["with_network"]["map_s"]
    ctx.close()
    return out


# ------------------------------------------------------------------- fit
def bench_fit(M, torch, fit_stars: int, tol: float, order: int, peak_fp32_lane_ops: float):
    """One far-field fit on the learned workload's ray grid (256 x 86 cells of 0.46875
    theta_E) with `fit_stars` stars at the same density (10^6: the learned section's
    field): its time split into the series coefficients, the training and the
    validation, the training step time, and the coefficient kernel's pair rate
    against its FP32 bound (about 249 FP32 lane operations per (cell, far star)
    pair)."""
    wl = W.config("learned")
    f, rays = wl.fields[0], wl.rays[0]
    if fit_stars != f.n:
        f = W.random_field(W.SEED_BASE + 4, fit_stars, f.kappa_star, f.kappa_c, f.gamma1, f.gamma2)
    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, M.MLENS_PREC_FP32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = M.mlens_fit_far_field(ctx, rays, M.fit_params(cells_x=256, order=order, use_network=1, tolerance=tol))
    fit_s = time.perf_counter() - t0
    ctx.close()
    pairs = rep["cells"] * f.n  # (cell, star) pairs; the near stars (~1e-5 of them) are counted too
    coef_s = rep["seconds_coefficients"]
    lane_ops = 249.0
    return {"stars": f.n, "cells": rep["cells"], "fit_s": fit_s,
            "seconds": {"coefficients": coef_s, "train": rep["seconds_train"], "validate": rep["seconds_validate"]},
            "train_steps": rep["train_steps"], "train_step_us": 1e6 * rep["seconds_train"] / max(rep["train_steps"], 1),
            "fallback_cells": rep["cells_fallback"], "val_max_err": rep["val_max_err_net"],
            "coefficients": {"pairs": pairs, "pairs_per_s": pairs / coef_s,
                             "roofline_frac": pairs * lane_ops / coef_s / peak_fp32_lane_ops,
                             "peak_basis": "FP32 pipe: 128 lane-ops/SM/clk x SMs x max SM clock; "
                                           f"{lane_ops:.0f} lane-ops per (cell, star) pair"}}


# ------------------------------------------------------------------- main
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = W.config(args.workload)
    f, rays = wl.fields[0], wl.rays[0]
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    n = max(f.n, 1)
    # per step: a bounded sample of the workload, sized so the whole run stays short
    per_step_s = max(1.0, min(10.0, 60.0 / max(1, args.steps + args.warmup)))
    probe = W.ray_sample(rays, 1000, 5)
    t0 = time.perf_counter()
    oracle.beta_rays(rays, probe, f)
    dt = max(time.perf_counter() - t0, 1e-4)
    k = int(min(rays.n, max(1000, 1000 * per_step_s / dt)))
    for w in range(args.warmup):
        oracle.beta_rays(rays, W.ray_sample(rays, max(1000, k // 10), 100 + w), f)
    times = []
    for s in range(args.steps):
        idx = W.ray_sample(rays, k, 1000 + s)
        t0 = time.perf_counter()
        oracle.beta_rays(rays, idx, f)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = k * n * args.steps / tot
    sample = f"{k} random rays x all {f.n} stars per step (FP64 oracle, {cores} threads)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args.workload, wl, "fp64 (CPU oracle)", "n/a (CPU)"),
        "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_mine(args):
    import torch
    import torch.distributed as dist

    from paper_1703_09707_gb300 import build as B
    from paper_1703_09707_gb300 import mlens as M

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    M.load()
    prec = M.PRECISIONS[args.precision]

    from paper_1703_09707_gb300 import partition as P

    wl = W.config(args.workload, rays_scale=args.rays_scale)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    strong = args.scaling == "strong"
    if not strong:
        f = rank_field(wl, rank)
    band = P.row_bands(rays.ny, world)[rank] if strong else (0, rays.ny)
    n_inter = rays.nx * (band[1] - band[0]) * f.n   # this rank's interactions per step
    n_inter_job = rays.n * f.n * (1 if strong else world)

    ctx = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, prec)
    M.mlens_set_tuning(ctx, args.rays_per_thread, args.star_stage, args.fma_pairs)
    counts = torch.empty(src.n, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(c, counts_buf):
        """One map: this rank's band, then (N > 1, strong) the sum over ranks."""
        if band[1] > band[0]:
            M.mlens_shoot_rows(c, rays, band, src, counts_buf)
        else:
            counts_buf.zero_()
        if strong:
            P.allreduce_counts(counts_buf)

    if band[1] > band[0]:  # checks the call works; warms the module
        st = M.mlens_shoot_rows(ctx, rays, band, src, counts, stats=True)
        assert st["rays_binned"] + st["rays_out"] + st["rays_nan"] == st["rays_total"]
    if strong:
        st = P.shoot_partitioned(ctx, rays, src, counts, stats=True)
        assert st["rays_total"] == rays.n and st["rays_binned"] + st["rays_out"] + st["rays_nan"] == rays.n
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step(ctx, counts)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))  # > L2 (129 MB) write between steps, outside the events
        ev[i][0].record(stream)
        step(ctx, counts)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    dev_s = max_over_ranks(dev_s, device="cuda")
    value = n_inter_job * args.steps / dev_s
    kernel_ms = statistics.mean(step_ms)

    # ------------------------------------------------ end to end through the C ABI
    # host star arrays -> mlens_create (upload) -> shoot -> map to host -> destroy
    host_counts = torch.empty(src.n, dtype=torch.int32, pin_memory=True)
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(e2e_steps):
        c2 = M.mlens_create(f.xy, f.m, f.kappa_c, f.gamma1, f.gamma2, prec)
        M.mlens_set_tuning(c2, args.rays_per_thread, args.star_stage, args.fma_pairs)
        step(c2, counts)
        host_counts.copy_(counts, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        c2.close()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, device="cuda")
    e2e_value = n_inter_job * e2e_steps / e2e_s
    n_pad = (f.n + 31) // 32 * 32  # the library pads the stars it uploads to a multiple of 32
    e2e = {"value": e2e_value, "unit": "interactions/s", "h2d_bytes_per_step": int(16 * n_pad),
           "d2h_bytes_per_step": int(4 * src.n), "steps": e2e_steps,
           "note": "mlens_create from host arrays + mlens_shoot_rows (+ map all-reduce for N > 1) + map download "
                   "+ mlens_destroy, wall clock"}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ----------------------------------------------------------------- roofline
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    per_clk, basis = interaction_bound(args.fma_pairs)
    peak = n_sm * per_clk * SM_MAX_MHZ * 1e6
    achieved = n_inter / (kernel_ms / 1e3)
    key = f"shoot_fp32_{args.workload}_rpt{args.rays_per_thread}_fma{args.fma_pairs}"
    traffic, _ = profile_traffic(key) if args.precision != "fp64" else (None, None)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "interactions/s", "frac": achieved / peak,
            "traffic": traffic,
            "peak_basis": f"{basis} x {n_sm} SMs x {SM_MAX_MHZ:.0f} MHz (max SM clock)",
            "kernel": "k_shoot_fp32" if args.precision != "fp64" else "k_fp64",
            "kernel_ms": kernel_ms}
    if args.fma_pairs:
        # context: the same rate against MUFU.RCP alone (every reciprocal on MUFU)
        roof["frac_of_mufu_only_bound"] = achieved / (n_sm * MUFU_RCP_PER_SM_CLK * SM_MAX_MHZ * 1e6)
    if clk and clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (n_sm * per_clk * clk["sm_mhz"] * 1e6)

    line = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": args.scaling, "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
        "data": "synthetic (seeded star field, paper-shaped)",
        "config": workload_config(args.workload, wl, args.precision,
                                  f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write, outside the events)"),
        "maps_per_s": args.steps * (1 if strong else world) / dev_s,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk,
        "wall_s_timed": t_wall,
        "device": props.name,
    }
    line["config"]["rays_per_thread"] = args.rays_per_thread
    line["config"]["fma_pairs"] = args.fma_pairs
    line["config"]["star_stage"] = args.star_stage
    if world > 1:
        line["config"]["parallelism"] = (f"ray rows split over {world} ranks ({P.row_bands(rays.ny, world)[0][1]} "
                                         "rows on rank 0), uint32 maps summed by NCCL all-reduce each step"
                                         if strong else f"one independent field per rank ({world} ranks)")
    extras = set(x for x in args.extras.split(",") if x)
    if not args.no_extras and world == 1 and args.workload == "paper" and args.rays_scale == 1.0:
        if "batched" in extras:
            bt = bench_batched(M, torch, max(2, min(args.steps, 5)), 2, flush)
            peak_b = n_sm * interaction_bound(bt["tuned"]["fma_pairs"])[0] * SM_MAX_MHZ * 1e6
            bt["roofline_frac"] = bt["interactions_per_s"] / peak_b
            line["batched"] = bt
        if "binning" in extras:
            bn = bench_binning(M, torch, max(3, min(args.steps, 10)), 3, flush)
            bn["fused_epilogue"]["share_of_paper_step"] = bn["fused_epilogue"]["ms"] / kernel_ms
            line["binning"] = bn
        if "lightcurve" in extras:
            line["lightcurve"] = bench_lightcurve(M, torch, max(3, min(args.steps, 10)), 2, flush,
                                                  n_sm * 128 * SM_MAX_MHZ * 1e6)
        if "split" in extras:
            line["split"] = bench_split(M, torch, flush, peak)
        if "learned" in extras:
            line["learned"] = bench_learned(M, torch, max(2, min(args.steps, 3)), flush, args.learned_tol,
                                            args.learned_order, bool(args.learned_errors))
        if "fit" in extras:
            line["fit"] = bench_fit(M, torch, args.fit_stars, args.learned_tol, args.learned_order,
                                    n_sm * 128 * SM_MAX_MHZ * 1e6)
    if not args.no_cpu_baseline and world == 1:
        v, cores, sample = cpu_oracle_rate(f, rays, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.print_kernel_hash:
        print(kernel_source_hash())
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
