"""One magnification map shot by several processes (one per GPU): the ray grid's rows
are split into bands on tile boundaries, each process shoots its band into its own
map with mlens_shoot_rows, and the maps are summed across processes.

Section 2.2 runs the method as MPI tasks that each trace part of the rays and reduces
their maps into one.  Here the tasks are torch.distributed ranks (NCCL between GPUs,
gloo on CPU for the tests), and the reduction is one all-reduce of the uint32 maps as
int32 with SUM: two's-complement addition is addition modulo 2^32, the same as the
uint32 maps' own arithmetic, so the summed map equals a one-process map bit for bit.
Rays keep their whole-grid positions and tiles, so every band's rays are those of the
one-process shot.  Stars are replicated (every rank holds the whole field).

Host logic only: the shooting runs in libmlens's kernels, the sum in the collective
library.
"""
from __future__ import annotations

from . import mlens as M


def row_bands(ny: int, world: int, align: int = M.MLENS_ROW_ALIGN):
    """Rows [r0, r1) of each of `world` ranks: the grid's blocks of `align` rows (the
    last possibly short) dealt out in contiguous runs whose lengths differ by at most
    one block.  Every row belongs to exactly one band; a rank may get an empty band
    when there are fewer blocks than ranks."""
    if ny < 0 or world < 1 or align < 1:
        raise ValueError("need ny >= 0, world >= 1, align >= 1")
    blocks = (ny + align - 1) // align
    out = []
    for r in range(world):
        b0, b1 = r * blocks // world, (r + 1) * blocks // world
        out.append((min(b0 * align, ny), min(b1 * align, ny)))
    return out


def _group_rank_world(group):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def allreduce_counts(counts, group=None):
    """Sum a uint32 (or int32) map tensor over the ranks of `group`, in place."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return counts
    t = counts.view(torch.int32) if counts.dtype != torch.int32 else counts
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return counts


def allreduce_stats(st: dict, device=None, group=None) -> dict:
    """Sum the ray bookkeeping of every rank's band."""
    import torch
    import torch.distributed as dist
    keys = ("rays_total", "rays_binned", "rays_out", "rays_nan")
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return dict(st)
    t = torch.tensor([st[k] for k in keys], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return {k: int(v) for k, v in zip(keys, t.tolist())}


def shoot_learned_partitioned(ctx, rays, src, counts, group=None, stats: bool = False, stream=None):
    """As shoot_partitioned, with the learned far field fitted on `ctx` (every rank
    fits the same field with the same parameters, or loads the same saved fit):
    this rank's band through mlens_shoot_learned, then the sum over the group.  The
    learned kernel's row restriction keeps whole 32-row tiles, so the bands add up to
    the one-process learned map bit for bit."""
    rank, world = _group_rank_world(group)
    g = M.grid(rays)
    r0, r1 = row_bands(int(g.ny), world)[rank]
    if r1 > r0:
        st = M.mlens_shoot_learned(ctx, rays, src, counts, rows=(r0, r1), stats=stats, stream=stream)
    else:
        counts.zero_()
        st = dict(rays_total=0, rays_binned=0, rays_out=0, rays_nan=0)
    allreduce_counts(counts, group)
    if stats:
        return allreduce_stats(st, device=counts.device, group=group)
    return None


def shoot_partitioned(ctx, rays, src, counts, group=None, stats: bool = False, stream=None):
    """This rank's band of the grid into `counts` (overwritten), then the sum over the
    group: afterwards every rank holds the whole map.  Returns the summed stats when
    asked (a synchronising call)."""
    rank, world = _group_rank_world(group)
    g = M.grid(rays)
    r0, r1 = row_bands(int(g.ny), world)[rank]
    if r1 > r0:
        st = M.mlens_shoot_rows(ctx, rays, (r0, r1), src, counts, stats=stats, stream=stream)
    else:  # more ranks than row blocks: this rank contributes an empty map
        counts.zero_()
        st = dict(rays_total=0, rays_binned=0, rays_out=0, rays_nan=0)
    allreduce_counts(counts, group)
    if stats:
        return allreduce_stats(st, device=counts.device, group=group)
    return None
