"""The multi-process logic on CPU with the gloo backend (world sizes 2 and 3): the
ray-row partition of one map (bands on tile boundaries covering every row once) and
the sum of the ranks' maps with the all-reduce the GPU path uses, checked against the
oracle's whole map; bench.py's weak-scaling mode (an independent field per rank) and
its max-over-ranks job time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W
    wl = W.config("tiny")
    f = bench.rank_field(wl, rank)
    t = bench.max_over_ranks(1.0 + rank)  # rank r took 1 + r seconds
    out[rank] = (t, float(f.xy.sum()), f.n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_and_max_time():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.0          # max over ranks
    assert out[0][2] == out[1][2]                 # same size per rank
    assert out[0][1] != out[1][1]                 # independent fields


# ----------------------------------------------------------- ray-row partition
def test_row_bands_cover_every_row_once_on_block_boundaries():
    from paper_1703_09707_gb300 import partition as P
    for ny in (1, 31, 32, 33, 1000, 8192, 32768, 65537):
        for world in (1, 2, 3, 4, 7, 8, 16):
            bands = P.row_bands(ny, world)
            assert len(bands) == world
            rows = np.zeros(ny, dtype=np.int64)
            for r0, r1 in bands:
                assert 0 <= r0 <= r1 <= ny
                assert r0 % 32 == 0 and (r1 % 32 == 0 or r1 == ny)
                rows[r0:r1] += 1
            assert np.all(rows == 1), (ny, world)
            assert bands[0][0] == 0 and bands[-1][1] == ny
            assert all(bands[i][1] == bands[i + 1][0] for i in range(world - 1))
            sizes = [(r1 - r0 + 31) // 32 for r0, r1 in bands]
            assert max(sizes) - min(sizes) <= 1, (ny, world, sizes)


def _band_map(f, rays, src, r0, r1):
    """The oracle's map of ray rows [r0, r1) and its bookkeeping."""
    import oracle
    idx = np.arange(r0 * rays.nx, r1 * rays.nx, dtype=np.int64)
    pix = oracle.pixels(oracle.beta_rays(rays, idx, f), src)
    c = np.bincount(pix[pix >= 0], minlength=src.n).astype(np.uint32)
    st = dict(rays_total=int(idx.size), rays_binned=int(np.sum(pix >= 0)), rays_out=int(np.sum(pix == -1)),
              rays_nan=int(np.sum(pix == -2)))
    return c, st


def _partition_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as W
    from paper_1703_09707_gb300 import partition as P
    wl = W.config("tiny", rays_scale=0.2)  # 200 x 200 rays: 7 row blocks, the last one short
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    r0, r1 = P.row_bands(rays.ny, world)[rank]
    c, st = _band_map(f, rays, src, r0, r1)
    counts = torch.from_numpy(c.view(np.int32).copy())
    P.allreduce_counts(counts)
    tot = P.allreduce_stats(st)
    out[rank] = (counts.numpy().view(np.uint32).tobytes(), tot, (r0, r1))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_maps_sum_to_the_whole_map(world):
    """Each gloo rank forms its band's map with the oracle and the maps are summed
    with the same all-reduce the GPU path uses: every rank ends with the whole
    oracle map, bit for bit, and the summed bookkeeping equals the whole grid's."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import workloads as W
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    wl = W.config("tiny", rays_scale=0.2)
    f, rays, src = wl.fields[0], wl.rays[0], wl.srcs[0]
    full, st = oracle.shoot(rays, src, f)
    for r in range(world):
        got = np.frombuffer(out[r][0], dtype=np.uint32).reshape(src.ny, src.nx)
        assert np.array_equal(got, full), r
        assert out[r][1] == st, (out[r][1], st)
    assert sorted(out[r][2] for r in range(world))[0][0] == 0


def test_int32_sum_is_uint32_addition_across_the_wrap():
    """The reduction adds uint32 counts as int32: two's-complement addition is the
    same bits as uint32 addition modulo 2^32, also past 2^31."""
    a = np.array([2 ** 31 - 1, 2 ** 32 - 5, 7, 2 ** 31], dtype=np.uint32)
    b = np.array([1, 9, 2 ** 31 + 3, 2 ** 31 - 1], dtype=np.uint32)
    s = (torch.from_numpy(a.view(np.int32)) + torch.from_numpy(b.view(np.int32))).numpy().view(np.uint32)
    assert np.array_equal(s, (a.astype(np.uint64) + b.astype(np.uint64)).astype(np.uint32))
