"""Source-profile convolution and light curves on the GPU against the FP64 oracle
(oracle/lightcurve.py): the disk convolution and the light curve bit for bit, the
Gaussian within a bound derived from FP32 accumulation, edge cases, a full-size
map on sampled pixels, and the point-lens finite-source magnification end to end."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from oracle import lightcurve as LC  # noqa: E402
from gpu_util import shoot_gpu  # noqa: E402
from paper_1703_09707_gb300 import mlens as M  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev_counts(c):
    return torch.from_numpy(np.ascontiguousarray(c).view(np.int32).reshape(-1)).cuda()


def _gpu_conv(c, src, profile, size, scale=1.0):
    out = torch.empty(src.ny * src.nx, dtype=torch.float32, device="cuda")
    M.mlens_convolve(_dev_counts(c), src, profile, size, out, scale=scale)
    return out.cpu().numpy().reshape(src.ny, src.nx)


def _gauss_bound(ref, src, size):
    # FP32: the row pass sums 2Kx+1 products, the column pass 2Ky+1, then the scale;
    # each rounding is at most 2^-24 relative to a partial sum of non-negative terms
    dx, dy = (src.x1 - src.x0) / src.nx, (src.y1 - src.y0) / src.ny
    kx, ky = math.ceil(4 * size / dx), math.ceil(4 * size / dy)
    return 2.0 * (2 * kx + 2 * ky + 8) * 2.0 ** -24 * np.abs(ref) + 1e-30


@pytest.mark.parametrize("nx,ny,box,size", [
    (301, 173, (-1.5, 1.5, -0.7, 1.0), 0.05),   # ragged tiles, anisotropic pixels
    (1024, 96, (-4.0, 4.0, -0.5, 0.5), 0.05),   # wide rows, several row tiles
    (64, 700, (-0.3, 0.3, -3.0, 3.0), 0.06),    # tall map, several column tiles
    (60, 40, (-0.3, 0.3, -0.2, 0.2), 0.6),      # 4 sigma = 240 px, near the 256 limit, wider than the map
])
def test_gaussian_matches_the_oracle(nx, ny, box, size):
    rng = np.random.default_rng(nx + ny)
    src = W.Grid(box[0], box[1], box[2], box[3], nx, ny)
    c = rng.poisson(30.0, (ny, nx)).astype(np.uint32)
    c[rng.random((ny, nx)) < 0.02] = 50000  # caustic-like spikes
    got = _gpu_conv(c, src, M.MLENS_PROFILE_GAUSSIAN, size, 0.37)
    ref = LC.convolve(c, src, LC.GAUSSIAN, size, 0.37)
    bad = np.abs(got - ref) > _gauss_bound(ref, src, size)
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - ref) / np.maximum(ref, 1e-30))))


@pytest.mark.parametrize("nx,ny,box,size", [
    (301, 173, (-1.5, 1.5, -0.7, 1.0), 0.1),
    (5000, 3, (-5.0, 5.0, -0.003, 0.003), 0.05),  # rows longer than one prefix chunk
    (2, 900, (-0.01, 0.01, -4.5, 4.5), 0.3),      # narrow map: runs clamp at both ends
    (50, 40, (-1.0, 1.0, -1.0, 1.0), 5.0),        # disk far larger than the map
    (77, 66, (-1.0, 1.0, -1.0, 1.0), 0.0),        # radius 0: the map itself
])
def test_disk_is_bit_exact(nx, ny, box, size):
    rng = np.random.default_rng(nx * ny)
    src = W.Grid(box[0], box[1], box[2], box[3], nx, ny)
    c = rng.poisson(30.0, (ny, nx)).astype(np.uint32)
    c[rng.random((ny, nx)) < 0.01] = 4_000_000_000  # near the uint32 limit: int64 sums
    got = _gpu_conv(c, src, M.MLENS_PROFILE_DISK, size, 1.7)
    ref = LC.convolve(c, src, LC.DISK, size, 1.7).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_one_pixel_map():
    src = W.Grid(0.0, 1.0, 0.0, 1.0, 1, 1)
    c = np.array([[12345]], dtype=np.uint32)
    # zero padding: the disk's other 28 offsets fall outside the map
    d = _gpu_conv(c, src, M.MLENS_PROFILE_DISK, 3.0, 2.0)[0, 0]
    assert d == np.float32(LC.convolve(c, src, LC.DISK, 3.0, 2.0)[0, 0]) == np.float32(12345 * 2.0 / 29)
    assert _gpu_conv(c, src, M.MLENS_PROFILE_DISK, 0.5, 2.0)[0, 0] == np.float32(12345 * 2.0)
    g = _gpu_conv(c, src, M.MLENS_PROFILE_GAUSSIAN, 0.5, 1.0)[0, 0]
    assert g == pytest.approx(LC.convolve(c, src, LC.GAUSSIAN, 0.5)[0, 0], rel=1e-6)


def test_light_curve_is_bit_exact():
    rng = np.random.default_rng(2)
    src = W.Grid(-2.0, 2.0, -1.0, 3.0, 131, 77)
    m = (rng.random((77, 131)) * 10).astype(np.float32)
    md = torch.from_numpy(m.reshape(-1)).cuda()
    for b0, b1, n in [((-1.9, -0.8), (1.7, 2.9), 1001), ((-3.0, 1.0), (3.0, 1.2), 64), ((0.3, 0.4), (0.3, 0.4), 1),
                      ((-2.0 + 2.0 / 131 * 7.5, -1.0 + 4.0 / 77 * 3.5), (5.0, 9.0), 2)]:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        M.mlens_light_curve(md, src, b0, b1, n, out)
        ref = LC.light_curve(m, src, b0, b1, n).astype(np.float32)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32)), (b0, b1, n)


def test_full_size_map_on_sampled_pixels():
    """The learned workload's 4096^2 map size (a paper-field map shot on the GPU):
    both profiles on 400 sampled pixels against the oracle's pointwise form."""
    wl = W.config("paper", rays_scale=0.5)
    f, rays = wl.fields[0], wl.rays[0]
    src = W.Grid(-10.0, 10.0, -10.0, 10.0, 4096, 4096)
    c, _, _ = shoot_gpu(f, rays, src, want_beta=False)
    scale = M.mlens_magnification_scale(rays, src)
    assert scale == pytest.approx(LC.magnification_scale(rays, src), rel=1e-15)
    rng = np.random.default_rng(4)
    js, is_ = rng.integers(0, 4096, 400), rng.integers(0, 4096, 400)
    for prof, oprof, size in ((M.MLENS_PROFILE_GAUSSIAN, LC.GAUSSIAN, 0.02), (M.MLENS_PROFILE_DISK, LC.DISK, 0.05)):
        got = _gpu_conv(c, src, prof, size, scale)[js, is_]
        ref = LC.convolve_at(c, src, oprof, size, scale, js, is_)
        if prof == M.MLENS_PROFILE_DISK:
            assert np.array_equal(got.view(np.uint32), ref.astype(np.float32).view(np.uint32))
        else:
            assert np.all(np.abs(got - ref) <= _gauss_bound(ref, src, size))


def test_point_lens_disk_source_light_curve():
    """GPU map of a point lens, GPU disk convolution, GPU light curve through the
    lens: at zero impact parameter the magnification is sqrt(1 + 4/rho^2), and the
    convolution of the GPU's own map equals the oracle's bit for bit."""
    f = W.Field(xy=np.zeros((1, 2)), m=np.ones(1), kappa_c=0.0, gamma1=0.0, gamma2=0.0)
    rays = W.Grid(-3.0, 3.0, -3.0, 3.0, 4096, 4096)
    src = W.Grid(-1.0, 1.0, -1.0, 1.0, 101, 101)
    c, _, _ = shoot_gpu(f, rays, src, want_beta=False)
    scale = M.mlens_magnification_scale(rays, src)
    rho = 0.5
    conv = torch.empty(src.n, dtype=torch.float32, device="cuda")
    M.mlens_convolve(_dev_counts(c), src, M.MLENS_PROFILE_DISK, rho, conv, scale=scale)
    ref = LC.convolve(c, src, LC.DISK, rho, scale).astype(np.float32)
    assert np.array_equal(conv.cpu().numpy().view(np.uint32), ref.reshape(-1).view(np.uint32))
    lc = torch.empty(201, dtype=torch.float32, device="cuda")
    M.mlens_light_curve(conv, src, (-0.5, 0.0), (0.5, 0.0), 201, lc)
    lc = lc.cpu().numpy()
    assert lc[100] == pytest.approx(math.sqrt(1 + 4 / rho ** 2), rel=0.01)
    assert np.all(lc[:100] <= lc[100] * 1.001) and np.all(lc[101:] <= lc[100] * 1.001)  # peak on the lens


def test_arguments_rejected():
    src = W.Grid(0.0, 1.0, 0.0, 1.0, 8, 8)
    c = torch.zeros(64, dtype=torch.int32, device="cuda")
    o = torch.empty(64, dtype=torch.float32, device="cuda")
    for prof, size in ((M.MLENS_PROFILE_GAUSSIAN, 0.0), (M.MLENS_PROFILE_GAUSSIAN, 100.0), (7, 0.1),
                       (M.MLENS_PROFILE_DISK, -1.0), (M.MLENS_PROFILE_DISK, float("nan"))):
        with pytest.raises(M.MlensError) as ei:
            M.mlens_convolve(c, src, prof, size, o)
        assert ei.value.code == M.MLENS_ERR_ARG, (prof, size)
    with pytest.raises(M.MlensError):
        M.mlens_convolve(c, src, M.MLENS_PROFILE_DISK, 0.1, c.view(torch.float32))  # out overlaps counts
    with pytest.raises(M.MlensError):
        M.mlens_light_curve(o, src, (0, 0), (1, 1), 0, o)


@pytest.mark.parametrize("profile,size", [(M.MLENS_PROFILE_GAUSSIAN, 0.04), (M.MLENS_PROFILE_DISK, 0.07)])
def test_workspace_call_is_asynchronous_and_graph_capturable(profile, size):
    """With a caller workspace nothing is allocated: the call can be captured in a CUDA
    graph; replays give the library-allocated call's map bit for bit."""
    rng = np.random.default_rng(12)
    src = W.Grid(-3.0, 3.0, -2.0, 2.0, 777, 555)
    c = rng.poisson(25.0, (src.ny, src.nx)).astype(np.uint32)
    ref = _gpu_conv(c, src, profile, size, 0.5)
    nb = M.mlens_convolve_workspace(src, profile, size)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    cd = _dev_counts(c)
    out = torch.full((src.n,), -1.0, dtype=torch.float32, device="cuda")
    before = M.mlens_device_memory_in_use()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        M.mlens_convolve(cd, src, profile, size, out, scale=0.5, work=work)  # warm-up on a side stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().reshape(src.ny, src.nx).view(np.uint32), ref.view(np.uint32))
    g = torch.cuda.CUDAGraph()
    out.fill_(-1.0)
    with torch.cuda.graph(g):
        M.mlens_convolve(cd, src, profile, size, out, scale=0.5, work=work)
    for _ in range(2):
        out.fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().reshape(src.ny, src.nx).view(np.uint32), ref.view(np.uint32))
    assert M.mlens_device_memory_in_use() == before
    with pytest.raises(M.MlensError):
        M.mlens_convolve(cd, src, profile, size, out, work=work[: nb // 2])
