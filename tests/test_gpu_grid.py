"""GPU gridding against the FP64 CPU oracle.

Tolerance: the weights are computed in FP64 and rounded to FP32 (6e-8
relative) and each cell is an FP32 sum of up to a few hundred terms (~K x
6e-8 relative to the largest term), so every cell is compared within 1e-5 of
the largest |G|.
Inputs are seeded int32 visibilities generated on the host (the gridding
does not care whether they came from the correlator) and seeded tile
positions."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

C_LIGHT = 299792458.0


@pytest.fixture(scope="module")
def mw(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return mwax_lib


def problem(seed, n_tiles, n_chan, Ng, du, f0=150e6, df=1e6, vmax=3000, spill=0.7):
    rng = np.random.default_rng(seed)
    N = 2 * n_tiles
    B = N * (N + 1) // 2
    reach = 0.5 * Ng * du * C_LIGHT / (f0 + (n_chan - 1) * df) / 2
    tile_xy = rng.uniform(-reach, reach, (n_tiles, 2)) * spill
    vis = rng.integers(-vmax, vmax + 1, (n_chan, B, 2)).astype(np.int32)
    return tile_xy, vis, f0, df


def gpu_grid(mw, tile_xy, vis, f0, df, Ng, du, W, sigma):
    import torch

    gp = mw.GridPlan(tile_xy, vis.shape[0], f0, df, Ng, du, W, sigma)
    g = gp.grid(torch.from_numpy(vis).cuda())
    torch.cuda.synchronize()
    out = g.cpu().numpy()
    n = gp.n_points
    gp.close()
    return out, n


def close(got, ref):
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= 1e-5 * scale, (err, scale)


@pytest.mark.parametrize("n_tiles,n_chan,Ng,du,W,sigma,spill", [
    (2, 1, 16, 1.0, 7, 1.0, 0.7),
    (5, 3, 64, 1.5, 7, 1.0, 0.7),
    (8, 6, 128, 2.0, 5, 0.8, 0.9),
    (12, 4, 96, 1.0, 7, 1.3, 1.6),   # points beyond the edge: partial supports dropped
    (7, 9, 200, 0.75, 9, 1.5, 0.8),
])
def test_grid_small(mw, n_tiles, n_chan, Ng, du, W, sigma, spill):
    tile_xy, vis, f0, df = problem(n_tiles * 100 + n_chan, n_tiles, n_chan, Ng, du, spill=spill)
    got, n = gpu_grid(mw, tile_xy, vis, f0, df, Ng, du, W, sigma)
    ref = oracle.grid(tile_xy, vis, f0, df, Ng, du, W, sigma)
    close(got, ref)
    assert 0 < n <= n_tiles * (n_tiles - 1) * n_chan


def test_grid_deterministic(mw):
    tile_xy, vis, f0, df = problem(5, 10, 8, 128, 1.0)
    a, _ = gpu_grid(mw, tile_xy, vis, f0, df, 128, 1.0, 7, 1.0)
    b, _ = gpu_grid(mw, tile_xy, vis, f0, df, 128, 1.0, 7, 1.0)
    np.testing.assert_array_equal(a, b)


def test_grid_hermitian_gpu(mw):
    """G[2p+q][Ng-r][Ng-s] = conj(G[2q+p][r][s]) up to FP32 summation order."""
    tile_xy, vis, f0, df = problem(6, 9, 5, 128, 1.0)
    G, _ = gpu_grid(mw, tile_xy, vis, f0, df, 128, 1.0, 7, 1.0)
    close(G[:, :0:-1, :0:-1], np.conj(G[[0, 2, 1, 3], 1:, 1:]))


def test_grid_invalid_args(mw):
    import torch

    gp = mw.GridPlan(np.zeros((3, 2)), 2, 150e6, 1e6, 32, 1.0)
    N = 6
    bad = torch.zeros((2, N * (N + 1) // 2 * 2 + 1), dtype=torch.int32, device="cuda")
    out = gp.empty_grids()
    L = mw.lib()
    assert L.mwax_grid(gp._h, bad.data_ptr() + 4, torch.view_as_real(out).data_ptr()) == 1
    host = torch.zeros(4, dtype=torch.int32)
    assert L.mwax_grid(gp._h, host.data_ptr(), torch.view_as_real(out).data_ptr()) == 1
    gp.close()


def test_grid_full_size_sampled(mw):
    """The gridding workload (128 tiles, 768 channels from 167.04 MHz,
    2048 x 2048 cells of one wavelength) on seeded int32 visibilities of the
    correlator's output shape, checked cell by cell on sampled cells."""
    import torch

    import synth

    geo = synth.grid_geometry_c1()
    n_tiles, n_chan = geo["tile_xy"].shape[0], 768
    rng = np.random.default_rng(77)
    N = 2 * n_tiles
    vis = rng.integers(-2 ** 20, 2 ** 20, (n_chan, N * (N + 1) // 2, 2)).astype(np.int32)
    gp = mw.GridPlan(geo["tile_xy"], n_chan, geo["f0"], geo["df"], geo["Ng"], geo["du"], geo["W"],
                     geo["sigma"])
    G = gp.grid(torch.from_numpy(vis).cuda()).cpu().numpy()
    gp.close()
    Ng = geo["Ng"]
    c = Ng // 2
    cells = [(0, c, c), (3, c, c), (1, c + 3, c - 2), (2, c - 40, c + 77), (0, c + 500, c - 300),
             (3, c - 900, c + 100), (1, 5, 5), (2, Ng - 1, Ng - 1)] + \
            [(int(p), int(r), int(s)) for p, r, s in zip(rng.integers(0, 4, 6),
                                                          rng.integers(c - 600, c + 600, 6),
                                                          rng.integers(c - 600, c + 600, 6))]
    scale = np.abs(G[:, c - 3:c + 4, c - 3:c + 4]).max()
    for pol, r, s in cells:
        ref = oracle.grid_cell(geo["tile_xy"], vis, geo["f0"], geo["df"], Ng, geo["du"], geo["W"],
                               geo["sigma"], pol, r, s)
        assert abs(G[pol, r, s] - ref) <= 1e-5 * max(scale, abs(ref)), (pol, r, s, G[pol, r, s], ref)
    torch.cuda.synchronize()
