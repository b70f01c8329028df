"""GPU calibration loss and adjoint (FP32) against the FP64 CPU oracle and
central finite differences of the FP64 loss.

Tolerances: the gradient within 1e-4 relative (max-norm) of the FP64
gradient, the stated target; the loss within 1e-5 relative, from FP32
(eps = 6e-8) Kahan-compensated sums with fixed-order trees."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mw(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return mwax_lib


def problem(N, C, seed, noise=0.05, gain_err=0.05):
    """Point-source-like model M, true gains, V = g g^H M + noise, and a
    perturbed gain estimate to evaluate at."""
    rng = np.random.default_rng(seed)
    B = N * (N + 1) // 2
    ii, jj = np.tril_indices(N)
    n_src = 20
    flux = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_src))
    phase_rate = rng.uniform(0, 2 * np.pi, (N, n_src))
    nu = 1.0 + 0.002 * np.arange(C)
    ph = phase_rate[None] * nu[:, None, None]  # [C, N, S]
    M = np.einsum("s,csb->cb", flux, np.exp(1j * (ph[:, ii, :] - ph[:, jj, :])).transpose(0, 2, 1))
    g_true = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))
    V = g_true[ii] * np.conj(g_true[jj]) * M
    V = V + noise * np.abs(M).mean() * (rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B)))
    g = g_true * (1 + gain_err * (rng.standard_normal(N) + 1j * rng.standard_normal(N)))
    return (np.ascontiguousarray(V, np.complex64), np.ascontiguousarray(M, np.complex64),
            np.ascontiguousarray(g, np.complex64))


def gpu_loss_grad(mw, V, M, g):
    import torch

    Vd = torch.from_numpy(V).cuda()
    Md = torch.from_numpy(M).cuda()
    gd = torch.from_numpy(g).cuda()
    loss, grad = mw.calib_loss_grad(Vd, Md, gd)
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy()


def check(V, M, g, loss, grad):
    V64, M64, g64 = V.astype(np.complex128), M.astype(np.complex128), g.astype(np.complex128)
    L64 = oracle.calib_loss(V64, M64, g64)
    G64 = oracle.calib_grad(V64, M64, g64)
    assert abs(loss - L64) / L64 <= 1e-5, (loss, L64)
    assert np.abs(grad - G64).max() / np.abs(G64).max() <= 1e-4
    return L64, G64


@pytest.mark.parametrize("N,C", [(2, 1), (33, 3), (70, 5), (130, 9)])
def test_calib_small(mw, N, C):
    V, M, g = problem(N, C, seed=N + C)
    loss, grad = gpu_loss_grad(mw, V, M, g)
    check(V, M, g, loss, grad)


def test_calib_deterministic(mw):
    V, M, g = problem(100, 12, seed=5)
    a = gpu_loss_grad(mw, V, M, g)
    b = gpu_loss_grad(mw, V, M, g)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_calib_autograd_function(mw):
    import torch

    V, M, g = problem(64, 4, seed=8)
    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    L = mw.calib_loss(gt, torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda())
    (3.0 * L).backward()
    G64 = oracle.calib_grad(V.astype(np.complex128), M.astype(np.complex128), g.astype(np.complex128))
    got = gt.grad.cpu().numpy()
    assert np.abs(got - 3.0 * G64).max() / np.abs(3.0 * G64).max() <= 1e-4
    # differentiable in g only: V or M asking for a gradient is refused, not dropped
    Vt = torch.from_numpy(V).cuda().requires_grad_(True)
    with pytest.raises(ValueError):
        mw.calib_loss(gt, Vt, torch.from_numpy(M).cuda())
    Mt = torch.from_numpy(M).cuda().requires_grad_(True)
    with pytest.raises(ValueError):
        mw.calib_loss(gt, torch.from_numpy(V).cuda(), Mt)


def test_calib_central_differences(mw):
    """GPU FP32 gradient against central differences (h = 1e-3) of the FP64
    loss: 32 seeded coordinates and 8 random directions."""
    N, C = 96, 16
    V, M, g = problem(N, C, seed=17)
    _, grad = gpu_loss_grad(mw, V, M, g)
    V64, M64, g64 = V.astype(np.complex128), M.astype(np.complex128), g.astype(np.complex128)
    h = 1e-3
    rng = np.random.default_rng(3)
    scale = np.abs(grad).max()
    for k in rng.choice(N, 16, replace=False):
        for unit in (1.0, 1j):
            gp, gm = g64.copy(), g64.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            fd = (oracle.calib_loss(V64, M64, gp) - oracle.calib_loss(V64, M64, gm)) / (2 * h)
            an = grad[k].real if unit == 1.0 else grad[k].imag
            assert abs(fd - an) <= 1e-4 * scale + 1e-3 * abs(fd)
    for _ in range(8):
        d = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        d /= np.linalg.norm(d)
        fd = (oracle.calib_loss(V64, M64, g64 + h * d) - oracle.calib_loss(V64, M64, g64 - h * d)) / (2 * h)
        an = float(np.sum(grad.real * d.real + grad.imag * d.imag))
        assert abs(fd - an) <= 1e-4 * np.abs(grad).sum() * 0.1 + 1e-3 * abs(fd)


def big_problem(N, C, seed, noise=0.05, gain_err=0.05):
    """Same structure with an unstructured complex Gaussian model (the parity
    of the loss does not depend on M's sky structure), built in float32 to
    bound host memory."""
    rng = np.random.default_rng(seed)
    B = N * (N + 1) // 2
    ii, jj = np.tril_indices(N)
    g_true = (rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))).astype(np.complex64)
    G = (g_true[ii] * np.conj(g_true[jj])).astype(np.complex64)
    M = np.empty((C, B), np.complex64)
    V = np.empty((C, B), np.complex64)
    for c in range(C):
        M[c].real = rng.standard_normal(B, dtype=np.float32)
        M[c].imag = rng.standard_normal(B, dtype=np.float32)
        V[c] = G * M[c]
        V[c].real += noise * rng.standard_normal(B, dtype=np.float32)
        V[c].imag += noise * rng.standard_normal(B, dtype=np.float32)
    g = (g_true * (1 + gain_err * (rng.standard_normal(N) + 1j * rng.standard_normal(N)))).astype(np.complex64)
    return V, M, g


def test_calib_full_size(mw):
    """1024 inputs x 768 channels (524,800 baselines per channel)."""
    V, M, g = big_problem(1024, 768, seed=4)
    loss, grad = gpu_loss_grad(mw, V, M, g)
    check(V, M, g, loss, grad)


# ---------------------------------------------------------------------------
# gain solve (alternating least-squares sweeps)
# ---------------------------------------------------------------------------
def gpu_solve(mw, V, M, g0, n_iter):
    import torch

    g, hist = mw.calib_solve(torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda(),
                             torch.from_numpy(g0).cuda(), n_iter)
    torch.cuda.synchronize()
    return g.cpu().numpy(), (hist.cpu().numpy() if hist is not None else None)


def check_solve(V, M, g0, n_iter, g_gpu, hist, tol_g):
    """Iterates within tol_g (max-norm, relative to max |g|) of the FP64
    oracle's from the same start; the first loss within 1e-5 (the FP32 loss
    tolerance), later ones within 1e-4 (they are losses of slightly different
    iterates, and near a minimum the loss is flat in the gains)."""
    V64, M64, g064 = V.astype(np.complex128), M.astype(np.complex128), g0.astype(np.complex128)
    g64, l64 = oracle.calib_solve(V64, M64, g064, n_iter)
    assert np.abs(g_gpu - g64).max() <= tol_g * np.abs(g64).max(), np.abs(g_gpu - g64).max()
    assert hist.shape == (n_iter,)
    assert abs(hist[0] - l64[0]) <= 1e-5 * l64[0]
    np.testing.assert_allclose(hist, l64, rtol=1e-4)
    return g64, l64


@pytest.mark.parametrize("N,C,n_iter", [(2, 1, 1), (33, 3, 1), (33, 3, 2), (70, 5, 5), (130, 9, 4)])
def test_solve_small(mw, N, C, n_iter):
    V, M, g0 = problem(N, C, seed=100 + N + C)
    g, hist = gpu_solve(mw, V, M, g0, n_iter)
    check_solve(V, M, g0, n_iter, g, hist, tol_g=1e-4)


def test_solve_zero_sweeps_leaves_gains(mw):
    V, M, g0 = problem(40, 2, seed=9)
    g, hist = gpu_solve(mw, V, M, g0, 0)
    np.testing.assert_array_equal(g, g0)
    assert hist.shape == (0,)


def test_solve_deterministic(mw):
    V, M, g0 = problem(100, 6, seed=10)
    a = gpu_solve(mw, V, M, g0, 3)
    b = gpu_solve(mw, V, M, g0, 3)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_solve_recovers_true_gains(mw):
    """Noise-free data in float32: the gains come back to FP32 accuracy up to
    one global phase, and the loss falls by many orders of magnitude."""
    rng = np.random.default_rng(11)
    N, C = 64, 8
    B = N * (N + 1) // 2
    ii, jj = np.tril_indices(N)
    M = (rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))).astype(np.complex64)
    g_true = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))
    V = (g_true[ii] * np.conj(g_true[jj]) * M).astype(np.complex64)
    g0 = (g_true * (1 + 0.2 * (rng.standard_normal(N) + 1j * rng.standard_normal(N)))).astype(np.complex64)
    g, hist = gpu_solve(mw, V, M, g0, 40)
    ph = np.vdot(g, g_true)
    err = np.abs(g * ph / abs(ph) - g_true).max() / np.abs(g_true).max()
    assert err <= 2e-5, err
    assert hist[-1] <= 1e-8 * hist[0]


def test_solve_full_size(mw):
    """1024 inputs x 768 channels: two sweeps against the FP64 oracle."""
    V, M, g0 = big_problem(1024, 768, seed=12)
    g, hist = gpu_solve(mw, V, M, g0, 2)
    check_solve(V, M, g0, 2, g, hist, tol_g=1e-4)


# ---------------------------------------------------------------------------
# per-channel gains g_k(nu)
# ---------------------------------------------------------------------------
def problem_chan(N, C, seed, noise=0.05, gain_err=0.05):
    """Point-source-like model, gains that change across the band, and a
    perturbed per-channel estimate G [C, N]."""
    V, M, _ = problem(N, C, seed, noise=0.0)
    rng = np.random.default_rng(seed + 1000)
    ii, jj = np.tril_indices(N)
    G_true = rng.uniform(0.8, 1.2, (C, N)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, N)))
    Vc = G_true[:, ii] * np.conj(G_true[:, jj]) * M.astype(np.complex128)
    Vc = Vc + noise * np.abs(M).mean() * (rng.standard_normal(Vc.shape) + 1j * rng.standard_normal(Vc.shape))
    G = G_true * (1 + gain_err * (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N))))
    return (np.ascontiguousarray(Vc, np.complex64), M,
            np.ascontiguousarray(G, np.complex64), G_true)


def gpu_chan_loss_grad(mw, V, M, G):
    import torch

    loss, grad = mw.calib_chan_loss_grad(torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda(),
                                         torch.from_numpy(G).cuda())
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy()


def check_chan(V, M, G, loss, grad, chans=None):
    """Loss within 1e-5 relative of the FP64 oracle (all channels); gradient
    within 1e-4 (max-norm, relative) on the channels checked."""
    chans = range(V.shape[0]) if chans is None else chans
    L64 = sum(oracle.calib_chan_loss(V[c:c + 1].astype(np.complex128), M[c:c + 1].astype(np.complex128),
                                     G[c:c + 1].astype(np.complex128)) for c in range(V.shape[0]))
    assert abs(loss - L64) / L64 <= 1e-5, (loss, L64)
    for c in chans:
        G64 = oracle.calib_chan_grad(V[c:c + 1].astype(np.complex128),
                                     M[c:c + 1].astype(np.complex128),
                                     G[c:c + 1].astype(np.complex128))[0]
        assert np.abs(grad[c] - G64).max() / np.abs(G64).max() <= 1e-4, c


@pytest.mark.parametrize("N,C", [(2, 1), (33, 3), (70, 9), (130, 17), (257, 8)])
def test_calib_chan_small(mw, N, C):
    """Ragged tiles (N not a multiple of 32) and channel counts that leave
    warps of the last CTA without a channel."""
    V, M, G, _ = problem_chan(N, C, seed=200 + N + C)
    loss, grad = gpu_chan_loss_grad(mw, V, M, G)
    check_chan(V, M, G, loss, grad)


def test_calib_chan_deterministic(mw):
    V, M, G, _ = problem_chan(100, 12, seed=6)
    a = gpu_chan_loss_grad(mw, V, M, G)
    b = gpu_chan_loss_grad(mw, V, M, G)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_calib_chan_autograd_function(mw):
    """calib_loss with [n_chan, N] gains takes the per-channel path."""
    import torch

    V, M, G, _ = problem_chan(48, 5, seed=7)
    gt = torch.from_numpy(G).cuda().requires_grad_(True)
    L = mw.calib_loss(gt, torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda())
    (2.0 * L).backward()
    G64 = oracle.calib_chan_grad(V.astype(np.complex128), M.astype(np.complex128), G.astype(np.complex128))
    got = gt.grad.cpu().numpy()
    assert got.shape == G.shape
    assert np.abs(got - 2.0 * G64).max() / np.abs(2.0 * G64).max() <= 1e-4


def test_calib_chan_shared_gains_match_the_per_input_kernel(mw):
    """The same gains in every channel: the per-channel loss equals the
    frequency-independent kernel's, and the channel sum of the per-channel
    gradient equals its gradient (two different kernels, same mathematics)."""
    V, M, g = problem(90, 7, seed=12)
    G = np.ascontiguousarray(np.tile(g, (7, 1)))
    lc, gc = gpu_chan_loss_grad(mw, V, M, G)
    l1, g1 = gpu_loss_grad(mw, V, M, g)
    assert abs(lc - l1) <= 1e-5 * l1
    assert np.abs(gc.sum(0) - g1).max() <= 1e-4 * np.abs(g1).max()


def test_calib_chan_full_size(mw):
    """1024 inputs x 768 channels: the loss over every channel, the gradient
    on 12 seeded channels including the first and last."""
    V, M, g = big_problem(1024, 768, seed=14)
    rng = np.random.default_rng(15)
    G = (g[None, :] * (1 + 0.02 * (rng.standard_normal((768, 1024)) + 1j * rng.standard_normal((768, 1024))))).astype(np.complex64)
    loss, grad = gpu_chan_loss_grad(mw, V, M, G)
    chans = sorted({0, 767, *rng.choice(768, 10, replace=False).tolist()})
    check_chan(V, M, G, loss, grad, chans)


def gpu_chan_solve(mw, V, M, G0, n_iter):
    import torch

    G, hist = mw.calib_chan_solve(torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda(),
                                  torch.from_numpy(G0).cuda(), n_iter)
    torch.cuda.synchronize()
    return G.cpu().numpy(), hist.cpu().numpy()


@pytest.mark.parametrize("N,C,n_iter", [(2, 1, 1), (33, 3, 2), (70, 9, 5), (130, 5, 4)])
def test_calib_chan_solve_small(mw, N, C, n_iter):
    V, M, G0, _ = problem_chan(N, C, seed=300 + N + C)
    G, hist = gpu_chan_solve(mw, V, M, G0, n_iter)
    G64, l64 = oracle.calib_chan_solve(V.astype(np.complex128), M.astype(np.complex128),
                                       G0.astype(np.complex128), n_iter)
    assert np.abs(G - G64).max() <= 1e-4 * np.abs(G64).max()
    assert hist.shape == (n_iter,)
    assert abs(hist[0] - l64[0]) <= 1e-5 * l64[0]
    np.testing.assert_allclose(hist, l64, rtol=1e-4)


def test_calib_chan_solve_recovers_band_dependent_gains(mw):
    """Noise-free data with gains that change across the band: every channel
    comes back to FP32 accuracy up to its own global phase."""
    V, M, G0, G_true = problem_chan(64, 6, seed=21, noise=0.0, gain_err=0.2)
    G, hist = gpu_chan_solve(mw, V, M, G0, 40)
    for c in range(6):
        ph = np.vdot(G[c], G_true[c])
        err = np.abs(G[c] * ph / abs(ph) - G_true[c]).max() / np.abs(G_true).max()
        assert err <= 2e-5, (c, err)
    assert hist[-1] <= 1e-8 * hist[0]


def test_calib_chan_rejects_bad_shapes(mw):
    import torch

    V, M, G, _ = problem_chan(20, 3, seed=2)
    Vd, Md = torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda()
    with pytest.raises(ValueError):
        mw.calib_chan_loss_grad(Vd, Md, torch.from_numpy(G[:2]).cuda())
    with pytest.raises(ValueError):
        mw.calib_chan_loss_grad(Vd, Md, torch.from_numpy(G[0]).cuda())
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    # host pointers are refused before any launch
    assert mw.lib().mwax_calib_chan_loss_grad(V.ctypes.data, M.ctypes.data, G.ctypes.data, 20, 3,
                                              ws.data_ptr(), ws.data_ptr(), None, None) != 0


# ---------------------------------------------------------------------------
# full 2x2 Jones matrices per tile
# ---------------------------------------------------------------------------
def rand_jones(rng, n_tiles, leak=0.2):
    d = rng.uniform(0.8, 1.2, (n_tiles, 2)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (n_tiles, 2)))
    J = np.zeros((n_tiles, 2, 2), complex)
    J[:, 0, 0], J[:, 1, 1] = d[:, 0], d[:, 1]
    J[:, 0, 1] = leak * (rng.standard_normal(n_tiles) + 1j * rng.standard_normal(n_tiles))
    J[:, 1, 0] = leak * (rng.standard_normal(n_tiles) + 1j * rng.standard_normal(n_tiles))
    return J


def problem_jones(n_tiles, C, seed, noise=0.05, err=0.05):
    """Point-source-like model, data from leaky Jones matrices plus noise, and
    a perturbed estimate."""
    N = 2 * n_tiles
    _, M, _ = problem(N, C, seed, noise=0.0)
    rng = np.random.default_rng(seed + 2000)
    J_true = rand_jones(rng, n_tiles)
    a, b, idx = oracle._jones_blocks(n_tiles)
    Mc = M.astype(np.complex128)
    V = rng.standard_normal(Mc.shape) + 1j * rng.standard_normal(Mc.shape)  # autos, intra-tile: ignored
    V *= noise * np.abs(M).mean()
    for c in range(C):
        V[c][idx] += J_true[a] @ Mc[c][idx] @ np.conj(np.swapaxes(J_true[b], -1, -2))
    J = J_true + err * (rng.standard_normal(J_true.shape) + 1j * rng.standard_normal(J_true.shape))
    return (np.ascontiguousarray(V, np.complex64), M, np.ascontiguousarray(J, np.complex64), J_true)


def gpu_jones_loss_grad(mw, V, M, J):
    import torch

    loss, grad = mw.calib_jones_loss_grad(torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda(),
                                          torch.from_numpy(J).cuda())
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy()


def check_jones(V, M, J, loss, grad):
    V64, M64, J64 = V.astype(np.complex128), M.astype(np.complex128), J.astype(np.complex128)
    L64 = oracle.calib_jones_loss(V64, M64, J64)
    G64 = oracle.calib_jones_grad(V64, M64, J64)
    assert abs(loss - L64) <= 1e-5 * L64, (loss, L64)
    assert np.abs(grad - G64).max() <= 1e-4 * np.abs(G64).max()


@pytest.mark.parametrize("n_tiles,C", [(1, 2), (2, 1), (17, 3), (40, 5), (65, 9), (33, 25)])
def test_calib_jones_small(mw, n_tiles, C):
    """Ragged calibration tiles (tile counts not a multiple of 32), channel
    counts above and below the 12 channel groups, one tile (no pairs)."""
    V, M, J, _ = problem_jones(n_tiles, C, seed=400 + n_tiles + C)
    loss, grad = gpu_jones_loss_grad(mw, V, M, J)
    if n_tiles == 1:
        assert loss == 0.0 and np.all(grad == 0)
        return
    check_jones(V, M, J, loss, grad)


def test_calib_jones_deterministic(mw):
    V, M, J, _ = problem_jones(50, 6, seed=8)
    a = gpu_jones_loss_grad(mw, V, M, J)
    b = gpu_jones_loss_grad(mw, V, M, J)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_calib_jones_diagonal_matches_per_input_kernel(mw):
    """Diagonal Jones with the intra-tile pairs zeroed: the loss and the
    diagonal of the gradient equal the per-input kernel's (two kernels, the
    same mathematics)."""
    n_tiles, C = 45, 4
    V, M, g = problem(2 * n_tiles, C, seed=13)
    for a in range(n_tiles):
        V[:, oracle.baseline_index(2 * a + 1, 2 * a)] = 0
        M[:, oracle.baseline_index(2 * a + 1, 2 * a)] = 0
    J = np.zeros((n_tiles, 2, 2), np.complex64)
    J[:, 0, 0], J[:, 1, 1] = g[0::2], g[1::2]
    lj, gj = gpu_jones_loss_grad(mw, V, M, J)
    l1, g1 = gpu_loss_grad(mw, V, M, g)
    assert abs(lj - l1) <= 1e-5 * l1
    scale = np.abs(g1).max()
    assert np.abs(gj[:, 0, 0] - g1[0::2]).max() <= 1e-4 * scale
    assert np.abs(gj[:, 1, 1] - g1[1::2]).max() <= 1e-4 * scale


def gpu_jones_solve(mw, V, M, J0, n_iter):
    import torch

    J, hist = mw.calib_jones_solve(torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda(),
                                   torch.from_numpy(J0).cuda(), n_iter)
    torch.cuda.synchronize()
    return J.cpu().numpy(), hist.cpu().numpy()


@pytest.mark.parametrize("n_tiles,C,n_iter", [(2, 1, 1), (17, 3, 2), (40, 5, 5)])
def test_calib_jones_solve_small(mw, n_tiles, C, n_iter):
    V, M, J0, _ = problem_jones(n_tiles, C, seed=500 + n_tiles + C)
    J, hist = gpu_jones_solve(mw, V, M, J0, n_iter)
    J64, l64 = oracle.calib_jones_solve(V.astype(np.complex128), M.astype(np.complex128),
                                        J0.astype(np.complex128), n_iter)
    assert np.abs(J - J64).max() <= 1e-4 * np.abs(J64).max()
    assert abs(hist[0] - l64[0]) <= 1e-5 * l64[0]
    np.testing.assert_allclose(hist, l64, rtol=1e-4)


def test_calib_jones_solve_recovers_leaky_jones(mw):
    """Noise-free data: the Jones matrices come back to FP32 accuracy up to
    one global phase."""
    V, M, J0, J_true = problem_jones(32, 6, seed=22, noise=0.0, err=0.1)
    J, hist = gpu_jones_solve(mw, V, M, J0, 60)
    ph = np.vdot(J.ravel(), J_true.ravel())
    err = np.abs(J * ph / abs(ph) - J_true).max() / np.abs(J_true).max()
    assert err <= 2e-5, err
    assert hist[-1] <= 1e-8 * hist[0]


def test_calib_jones_full_size(mw):
    """1024 inputs (512 tiles) x 96 channels against the FP64 oracle."""
    V, M, g = big_problem(1024, 96, seed=16)
    rng = np.random.default_rng(17)
    J = rand_jones(rng, 512).astype(np.complex64)
    loss, grad = gpu_jones_loss_grad(mw, V, M, J)
    check_jones(V, M, J, loss, grad)


def test_calib_jones_rejects_bad_shapes(mw):
    import torch

    V, M, J, _ = problem_jones(5, 2, seed=3)
    Vd, Md = torch.from_numpy(V).cuda(), torch.from_numpy(M).cuda()
    with pytest.raises(ValueError):
        mw.calib_jones_loss_grad(Vd, Md, torch.from_numpy(J[:4]).cuda())
    assert mw.lib().mwax_calib_jones_workspace_bytes(11, 2) == -1  # odd input count


# ---------------------------------------------------------------------------
# the c4 workload end to end: correlator output -> FP32 V -> calibration
# ---------------------------------------------------------------------------
def test_c4_workload_parity_sampled(mw):
    """The configured data path at full size (1024 inputs x 768 channels,
    T = 10000, 8-bit voltages carrying 20 point sources through true gains):
    the library correlates all channels; on 8 sampled channels (first, last,
    six seeded) its int32 visibilities equal the oracle's correlation of the
    same seeded voltages, both sides form the FP32 V = vis / (2 T scale^2)
    identically, and the GPU loss, gradient, one gain-solve sweep, per-channel
    loss and gradient and the Jones loss and gradient agree with the FP64
    oracle on those channels (loss 1e-5, gradient and iterates 1e-4
    relative); the gradient also matches central differences (h = 1e-3) of
    the FP64 loss on a few coordinates."""
    import torch

    import synth

    spec = synth.spec_c4()
    N, C, T = spec.n_inputs, spec.n_chan, spec.n_time
    B = N * (N + 1) // 2
    rng = np.random.default_rng(44)
    sub = sorted({0, C - 1, *rng.choice(np.arange(1, C - 1), 6, replace=False).tolist()})
    # GPU: every channel of the workload
    vol = torch.empty(C * T * N * 2, dtype=torch.uint8, device="cuda")
    synth.fill_device(spec, vol)
    plan = mw.Plan(N, C, T, 8)
    vis = plan.correlate(vol)
    assert plan.status() == 0
    plan.close()
    del vol
    subd = torch.tensor(sub, device="cuda")
    vis_s = vis.index_select(0, subd)
    del vis
    scale2 = np.float32(2.0 * spec.meta["scale"] ** 2 * T)
    # a CUDA 0-d divisor: element-wise IEEE division (torch turns a Python-scalar
    # divisor into a multiply by its reciprocal, which can differ by one ulp)
    sdev = torch.tensor(scale2, dtype=torch.float32, device="cuda")
    V_gpu = torch.complex(vis_s[..., 0].float() / sdev, vis_s[..., 1].float() / sdev)
    # oracle: the same channels correlated from the host copy of the voltages
    vis64 = oracle.correlate(synth.fill_host(spec, chans=sub), 8, N, len(sub), T)
    np.testing.assert_array_equal(vis_s.cpu().numpy(), vis64)
    V_host = (vis64[..., 0].astype(np.float32) / scale2
              + 1j * (vis64[..., 1].astype(np.float32) / scale2)).astype(np.complex64)
    assert np.array_equal(V_gpu.cpu().numpy().view(np.uint32), V_host.view(np.uint32))
    M_host = synth.model_visibilities_host(spec, sub).astype(np.complex64)
    M_gpu = torch.from_numpy(M_host).cuda()
    g_true = np.asarray(spec.gains, np.complex128)
    g = (g_true * (1 + 0.05 * (rng.standard_normal(N) + 1j * rng.standard_normal(N)))).astype(np.complex64)
    V64, M64, g64 = V_host.astype(np.complex128), M_host.astype(np.complex128), g.astype(np.complex128)
    # loss and gradient
    loss, grad = mw.calib_loss_grad(V_gpu, M_gpu, torch.from_numpy(g).cuda())
    L64 = oracle.calib_loss(V64, M64, g64)
    G64 = oracle.calib_grad(V64, M64, g64)
    assert abs(float(loss) - L64) <= 1e-5 * L64, (float(loss), L64)
    gg = grad.cpu().numpy()
    assert np.abs(gg - G64).max() <= 1e-4 * np.abs(G64).max()
    # central differences of the FP64 loss (h = 1e-3) on seeded coordinates
    h = 1e-3
    for k in rng.choice(N, 4, replace=False):
        for unit in (1.0, 1j):
            gp, gm = g64.copy(), g64.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            fd = (oracle.calib_loss(V64, M64, gp) - oracle.calib_loss(V64, M64, gm)) / (2 * h)
            an = gg[k].real if unit == 1.0 else gg[k].imag
            assert abs(an - fd) <= 1e-4 * np.abs(G64).max() + 1e-3 * abs(fd), (k, unit, an, fd)
    # one gain-solve sweep
    gs, hist = mw.calib_solve(V_gpu, M_gpu, torch.from_numpy(g).cuda(), 1)
    gs64, h64 = oracle.calib_solve(V64, M64, g64, 1)
    assert np.abs(gs.cpu().numpy() - gs64).max() <= 1e-4 * np.abs(gs64).max()
    assert abs(float(hist[0]) - h64[0]) <= 1e-5 * h64[0]
    # per-channel gains
    G = (g[None, :] * (1 + 0.02 * (rng.standard_normal((len(sub), N))
                                   + 1j * rng.standard_normal((len(sub), N))))).astype(np.complex64)
    lc, gc = mw.calib_chan_loss_grad(V_gpu, M_gpu, torch.from_numpy(G).cuda())
    Lc64 = oracle.calib_chan_loss(V64, M64, G.astype(np.complex128))
    Gc64 = oracle.calib_chan_grad(V64, M64, G.astype(np.complex128))
    assert abs(float(lc) - Lc64) <= 1e-5 * Lc64
    gcn = gc.cpu().numpy()
    for c in range(len(sub)):
        assert np.abs(gcn[c] - Gc64[c]).max() <= 1e-4 * np.abs(Gc64[c]).max(), c
    # 2x2 Jones matrices: diagonal gains plus 5 % leakage
    n_t = N // 2
    J = np.zeros((n_t, 2, 2), np.complex64)
    J[:, 0, 0], J[:, 1, 1] = g[0::2], g[1::2]
    J[:, 0, 1] = 0.05 * (rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t))
    J[:, 1, 0] = 0.05 * (rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t))
    lj, gj = mw.calib_jones_loss_grad(V_gpu, M_gpu, torch.from_numpy(J).cuda())
    Lj64 = oracle.calib_jones_loss(V64, M64, J.astype(np.complex128))
    Gj64 = oracle.calib_jones_grad(V64, M64, J.astype(np.complex128))
    assert abs(float(lj) - Lj64) <= 1e-5 * Lj64
    assert np.abs(gj.cpu().numpy() - Gj64).max() <= 1e-4 * np.abs(Gj64).max()
    torch.cuda.synchronize()
