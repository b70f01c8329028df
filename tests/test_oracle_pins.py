"""Pins for the CPU oracle: checks against facts fixed by the mathematics of
V_ij = sum_t x_i(t) conj(x_j(t)) (paper Sec. 2: all antenna pairs are
cross-correlated per channel and the products integrated) and of the
least-squares gain loss (Sec. 2: complex gain of each element), never
against the oracle's own formula retyped.

The test packs its own samples (two's complement nibbles / int8 bytes), so a
decoding mistake in the oracle fails the brute-force comparison.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers (test-side encoding, independent of the oracle)
# ---------------------------------------------------------------------------
def pack(re: np.ndarray, im: np.ndarray, bits: int) -> np.ndarray:
    """re, im int arrays [C, T, N] -> packed bytes [C, T, N*bps]."""
    re = np.asarray(re, np.int64)
    im = np.asarray(im, np.int64)
    if bits == 4:
        return ((re & 0xF) | ((im & 0xF) << 4)).astype(np.uint8)
    out = np.empty(re.shape[:-1] + (2 * re.shape[-1],), np.uint8)
    out[..., 0::2] = (re & 0xFF).astype(np.uint8)
    out[..., 1::2] = (im & 0xFF).astype(np.uint8)
    return out


def tri(full: np.ndarray) -> np.ndarray:
    """[C, N, N] complex -> [C, N(N+1)/2, 2] int64 lower triangle, row-major."""
    C, N, _ = full.shape
    ii, jj = np.tril_indices(N)
    v = full[:, ii, jj]
    return np.stack([np.rint(v.real), np.rint(v.imag)], axis=-1).astype(np.int64)


def brute(re, im):
    """Library matmul on complex128 (exact for these small integers)."""
    x = np.asarray(re, np.float64) + 1j * np.asarray(im, np.float64)  # [C, T, N]
    full = np.einsum("cti,ctj->cij", x, np.conj(x))
    return tri(full)


def run_oracle(re, im, bits):
    C, T, N = re.shape
    _, o64 = oracle.correlate(pack(re, im, bits), bits, N, C, T, want64=True)
    return o64


def rand_samples(rng, C, T, N, bits):
    m = 7 if bits == 4 else 127
    return rng.integers(-m, m + 1, (C, T, N)), rng.integers(-m, m + 1, (C, T, N))


# ---------------------------------------------------------------------------
# correlation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bits", [4, 8])
@pytest.mark.parametrize("N,T,C", [(1, 1, 1), (2, 7, 1), (3, 8, 3), (17, 33, 2), (5, 1, 3)])
def test_brute_force(bits, N, T, C):
    rng = np.random.default_rng(1000 * N + 10 * T + C + bits)
    re, im = rand_samples(rng, C, T, N, bits)
    np.testing.assert_array_equal(run_oracle(re, im, bits), brute(re, im))


def test_golden_conjugation_side():
    """Two inputs, one sample: x0 = 1, x1 = i.  V_10 = x1 conj(x0) = i."""
    g = np.loadtxt(os.path.join(GOLDEN, "conj_side.txt"), dtype=np.int64)
    re = np.array([[[1, 0]]])
    im = np.array([[[0, 1]]])
    np.testing.assert_array_equal(run_oracle(re, im, 8)[0], g)
    np.testing.assert_array_equal(run_oracle(re, im, 4)[0], g)


def test_golden_decode():
    """Nibble/byte decoding of hand-written packed values."""
    rows = np.loadtxt(os.path.join(GOLDEN, "decode4.txt"), dtype=np.int64)
    re, im = oracle.decode(rows[:, 0].astype(np.uint8), 4)
    np.testing.assert_array_equal(re, rows[:, 1])
    np.testing.assert_array_equal(im, rows[:, 2])
    rows8 = np.loadtxt(os.path.join(GOLDEN, "decode8.txt"), dtype=np.int64)
    raw = np.stack([rows8[:, 0], rows8[:, 1]], 1).astype(np.uint8).ravel()
    re, im = oracle.decode(raw, 8)
    np.testing.assert_array_equal(re, rows8[:, 2])
    np.testing.assert_array_equal(im, rows8[:, 3])


@pytest.mark.parametrize("bits", [4, 8])
def test_hermitian_by_reversal(bits):
    """Reversing the input order maps V_ij to V_{N-1-j, N-1-i}^* (Hermitian)."""
    rng = np.random.default_rng(7 + bits)
    re, im = rand_samples(rng, 2, 19, 9, bits)
    a = run_oracle(re, im, bits)
    b = run_oracle(re[..., ::-1], im[..., ::-1], bits)
    N = 9
    for i in range(N):
        for j in range(i + 1):
            ba = oracle.baseline_index(i, j)
            bb = oracle.baseline_index(N - 1 - j, N - 1 - i)
            np.testing.assert_array_equal(b[:, bb, 0], a[:, ba, 0])
            np.testing.assert_array_equal(b[:, bb, 1], -a[:, ba, 1])


@pytest.mark.parametrize("bits", [4, 8])
def test_autos_are_power(bits):
    rng = np.random.default_rng(11)
    re, im = rand_samples(rng, 3, 25, 6, bits)
    o = run_oracle(re, im, bits)
    power = (re.astype(np.int64) ** 2 + im.astype(np.int64) ** 2).sum(axis=1)  # [C, N]
    for i in range(6):
        b = oracle.baseline_index(i, i)
        np.testing.assert_array_equal(o[:, b, 1], 0)
        np.testing.assert_array_equal(o[:, b, 0], power[:, i])
        assert (o[:, b, 0] >= 0).all()


@pytest.mark.parametrize("bits", [4, 8])
def test_phase_invariance(bits):
    """x -> -x and x -> i x leave every V_ij unchanged."""
    rng = np.random.default_rng(21)
    re, im = rand_samples(rng, 2, 13, 7, bits)
    a = run_oracle(re, im, bits)
    np.testing.assert_array_equal(run_oracle(-re, -im, bits), a)
    np.testing.assert_array_equal(run_oracle(-im, re, bits), a)  # i*(re + i im) = -im + i re


def test_zero_padding_changes_nothing():
    rng = np.random.default_rng(5)
    re, im = rand_samples(rng, 2, 10, 5, 4)
    a = run_oracle(re, im, 4)
    rp = np.zeros((2, 16, 8), np.int64)
    ip = np.zeros((2, 16, 8), np.int64)
    rp[:, :10, :5] = re
    ip[:, :10, :5] = im
    b = run_oracle(rp, ip, 4)
    for i in range(5):
        for j in range(i + 1):
            np.testing.assert_array_equal(b[:, oracle.baseline_index(i, j)], a[:, oracle.baseline_index(i, j)])
    for i in range(5, 8):
        for j in range(i + 1):
            np.testing.assert_array_equal(b[:, oracle.baseline_index(i, j)], 0)


@pytest.mark.parametrize("T", [1, 2, 5, 64, 1001])
def test_quarter_rate_tone_closed_form(T):
    """x_i(t) = c_i i^t gives V_ij = T c_i conj(c_j) exactly (|i^t| = 1)."""
    rng = np.random.default_rng(T)
    N = 6
    c = rng.integers(-7, 8, (N, 2))
    spec = synth.Spec("q", N, 1, T, 4, seed=0, kind=synth.SYNTH_QUARTER, ci=c)
    v = synth.fill_host(spec)
    o = oracle.correlate(v, 4, N, 1, T)
    cc = c[:, 0] + 1j * c[:, 1]
    for i in range(N):
        for j in range(i + 1):
            e = T * cc[i] * np.conj(cc[j])
            b = oracle.baseline_index(i, j)
            assert o[0, b, 0] == int(e.real) and o[0, b, 1] == int(e.imag)


def test_int32_bound_special_case():
    """All samples (127, 127): V_ii = 32258 T.  T = 66572 is the largest
    integration that fits int32 (2,147,479,576); T = 66573 overflows."""
    T = 66572
    re = np.full((1, T, 2), 127)
    im = np.full((1, T, 2), 127)
    o = oracle.correlate(pack(re, im, 8), 8, 2, 1, T)
    assert o[0, 0, 0] == 2_147_479_576 == 32258 * T
    assert o[0, 1, 0] == 2_147_479_576 and o[0, 1, 1] == 0
    re = np.full((1, T + 1, 1), 127)
    with pytest.raises(OverflowError):
        oracle.correlate(pack(re, re, 8), 8, 1, 1, T + 1)


def test_baseline_helpers():
    assert oracle.n_baselines(512) == 131_328  # ~130,000 baseline pairs (Sec. 2)
    assert oracle.n_baselines(1024) == 524_800
    assert oracle.baseline_index(0, 0) == 0
    assert oracle.baseline_index(3, 1) == 7
    assert oracle.baseline_index(1, 2) == -1
    seen = [oracle.baseline_index(i, j) for i in range(20) for j in range(i + 1)]
    assert seen == list(range(oracle.n_baselines(20)))


# ---------------------------------------------------------------------------
# calibration loss / gradient
# ---------------------------------------------------------------------------
def rand_cal(rng, N, C, scale=1.0):
    B = N * (N + 1) // 2
    V = (rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))) * scale
    M = rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))
    g = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))
    return V, M, g


def test_calib_golden_two_inputs():
    """N = 2, one channel, g = (1, i), M_10 = 1, V_10 = 0: R_10 = i, L = 1,
    grad = (2, 2i) (hand derivation: L = |g0|^2 |g1|^2)."""
    V = np.zeros((1, 3), complex)
    M = np.zeros((1, 3), complex)
    M[0, 1] = 1.0
    g = np.array([1.0, 1j])
    assert oracle.calib_loss(V, M, g) == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(oracle.calib_grad(V, M, g), [2.0, 2j], atol=1e-14)


def test_calib_zero_at_truth():
    rng = np.random.default_rng(3)
    N, C = 9, 4
    _, M, g = rand_cal(rng, N, C)
    ii, jj = np.tril_indices(N)
    V = g[ii] * np.conj(g[jj]) * M
    V[:, ii == jj] = 17.0  # autos carry weight 0
    assert oracle.calib_loss(V, M, g) == pytest.approx(0.0, abs=1e-20)
    np.testing.assert_allclose(oracle.calib_grad(V, M, g), 0.0, atol=1e-12)


def test_calib_against_autograd():
    """Gradient convention pinned by torch autograd on a complex128 loss."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    N, C = 7, 3
    V, M, g = rand_cal(rng, N, C)
    Vf = np.zeros((C, N, N), complex)
    Mf = np.zeros((C, N, N), complex)
    ii, jj = np.tril_indices(N)
    Vf[:, ii, jj] = V
    Mf[:, ii, jj] = M
    gt = torch.tensor(g, dtype=torch.complex128, requires_grad=True)
    Gm = gt[:, None] * torch.conj(gt)[None, :]
    R = Gm[None] * torch.tensor(Mf) - torch.tensor(Vf)
    mask = torch.tril(torch.ones(N, N, dtype=torch.bool), diagonal=-1)
    L = (R.abs() ** 2)[:, mask].sum()
    L.backward()
    assert oracle.calib_loss(V, M, g) == pytest.approx(L.item(), rel=1e-12)
    np.testing.assert_allclose(oracle.calib_grad(V, M, g), gt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_calib_central_differences():
    rng = np.random.default_rng(5)
    N, C = 8, 3
    V, M, g = rand_cal(rng, N, C)
    grad = oracle.calib_grad(V, M, g)
    h = 1e-3
    for k in range(N):
        for part, unit in ((0, 1.0), (1, 1j)):
            gp = g.copy()
            gm = g.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            fd = (oracle.calib_loss(V, M, gp) - oracle.calib_loss(V, M, gm)) / (2 * h)
            an = grad[k].real if part == 0 else grad[k].imag
            assert fd == pytest.approx(an, rel=1e-5, abs=1e-6)


def test_calib_phase_and_radial_identities():
    """L(g e^{i th}) is constant -> sum Im(conj(g_k) grad_k) = 0.
    L(a g) = a^4 A - 2 a^2 B + C (quartic, even) -> d/da at a=1 equals
    Re sum conj(g_k) grad_k, and L(0) = sum_{i>j} |V|^2."""
    rng = np.random.default_rng(6)
    N, C = 10, 2
    V, M, g = rand_cal(rng, N, C)
    grad = oracle.calib_grad(V, M, g)
    s = np.sum(np.conj(g) * grad)
    assert abs(s.imag) <= 1e-10 * np.abs(np.conj(g) * grad).sum()
    L = oracle.calib_loss(V, M, g)
    assert oracle.calib_loss(V, M, g * np.exp(0.7j)) == pytest.approx(L, rel=1e-12)
    alphas = np.array([0.0, 0.5, 0.9, 1.0, 1.3, 2.0])
    Ls = np.array([oracle.calib_loss(V, M, a * g) for a in alphas])
    coef = np.polyfit(alphas, Ls, 4)  # a^4 .. a^0
    assert abs(coef[1]) < 1e-8 * Ls.max() and abs(coef[3]) < 1e-8 * Ls.max()
    np.testing.assert_allclose(np.polyval(coef, alphas), Ls, rtol=1e-10)
    dL = 4 * coef[0] + 2 * coef[2]
    assert s.real == pytest.approx(dL, rel=1e-8)
    ii, jj = np.tril_indices(N)
    assert Ls[0] == pytest.approx(float((np.abs(V[:, ii != jj]) ** 2).sum()), rel=1e-12)


# ---------------------------------------------------------------------------
# gain solve (alternating least squares)
# ---------------------------------------------------------------------------
def full_hermitian(X, N):
    """[C, B] lower triangle -> [C, N, N] with X_ji = conj(X_ij)."""
    C = X.shape[0]
    F = np.zeros((C, N, N), complex)
    ii, jj = np.tril_indices(N)
    F[:, ii, jj] = X
    F[:, jj, ii] = np.conj(X)
    return F


def test_als_target_is_per_input_least_squares():
    """h_k equals numpy's least-squares solution of min_x sum |x conj(g_j) M_kj - V_kj|^2
    over channels and j != k, built from the full Hermitian matrices."""
    rng = np.random.default_rng(21)
    N, C = 7, 3
    V, M, g = rand_cal(rng, N, C)
    h = oracle.calib_als_target(V, M, g)
    Vf, Mf = full_hermitian(V, N), full_hermitian(M, N)
    for k in range(N):
        js = [j for j in range(N) if j != k]
        a = (np.conj(g[js])[None, :] * Mf[:, k, js]).ravel()
        b = Vf[:, k, js].ravel()
        x = np.linalg.lstsq(a[:, None], b, rcond=None)[0][0]
        assert h[k] == pytest.approx(x, rel=1e-12)


def test_als_target_zeroes_its_gradient_component():
    """Replacing g_k by h_k (others fixed) makes the k-th gradient component vanish."""
    rng = np.random.default_rng(22)
    N, C = 9, 4
    V, M, g = rand_cal(rng, N, C)
    h = oracle.calib_als_target(V, M, g)
    scale = np.abs(oracle.calib_grad(V, M, g)).max()
    for k in range(N):
        gk = g.copy()
        gk[k] = h[k]
        assert abs(oracle.calib_grad(V, M, gk)[k]) <= 1e-11 * scale


def test_als_fixed_point_at_truth():
    rng = np.random.default_rng(23)
    N, C = 11, 3
    _, M, g = rand_cal(rng, N, C)
    ii, jj = np.tril_indices(N)
    V = g[ii] * np.conj(g[jj]) * M
    V[:, ii == jj] = -5.0  # autos carry weight 0
    np.testing.assert_allclose(oracle.calib_als_target(V, M, g), g, rtol=1e-13)


def test_solve_golden_two_inputs():
    """N = 2, V_10 = 2i, M_10 = 1, g0 = (1, 1), by hand: sweep 1 (plain) gives
    h = (conj(V_10) g_1 / |g_1|^2, V_10 g_0 / |g_0|^2) = (-2i, 2i); sweep 2 gives
    h = (1, 1) from (-2i, 2i) and averages to (0.5 - i, 0.5 + i)."""
    V = np.zeros((1, 3), complex)
    M = np.zeros((1, 3), complex)
    V[0, 1], M[0, 1] = 2j, 1.0
    g1, l1 = oracle.calib_solve(V, M, np.array([1.0, 1.0]), 1)
    np.testing.assert_allclose(g1, [-2j, 2j], atol=1e-15)
    assert l1[0] == pytest.approx(abs(1 - 2j) ** 2)
    g2, _ = oracle.calib_solve(V, M, np.array([1.0, 1.0]), 2)
    np.testing.assert_allclose(g2, [0.5 - 1j, 0.5 + 1j], atol=1e-15)


def test_solve_recovers_true_gains():
    """Noise-free data: the solve converges to the true gains up to one global
    phase (the loss cannot see it), and the loss falls to rounding level."""
    rng = np.random.default_rng(24)
    N, C = 16, 5
    _, M, g_true = rand_cal(rng, N, C)
    ii, jj = np.tril_indices(N)
    V = g_true[ii] * np.conj(g_true[jj]) * M
    g0 = g_true * (1 + 0.2 * (rng.standard_normal(N) + 1j * rng.standard_normal(N)))
    g, losses = oracle.calib_solve(V, M, g0, 60)
    ph = np.vdot(g, g_true)
    g_al = g * ph / abs(ph)
    assert np.abs(g_al - g_true).max() <= 1e-9 * np.abs(g_true).max()
    assert losses[-1] <= 1e-16 * losses[0]
    assert oracle.calib_loss(V, M, g) <= 1e-20 * losses[0]


# ---------------------------------------------------------------------------
# per-channel gains
# ---------------------------------------------------------------------------
def test_calib_chan_golden_two_inputs():
    """N = 2, two channels, by hand.  Channel 0: g = (1, i), M_10 = 1, V_10 = 0:
    R = i, L_0 = 1, grad = (2, 2i).  Channel 1: g = (2, 1), M_10 = 1, V_10 = 1:
    R = g_1 conj(g_0) M - V = 1, L_1 = 1, grad_1 = 2 R g_0 conj(M) = 4,
    grad_0 = 2 conj(R) g_1 M = 2."""
    V = np.zeros((2, 3), complex)
    M = np.zeros((2, 3), complex)
    M[:, 1] = 1.0
    V[1, 1] = 1.0
    G = np.array([[1.0, 1j], [2.0, 1.0]])
    assert oracle.calib_chan_loss(V, M, G) == pytest.approx(2.0, abs=1e-15)
    np.testing.assert_allclose(oracle.calib_chan_grad(V, M, G), [[2.0, 2j], [2.0, 4.0]],
                               atol=1e-14)


def test_calib_chan_against_autograd():
    """Per-channel loss and gradient pinned by torch autograd on a complex128
    loss over the full matrices, G_c g_i(c) conj(g_j(c)) per channel."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    N, C = 6, 4
    V, M, _ = rand_cal(rng, N, C)
    G = rng.uniform(0.8, 1.2, (C, N)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, N)))
    Vf = np.zeros((C, N, N), complex)
    Mf = np.zeros((C, N, N), complex)
    ii, jj = np.tril_indices(N)
    Vf[:, ii, jj] = V
    Mf[:, ii, jj] = M
    gt = torch.tensor(G, dtype=torch.complex128, requires_grad=True)
    Gm = gt[:, :, None] * torch.conj(gt)[:, None, :]
    R = Gm * torch.tensor(Mf) - torch.tensor(Vf)
    mask = torch.tril(torch.ones(N, N, dtype=torch.bool), diagonal=-1)
    L = (R.abs() ** 2)[:, mask].sum()
    L.backward()
    assert oracle.calib_chan_loss(V, M, G) == pytest.approx(L.item(), rel=1e-12)
    np.testing.assert_allclose(oracle.calib_chan_grad(V, M, G), gt.grad.numpy(), rtol=1e-10,
                               atol=1e-12)


def test_calib_chan_reduces_to_shared_gains():
    """With the same gains in every channel the per-channel loss is the
    frequency-independent loss, the channel sum of the per-channel gradients
    is its gradient, and the per-channel target differs from it only through
    the per-channel normal equations (equal when there is one channel)."""
    rng = np.random.default_rng(32)
    N, C = 8, 5
    V, M, g = rand_cal(rng, N, C)
    G = np.tile(g, (C, 1))
    assert oracle.calib_chan_loss(V, M, G) == pytest.approx(oracle.calib_loss(V, M, g), rel=1e-13)
    np.testing.assert_allclose(oracle.calib_chan_grad(V, M, G).sum(0), oracle.calib_grad(V, M, g),
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.calib_chan_als_target(V[:1], M[:1], G[:1])[0],
                               oracle.calib_als_target(V[:1], M[:1], g), rtol=1e-13)


def test_calib_chan_phase_per_channel():
    """Each channel's loss sees only that channel's gains, up to a phase of
    its own: G[c] -> G[c] e^{i th_c} with independent th_c leaves the loss
    unchanged and rotates channel c's gradient by e^{i th_c}."""
    rng = np.random.default_rng(35)
    N, C = 7, 4
    V, M, _ = rand_cal(rng, N, C)
    G = rng.uniform(0.8, 1.2, (C, N)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, N)))
    ph = np.exp(1j * rng.uniform(0, 2 * np.pi, C))[:, None]
    assert oracle.calib_chan_loss(V, M, G * ph) == pytest.approx(oracle.calib_chan_loss(V, M, G), rel=1e-12)
    np.testing.assert_allclose(oracle.calib_chan_grad(V, M, G * ph), oracle.calib_chan_grad(V, M, G) * ph,
                               rtol=1e-10, atol=1e-12)


def test_calib_chan_target_zeroes_its_gradient_component():
    rng = np.random.default_rng(33)
    N, C = 7, 3
    V, M, _ = rand_cal(rng, N, C)
    G = rng.uniform(0.8, 1.2, (C, N)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, N)))
    H = oracle.calib_chan_als_target(V, M, G)
    scale = np.abs(oracle.calib_chan_grad(V, M, G)).max()
    for c in range(C):
        for k in range(N):
            Gk = G.copy()
            Gk[c, k] = H[c, k]
            assert abs(oracle.calib_chan_grad(V, M, Gk)[c, k]) <= 1e-11 * scale


def test_calib_chan_solve_recovers_channel_dependent_gains():
    """Noise-free data whose gains change across the band: the per-channel
    solve recovers every channel's gains up to that channel's global phase,
    which a single frequency-independent gain per input cannot fit."""
    rng = np.random.default_rng(34)
    N, C = 12, 4
    _, M, _ = rand_cal(rng, N, C)
    G_true = rng.uniform(0.8, 1.2, (C, N)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, N)))
    ii, jj = np.tril_indices(N)
    V = G_true[:, ii] * np.conj(G_true[:, jj]) * M
    G0 = G_true * (1 + 0.2 * (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N))))
    G, losses = oracle.calib_chan_solve(V, M, G0, 60)
    for c in range(C):
        ph = np.vdot(G[c], G_true[c])
        assert np.abs(G[c] * ph / abs(ph) - G_true[c]).max() <= 1e-9 * np.abs(G_true).max()
    assert losses[-1] <= 1e-16 * losses[0]
    g_shared, l_shared = oracle.calib_solve(V, M, G0.mean(0), 60)
    assert l_shared[-1] > 1e3 * losses[-1]


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


def test_jones_golden_two_tiles():
    """Two tiles, one channel, M_10 = I, V = 0, J_0 = I, J_1 = [[1, 1], [0, 1]]
    (leakage), by hand: R = J_1, L = ||J_1||^2 = 3, grad_1 = 2 R J_0 M^H =
    2 J_1, grad_0 = 2 R^H J_1 M = 2 J_1^H J_1 = [[2, 2], [2, 4]]."""
    B = 4 * 5 // 2
    V = np.zeros((1, B), complex)
    M = np.zeros((1, B), complex)
    M[0, oracle.baseline_index(2, 0)] = 1.0
    M[0, oracle.baseline_index(3, 1)] = 1.0
    J = np.array([np.eye(2), [[1.0, 1.0], [0.0, 1.0]]], complex)
    assert oracle.calib_jones_loss(V, M, J) == pytest.approx(3.0, abs=1e-15)
    np.testing.assert_allclose(oracle.calib_jones_grad(V, M, J),
                               [[[2, 2], [2, 4]], [[2, 2], [0, 2]]], atol=1e-14)


def test_jones_against_autograd():
    """Loss and gradient pinned by torch autograd on a complex128 loss over
    the full N x N matrices cut into 2x2 tile blocks."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(41)
    n_tiles, C = 5, 3
    N = 2 * n_tiles
    V, M, _ = rand_cal(rng, N, C)
    J = rand_jones(rng, n_tiles)
    Vf, Mf = np.zeros((C, N, N), complex), np.zeros((C, N, N), complex)
    ii, jj = np.tril_indices(N)
    Vf[:, ii, jj] = V
    Mf[:, ii, jj] = M
    Jt = torch.tensor(J, requires_grad=True)
    # block-diagonal N x N Jones: Jfull[2a+p, 2a+r] = J_a[p, r]
    Jfull = torch.block_diag(*[Jt[t] for t in range(n_tiles)])
    R = Jfull[None] @ torch.tensor(Mf) @ torch.conj(Jfull).T[None] - torch.tensor(Vf)
    tile = np.arange(N) // 2
    mask = torch.tensor(tile[:, None] > tile[None, :])
    L = (R.abs() ** 2)[:, mask].sum()
    L.backward()
    assert oracle.calib_jones_loss(V, M, J) == pytest.approx(L.item(), rel=1e-12)
    np.testing.assert_allclose(oracle.calib_jones_grad(V, M, J), Jt.grad.numpy(), rtol=1e-10,
                               atol=1e-12)


def test_jones_diagonal_is_per_input_gains():
    """Diagonal J_a = diag(g_2a, g_2a+1) with the intra-tile pair zeroed in V
    and M: the Jones loss is the per-input loss and the diagonal of the Jones
    gradient is the per-input gradient."""
    rng = np.random.default_rng(42)
    n_tiles, C = 6, 4
    N = 2 * n_tiles
    V, M, g = rand_cal(rng, N, C)
    for a in range(n_tiles):
        V[:, oracle.baseline_index(2 * a + 1, 2 * a)] = 0
        M[:, oracle.baseline_index(2 * a + 1, 2 * a)] = 0
    J = np.zeros((n_tiles, 2, 2), complex)
    J[:, 0, 0], J[:, 1, 1] = g[0::2], g[1::2]
    assert oracle.calib_jones_loss(V, M, J) == pytest.approx(oracle.calib_loss(V, M, g), rel=1e-12)
    Gj = oracle.calib_jones_grad(V, M, J)
    Gi = oracle.calib_grad(V, M, g)
    np.testing.assert_allclose(Gj[:, 0, 0], Gi[0::2], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(Gj[:, 1, 1], Gi[1::2], rtol=1e-11, atol=1e-12)


def test_jones_target_is_least_squares():
    """H_a equals numpy's least-squares solution of X [B_1 B_2 ...] = [W_1 W_2 ...]
    built from the full Hermitian matrices: B = M_ab J_b^H, W = V_ab over every
    other tile b and channel (the full matrix holds both orientations)."""
    rng = np.random.default_rng(43)
    n_tiles, C = 5, 2
    N = 2 * n_tiles
    V, M, _ = rand_cal(rng, N, C)
    J = rand_jones(rng, n_tiles)
    H = oracle.calib_jones_als_target(V, M, J)
    Vf, Mf = full_hermitian(V, N), full_hermitian(M, N)
    for a in range(n_tiles):
        Bs, Ws = [], []
        for c in range(C):
            for b in range(n_tiles):
                if b == a:
                    continue
                Mab = Mf[c, 2 * a:2 * a + 2, 2 * b:2 * b + 2]
                Bs.append(Mab @ np.conj(J[b]).T)
                Ws.append(Vf[c, 2 * a:2 * a + 2, 2 * b:2 * b + 2])
        Bc, Wc = np.hstack(Bs), np.hstack(Ws)
        X = np.linalg.lstsq(Bc.T, Wc.T, rcond=None)[0].T
        np.testing.assert_allclose(H[a], X, rtol=1e-11, atol=1e-12)


def test_jones_target_zeroes_its_gradient_block():
    rng = np.random.default_rng(44)
    n_tiles, C = 6, 3
    V, M, _ = rand_cal(rng, 2 * n_tiles, C)
    J = rand_jones(rng, n_tiles)
    H = oracle.calib_jones_als_target(V, M, J)
    scale = np.abs(oracle.calib_jones_grad(V, M, J)).max()
    for a in range(n_tiles):
        Ja = J.copy()
        Ja[a] = H[a]
        assert np.abs(oracle.calib_jones_grad(V, M, Ja)[a]).max() <= 1e-11 * scale


def test_jones_unitary_invariance_for_unpolarised_model():
    """M_ab = m_ab I (an unpolarised model): J_a M J_b^H = m J_a J_b^H, so
    replacing every J_a by J_a U for one unitary U leaves the loss unchanged
    and turns the gradient into grad U (grad_a = 2 sum R J_b M^H ...).  Using
    J^T or conj(J) where J^H belongs breaks both for a complex U."""
    rng = np.random.default_rng(46)
    n_tiles, C = 6, 3
    N = 2 * n_tiles
    B = N * (N + 1) // 2
    V = rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))
    M = np.zeros((C, B), complex)
    a, b, idx = oracle._jones_blocks(n_tiles)
    m = rng.standard_normal((C, len(a))) + 1j * rng.standard_normal((C, len(a)))
    for c in range(C):
        M[c][idx[:, 0, 0]] = m[c]
        M[c][idx[:, 1, 1]] = m[c]
    J = rand_jones(rng, n_tiles)
    Q, _ = np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))
    JU = J @ Q
    assert oracle.calib_jones_loss(V, M, JU) == pytest.approx(oracle.calib_jones_loss(V, M, J), rel=1e-12)
    np.testing.assert_allclose(oracle.calib_jones_grad(V, M, JU), oracle.calib_jones_grad(V, M, J) @ Q,
                               rtol=1e-10, atol=1e-12)


def test_jones_solve_recovers_leaky_jones():
    """Noise-free data from Jones matrices with leakage: the solve recovers
    them up to one global phase (the only freedom the loss leaves for a
    generic model), which per-input gains cannot fit."""
    rng = np.random.default_rng(45)
    n_tiles, C = 7, 3
    N = 2 * n_tiles
    _, M, g = rand_cal(rng, N, C)
    J_true = rand_jones(rng, n_tiles)
    a, b, idx = oracle._jones_blocks(n_tiles)
    V = np.zeros_like(M)
    for c in range(C):
        V[c][idx] = J_true[a] @ M[c][idx] @ np.conj(np.swapaxes(J_true[b], -1, -2))
    J0 = J_true + 0.1 * (rng.standard_normal(J_true.shape) + 1j * rng.standard_normal(J_true.shape))
    J, losses = oracle.calib_jones_solve(V, M, J0, 80)
    ph = np.vdot(J.ravel(), J_true.ravel())
    assert np.abs(J * ph / abs(ph) - J_true).max() <= 1e-8 * np.abs(J_true).max()
    assert losses[-1] <= 1e-14 * losses[0]


# ---------------------------------------------------------------------------
# gridding
# ---------------------------------------------------------------------------
C_LIGHT = 299792458.0


def grid_problem(rng, n_tiles, n_chan, Ng, du, f0=150e6, df=1e6, vmax=1000):
    """Tile positions that keep every point inside the grid, random int32 visibilities."""
    N = 2 * n_tiles
    B = N * (N + 1) // 2
    reach = (0.5 * Ng - 5) * du * C_LIGHT / (f0 + (n_chan - 1) * df) / 2
    tile_xy = rng.uniform(-reach, reach, (n_tiles, 2)) * 0.7
    vis = rng.integers(-vmax, vmax + 1, (n_chan, B, 2)).astype(np.int32)
    return tile_xy, vis, f0, df


def numpy_points(tile_xy, vis, f0, df, Ng, du):
    """(x, y, V[4]) of every gridded point, both orientations, from the definition."""
    n_tiles = tile_xy.shape[0]
    n_chan = vis.shape[0]
    Vc = vis[..., 0].astype(np.float64) + 1j * vis[..., 1]
    pts = []
    for c in range(n_chan):
        nu = f0 + c * df
        for a in range(n_tiles):
            for b in range(a):
                u = (tile_xy[a] - tile_xy[b]) * nu / C_LIGHT / du
                V = np.array([Vc[c, oracle.baseline_index(2 * a + p, 2 * b + q)]
                              for p in (0, 1) for q in (0, 1)])
                Vr = np.array([np.conj(Vc[c, oracle.baseline_index(2 * a + q, 2 * b + p)])
                               for p in (0, 1) for q in (0, 1)])
                pts.append((u[0] + Ng / 2, u[1] + Ng / 2, V))
                pts.append((Ng / 2 - u[0], Ng / 2 - u[1], Vr))
    return pts


def test_grid_brute_force_numpy():
    rng = np.random.default_rng(31)
    Ng, du, W, sigma = 40, 2.0, 7, 1.1
    tile_xy, vis, f0, df = grid_problem(rng, 4, 3, Ng, du)
    G = oracle.grid(tile_xy, vis, f0, df, Ng, du, W, sigma)
    ref = np.zeros((4, Ng, Ng), complex)
    cells = np.arange(Ng)
    for x, y, V in numpy_points(tile_xy, vis, f0, df, Ng, du):
        sx = cells[np.abs(cells - x) < W / 2]
        sy = cells[np.abs(cells - y) < W / 2]
        w = np.exp(-((sy[:, None] - y) ** 2 + (sx[None, :] - x) ** 2) / (2 * sigma ** 2))
        for pol in range(4):
            np.add.at(ref[pol], (sy[:, None], sx[None, :]), w * V[pol])
    np.testing.assert_allclose(G, ref, rtol=1e-12, atol=1e-9)


def test_grid_golden_single_baseline():
    """Two tiles on the x axis, one channel, u = 5 cells exactly: the XX grid
    holds V at (Ng/2, Ng/2 + 5), V e^{-1/(2 sigma^2)} one cell away, conj(V) at
    (Ng/2, Ng/2 - 5), and nothing beyond three cells."""
    Ng, du, W, sigma, nu = 32, 1.0, 7, 1.0, 200e6
    tile_xy = np.array([[0.0, 0.0], [5 * du * C_LIGHT / nu, 0.0]])
    vis = np.zeros((1, 10, 2), np.int32)
    vis[0, oracle.baseline_index(2, 0)] = (3, -2)  # tile 1 X with tile 0 X
    G = oracle.grid(tile_xy, vis, nu, 0.0, Ng, du, W, sigma)
    c = Ng // 2
    assert G[0, c, c + 5] == pytest.approx(3 - 2j, abs=1e-9)
    assert G[0, c, c + 6] == pytest.approx((3 - 2j) * np.exp(-0.5), abs=1e-9)
    assert G[0, c + 1, c + 4] == pytest.approx((3 - 2j) * np.exp(-1.0), abs=1e-9)
    assert G[0, c, c - 5] == pytest.approx(3 + 2j, abs=1e-9)
    assert G[0, c, c + 9] == 0 and G[0, c + 4, c + 5] == 0
    assert np.abs(G[1:]).max() == 0  # only the XX product is non-zero


def test_grid_hermitian():
    """The reversed baseline makes G_pq(-u) = conj(G_qp(u)):
    G[2p+q][Ng-r][Ng-s] = conj(G[2q+p][r][s]) for r, s >= 1."""
    rng = np.random.default_rng(32)
    Ng, du, W, sigma = 48, 1.5, 7, 1.3
    tile_xy, vis, f0, df = grid_problem(rng, 5, 4, Ng, du)
    G = oracle.grid(tile_xy, vis, f0, df, Ng, du, W, sigma)
    flip = G[:, :0:-1, :0:-1]  # [pol][Ng - r][Ng - s] for r, s = 1 .. Ng-1
    swap = G[[0, 2, 1, 3], 1:, 1:]
    np.testing.assert_allclose(flip, np.conj(swap), rtol=1e-12, atol=1e-9)


def test_grid_total_weight():
    """Sum over the grid = sum over points of V Sx Sy, with Sx the sum of the
    1D kernel over the cells in the point's support (the Gaussian factorises)."""
    rng = np.random.default_rng(33)
    Ng, du, W, sigma = 36, 2.5, 7, 0.9
    tile_xy, vis, f0, df = grid_problem(rng, 4, 5, Ng, du)
    G = oracle.grid(tile_xy, vis, f0, df, Ng, du, W, sigma)
    cells = np.arange(Ng)
    tot = np.zeros(4, complex)
    for x, y, V in numpy_points(tile_xy, vis, f0, df, Ng, du):
        Sx = np.exp(-((cells - x) ** 2) / (2 * sigma ** 2))[np.abs(cells - x) < W / 2].sum()
        Sy = np.exp(-((cells - y) ** 2) / (2 * sigma ** 2))[np.abs(cells - y) < W / 2].sum()
        tot += V * Sx * Sy
    np.testing.assert_allclose(G.sum(axis=(1, 2)), tot, rtol=1e-11)


def test_grid_cell_matches_grid():
    rng = np.random.default_rng(34)
    Ng, du, W, sigma = 44, 1.7, 7, 1.0
    tile_xy, vis, f0, df = grid_problem(rng, 6, 3, Ng, du)
    G = oracle.grid(tile_xy, vis, f0, df, Ng, du, W, sigma)
    for _ in range(25):
        pol, r, s = rng.integers(0, 4), rng.integers(0, Ng), rng.integers(0, Ng)
        assert oracle.grid_cell(tile_xy, vis, f0, df, Ng, du, W, sigma, pol, r, s) == \
            pytest.approx(G[pol, r, s], rel=1e-12, abs=1e-9)


# ---------------------------------------------------------------------------
# Stokes conversion
# ---------------------------------------------------------------------------
def test_stokes_zenith_is_plain_sum_and_difference():
    """At the zenith J is the rotation by chi; with chi = 0 it is the identity
    and I = XX + YY, Q = XX - YY, U = XY + YX, V = -i (XY - YX)."""
    n = 8
    rng = np.random.default_rng(41)
    inst = rng.standard_normal((4, n, n)) + 1j * rng.standard_normal((4, n, n))
    S = oracle.stokes(inst, 0.1, 0.0)
    XX, XY, YX, YY = inst[:, n // 2, n // 2]
    np.testing.assert_allclose(S[:, n // 2, n // 2],
                               [XX + YY, XX - YY, XY + YX, -1j * (XY - YX)], rtol=1e-14)


def test_stokes_round_trip_of_a_known_sky():
    """Instrumental images made from known Stokes through J B J^H (written
    here independently) convert back to those Stokes."""
    n = 16
    dl, chi = 0.11, 0.37
    rng = np.random.default_rng(42)
    I, Q, U, V = rng.standard_normal((4, n, n))
    inst = np.zeros((4, n, n), complex)
    idx = np.arange(n) - n / 2
    for r in range(n):
        for c in range(n):
            l, m = idx[c] * dl, idx[r] * dl
            rho = np.hypot(l, m)
            if rho >= 1:
                continue
            th, ph = np.arcsin(rho), np.arctan2(m, l) + chi
            J = np.array([[np.cos(th) * np.cos(ph), -np.sin(ph)], [np.cos(th) * np.sin(ph), np.cos(ph)]])
            B = 0.5 * np.array([[I[r, c] + Q[r, c], U[r, c] + 1j * V[r, c]],
                                [U[r, c] - 1j * V[r, c], I[r, c] - Q[r, c]]])
            C = J @ B @ J.T
            inst[:, r, c] = [C[0, 0], C[0, 1], C[1, 0], C[1, 1]]
    S = oracle.stokes(inst, dl, chi)
    up = np.hypot(*np.meshgrid(idx * dl, idx * dl)) < 1
    for k, ref in enumerate((I, Q, U, V)):
        np.testing.assert_allclose(S[k][up], ref[up], rtol=1e-10, atol=1e-12)
    assert np.all(S[:, ~up] == 0)


def test_stokes_unpolarised_source_stays_unpolarised():
    """An unpolarised sky (B = I/2 1) seen anywhere above the horizon gives
    Q = U = V = 0 after conversion, though the instrumental XY is not zero."""
    n = 12
    dl, chi = 0.15, -0.8
    idx = np.arange(n) - n / 2
    inst = np.zeros((4, n, n), complex)
    for r in range(n):
        for c in range(n):
            l, m = idx[c] * dl, idx[r] * dl
            rho = np.hypot(l, m)
            if rho >= 1:
                continue
            ct, ph = np.sqrt(1 - rho ** 2), np.arctan2(m, l) + chi
            # J J^T for the dipole response, times 1/2 (unit Stokes I)
            a, b, cc, d = ct * np.cos(ph), -np.sin(ph), ct * np.sin(ph), np.cos(ph)
            inst[:, r, c] = 0.5 * np.array([a * a + b * b, a * cc + b * d, cc * a + d * b, cc * cc + d * d])
    S = oracle.stokes(inst, dl, chi)
    up = np.hypot(*np.meshgrid(idx * dl, idx * dl)) < 1
    np.testing.assert_allclose(S[0][up], 1.0, rtol=1e-12)
    np.testing.assert_allclose(S[1:, up], 0.0, atol=1e-12)
    assert np.abs(inst[1][up]).max() > 0.05
