"""GPU per-pixel Stokes conversion against the FP64 oracle.

Tolerance, from the FP32 arithmetic: a pixel's result is bounded by
sum|C| / cos^2(theta) (two factors 1/cos(theta) from J^-1).  The products
and sums add ~1e-6 of that bound; cos^2(theta) = 1 - rho^2 carries an
absolute error of ~1e-7 (dl and rho^2 in float), i.e. a relative error of
1e-7 / cos^2(theta) in a result that scales as 1/cos^2(theta).  So
|dS| <= sum|C| (2e-6 / cos^2 + 4e-7 / cos^4), checked where
cos(theta) >= 0.05 (up to 87 degrees from the zenith).  Pixels clearly below
the horizon must be exactly zero."""
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


def geometry(n, dl):
    idx = np.arange(n) - n / 2
    l, m = np.meshgrid(idx * dl, idx * dl)
    return np.hypot(l, m)


def gpu(mw, inst, dl, chi):
    import torch

    out = mw.stokes(torch.from_numpy(inst.astype(np.complex64)).cuda(), dl, chi)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(got, ref, inst, n, dl, pixels=None):
    rho = geometry(n, dl)
    ct2 = np.clip(1 - rho ** 2, 1e-30, None)
    bound = np.abs(inst).sum(axis=0) * (2e-6 / ct2 + 4e-7 / ct2 ** 2)
    ok = (ct2 >= 0.05 ** 2)
    sel = np.zeros((n, n), bool)
    if pixels is None:
        sel[:] = True
    else:
        for r, c in pixels:
            sel[r, c] = True
    m = ok & sel
    err = np.abs(got - ref)[:, m]
    assert (err <= bound[m][None, :]).all(), (err / bound[m][None, :]).max()
    below = (rho >= 1 + 1e-5) & sel
    assert np.all(got[:, below] == 0)


@pytest.mark.parametrize("n,dl,chi", [(8, 0.3, 0.2), (64, 0.031, 1.1), (130, 0.0152, -0.4),
                                      (2, 0.5, 0.0)])
def test_stokes_small(mw, n, dl, chi):
    rng = np.random.default_rng(n)
    inst = (rng.standard_normal((4, n, n)) + 1j * rng.standard_normal((4, n, n))).astype(np.complex64)
    got = gpu(mw, inst, dl, chi)
    check(got, oracle.stokes(inst.astype(np.complex128), dl, chi), inst, n, dl)


def test_stokes_round_trip_gpu(mw):
    """A known sky pushed through J B J^T (numpy, FP64) comes back."""
    n, dl, chi = 256, 1.6 / 256, 0.65
    rng = np.random.default_rng(3)
    I, Q, U, V = rng.standard_normal((4, n, n))
    idx = np.arange(n) - n / 2
    l, m = np.meshgrid(idx * dl, idx * dl)
    rho = np.hypot(l, m)
    ct = np.sqrt(np.clip(1 - rho ** 2, 0, None))
    ph = np.arctan2(m, l) + chi
    a, b, c, d = ct * np.cos(ph), -np.sin(ph), ct * np.sin(ph), np.cos(ph)
    B00, B01, B10, B11 = 0.5 * (I + Q), 0.5 * (U + 1j * V), 0.5 * (U - 1j * V), 0.5 * (I - Q)
    # C = J B J^T with J = [[a, b], [c, d]]: C_kl = sum_ij J_ki B_ij J_lj
    XX = a * (a * B00 + b * B01) + b * (a * B10 + b * B11)
    XY = a * (c * B00 + d * B01) + b * (c * B10 + d * B11)
    YX = c * (a * B00 + b * B01) + d * (a * B10 + b * B11)
    YY = c * (c * B00 + d * B01) + d * (c * B10 + d * B11)
    inst = np.stack([XX, XY, YX, YY]).astype(np.complex64)
    got = gpu(mw, inst, dl, chi)
    up = rho < 0.99
    for k, ref in enumerate((I, Q, U, V)):
        np.testing.assert_allclose(got[k][up], ref[up], rtol=2e-4, atol=2e-4)


def test_stokes_full_size_sampled(mw):
    """The 4096 x 4096 whole-hemisphere image of the benchmark (dl = 2/n),
    on seeded values, checked on sampled pixels."""
    import torch

    n, dl, chi = 4096, 2.0 / 4096, 0.3
    rng = np.random.default_rng(8)
    inst = (rng.standard_normal((4, n, n), dtype=np.float32)
            + 1j * rng.standard_normal((4, n, n), dtype=np.float32)).astype(np.complex64)
    got = gpu(mw, inst, dl, chi)
    pix = [(n // 2, n // 2), (0, 0), (n - 1, n - 1), (n // 2, 5), (17, n // 2), (n // 2 + 1000, n // 2 - 1200)]
    pix += [(int(r), int(c)) for r, c in rng.integers(0, n, (30, 2))]
    ref = oracle.stokes(inst.astype(np.complex128), dl, chi, pixels=pix)
    check(got, ref, inst, n, dl, pixels=pix)
    torch.cuda.synchronize()


def test_stokes_invalid_args(mw):
    import torch

    x = torch.zeros((4, 8, 8), dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    L = mw.lib()
    xp, yp = torch.view_as_real(x).data_ptr(), torch.view_as_real(y).data_ptr()
    assert L.mwax_stokes(xp, 7, 0.1, 0.0, yp, None) == 1      # odd n
    assert L.mwax_stokes(xp, 8, 0.0, 0.0, yp, None) == 1      # dl <= 0
    assert L.mwax_stokes(xp, 8, 0.1, 0.0, xp, None) == 1      # in place
    assert L.mwax_stokes(xp + 4, 8, 0.1, 0.0, yp, None) == 1  # misaligned
    h = torch.zeros((4, 8, 8), dtype=torch.complex64)
    assert L.mwax_stokes(torch.view_as_real(h).data_ptr(), 8, 0.1, 0.0, yp, None) == 1
    # partly overlapping ranges (either order, by one pixel or by most of a plane)
    big = torch.zeros((2, 4, 8, 8), dtype=torch.complex64, device="cuda")
    bp = torch.view_as_real(big).data_ptr()
    for off in (8, 8 * 100, 8 * (4 * 64 - 1)):
        assert L.mwax_stokes(bp, 8, 0.1, 0.0, bp + off, None) == 1
        assert L.mwax_stokes(bp + off, 8, 0.1, 0.0, bp, None) == 1
    # adjacent ranges do not overlap
    assert L.mwax_stokes(bp, 8, 0.1, 0.0, bp + 8 * 4 * 64, None) == 0
    torch.cuda.synchronize()
