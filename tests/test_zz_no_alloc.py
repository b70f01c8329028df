"""The allocation-free calibration entry point (mwax_calib_loss_grad_static)
gives exactly the loss and gradient of mwax_calib_loss_grad with a caller
workspace, call after call.

It exists for callers that cannot allocate device memory at the point of
use -- for instance a real-time integration loop, where cudaMalloc would
synchronise the device and add unpredictable latency, or an application
whose device memory all belongs to another allocator.  Both entry points run
the same deterministic kernels on the same inputs, so the results must be
bit-identical, not merely close.  The file is named so that pytest collects
it last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(N, C, seed):
    rng = np.random.default_rng(seed)
    B = N * (N + 1) // 2
    V = (rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))).astype(np.complex64)
    M = (rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))).astype(np.complex64)
    g = (rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))).astype(np.complex64)
    return V, M, g


def _both(mw, torch, V, M, g, N, C):
    """(loss, grad) from the caller-workspace call and from the static call."""
    L = mw.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Vp, Mp, gp = (torch.view_as_real(t).data_ptr() for t in (V, M, g))
    ws = mw.calib_workspace(N, C)
    loss_ref = torch.empty((), dtype=torch.float32, device="cuda")
    grad_ref = torch.empty((N, 2), dtype=torch.float32, device="cuda")
    assert L.mwax_calib_loss_grad(Vp, Mp, gp, N, C, ws.data_ptr(), loss_ref.data_ptr(),
                                  grad_ref.data_ptr(), stream) == 0
    loss = torch.full((), float("nan"), dtype=torch.float32, device="cuda")
    grad = torch.full((N, 2), float("nan"), dtype=torch.float32, device="cuda")
    assert L.mwax_calib_loss_grad_static(Vp, Mp, gp, N, C, loss.data_ptr(), grad.data_ptr(),
                                         stream) == 0
    torch.cuda.synchronize()
    return (loss_ref.cpu().numpy(), grad_ref.cpu().numpy()), (loss.cpu().numpy(), grad.cpu().numpy())


def test_static_workspace_matches_caller_workspace(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for call, (N, C, seed) in enumerate([(1024, 24, 1), (300, 7, 2)]):
        V, M, g = (torch.from_numpy(a).cuda() for a in _inputs(N, C, seed))
        (lr, gr), (ls, gs) = _both(mwax_lib, torch, V, M, g, N, C)
        assert np.isfinite(ls) and np.all(np.isfinite(gs)), call
        assert np.array_equal(ls.view(np.uint32), lr.view(np.uint32)), (call, ls, lr)
        assert np.array_equal(gs.view(np.uint32), gr.view(np.uint32)), call


def test_static_workspace_leftovers_do_not_leak(mwax_lib):
    """A call whose partial sums are all NaN leaves them in the shared array;
    the next call, at a shape with other tile and channel-group counts (so the
    partial sums sit at other offsets), must still equal the caller-workspace
    result bit for bit: every slot a call reads it has written itself."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N0, C0 = 1024, 24
    V, M, g = (torch.from_numpy(a).cuda() for a in _inputs(N0, C0, 3))
    V.fill_(float("nan"))
    _, (lp, gp) = _both(mwax_lib, torch, V, M, g, N0, C0)
    assert np.isnan(lp) and np.all(np.isnan(gp))  # the array now holds NaN partial sums
    for N, C, seed in [(300, 7, 4), (64, 2, 5)]:
        V, M, g = (torch.from_numpy(a).cuda() for a in _inputs(N, C, seed))
        (lr, gr), (ls, gs) = _both(mwax_lib, torch, V, M, g, N, C)
        assert np.isfinite(ls) and np.all(np.isfinite(gs)), (N, C)
        assert np.array_equal(ls.view(np.uint32), lr.view(np.uint32)), (N, C, ls, lr)
        assert np.array_equal(gs.view(np.uint32), gr.view(np.uint32)), (N, C)


def test_static_workspace_rejects_oversize_shapes(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = mwax_lib.lib()
    cap = L.mwax_calib_static_workspace_bytes()
    N = 4096
    assert L.mwax_calib_workspace_bytes(N, 8) > cap
    t = torch.zeros(4, dtype=torch.float32, device="cuda")
    p = t.data_ptr()
    assert L.mwax_calib_loss_grad_static(p, p, p, N, 8, p, p, None) == 1  # MWAX_ERR_INVALID_ARG
