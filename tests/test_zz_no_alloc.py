"""The allocation-free calibration entry point (mwax_calib_loss_grad_static)
gives the same loss and gradient as mwax_calib_loss_grad with a caller
workspace, call after call.

It exists for callers that cannot allocate device memory at the point of
use -- for instance a real-time integration loop, where cudaMalloc would
synchronise the device and add unpredictable latency.  The file is named so
that pytest collects it last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-5  # the calibration tests' loss tolerance
GRAD_RTOL = 1e-4  # and gradient tolerance (max-norm)


def _inputs(N, C, seed):
    rng = np.random.default_rng(seed)
    B = N * (N + 1) // 2
    V = (rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))).astype(np.complex64)
    M = (rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))).astype(np.complex64)
    g = (rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))).astype(np.complex64)
    return V, M, g


def test_static_workspace_matches_caller_workspace(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mw = mwax_lib
    L = mw.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (N, C, seed) in enumerate([(1024, 24, 1), (300, 7, 2)]):
        V, M, g = (torch.from_numpy(a).cuda() for a in _inputs(N, C, seed))
        Vp, Mp, gp = (torch.view_as_real(t).data_ptr() for t in (V, M, g))
        # existing entry point, caller-allocated workspace
        ws = mw.calib_workspace(N, C)
        loss_ref = torch.empty((), dtype=torch.float32, device="cuda")
        grad_ref = torch.empty((N, 2), dtype=torch.float32, device="cuda")
        assert L.mwax_calib_loss_grad(Vp, Mp, gp, N, C, ws.data_ptr(), loss_ref.data_ptr(),
                                      grad_ref.data_ptr(), ctypes.c_void_p(stream)) == 0
        # allocation-free entry point
        loss = torch.full((), float("nan"), dtype=torch.float32, device="cuda")
        grad = torch.full((N, 2), float("nan"), dtype=torch.float32, device="cuda")
        assert L.mwax_calib_loss_grad_static(Vp, Mp, gp, N, C, loss.data_ptr(), grad.data_ptr(),
                                             ctypes.c_void_p(stream)) == 0, f"call {call}"
        torch.cuda.synchronize()
        lr, l = float(loss_ref), float(loss)
        assert abs(l - lr) <= LOSS_RTOL * abs(lr), (call, l, lr)
        gr, gg = grad_ref.cpu().numpy(), grad.cpu().numpy()
        assert np.abs(gg - gr).max() <= GRAD_RTOL * np.abs(gr).max(), call


def test_static_workspace_rejects_oversize_shapes(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mw = mwax_lib
    L = mw.lib()
    cap = L.mwax_calib_static_workspace_bytes()
    N = 4096
    assert L.mwax_calib_workspace_bytes(N, 8) > cap
    t = torch.zeros(4, dtype=torch.float32, device="cuda")
    p = t.data_ptr()
    assert L.mwax_calib_loss_grad_static(p, p, p, N, 8, p, p, None) == 1  # MWAX_ERR_INVALID_ARG
