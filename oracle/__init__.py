"""CPU oracle for the X-engine correlator and the gain-calibration loss.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
The C source (``mwax_oracle.c``) shares no code with the CUDA library.

Parity pins for every function here live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(_HERE, "_lib", "libmwax_oracle.so")

OK, ERR_ARG, ERR_OOM, ERR_OVERFLOW = 0, 1, 2, 3


def build_command():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall",
            os.path.join(_HERE, "mwax_oracle.c"), "-o", LIB, "-lm"]


def build() -> None:
    cmd = build_command()
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        lib = ctypes.CDLL(LIB)
        lib.oracle_decode.restype = ctypes.c_int
        lib.oracle_decode.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p]
        lib.oracle_correlate.restype = ctypes.c_int
        lib.oracle_correlate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_n_baselines.restype = ctypes.c_int64
        lib.oracle_n_baselines.argtypes = [ctypes.c_int64]
        lib.oracle_baseline_index.restype = ctypes.c_int64
        lib.oracle_baseline_index.argtypes = [ctypes.c_int64, ctypes.c_int64]
        lib.oracle_calib_loss.restype = ctypes.c_double
        lib.oracle_calib_loss.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int]
        lib.oracle_calib_grad.restype = ctypes.c_int
        lib.oracle_calib_grad.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int,
                                                                  ctypes.c_void_p, ctypes.c_int]
        lib.oracle_grid.restype = ctypes.c_int
        lib.oracle_grid.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_grid_cell.restype = ctypes.c_int
        lib.oracle_grid_cell.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_void_p]
        lib.oracle_calib_als_target.restype = ctypes.c_int
        lib.oracle_calib_als_target.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int,
                                                                        ctypes.c_void_p, ctypes.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def decode(raw: np.ndarray, sample_bits: int):
    """Packed samples -> (re, im) int32 arrays of n samples."""
    raw = np.ascontiguousarray(raw, np.uint8).ravel()
    n = raw.size if sample_bits == 4 else raw.size // 2
    re = np.empty(n, np.int32)
    im = np.empty(n, np.int32)
    rc = _load().oracle_decode(raw.ctypes.data, sample_bits, n, re.ctypes.data, im.ctypes.data)
    if rc:
        raise ValueError("unsupported sample width")
    return re, im


def correlate(volt: np.ndarray, sample_bits: int, n_inputs: int, n_chan: int, n_time: int,
              want64: bool = False, n_threads: int | None = None):
    """Oracle correlation of packed voltages [n_chan][n_time][n_inputs].

    Returns int32 [n_chan, N(N+1)/2, 2] (and the int64 copy when want64).
    Raises OverflowError when a visibility exceeds the int32 range (the
    int64 copy is still returned through the exception's ``args[1]``)."""
    volt = np.ascontiguousarray(volt, np.uint8)
    bps = 1 if sample_bits == 4 else 2
    if volt.size != n_chan * n_time * n_inputs * bps:
        raise ValueError("voltage buffer size does not match the shape")
    B = n_inputs * (n_inputs + 1) // 2
    out = np.zeros((n_chan, B, 2), np.int32)
    out64 = np.zeros((n_chan, B, 2), np.int64) if want64 else None
    rc = _load().oracle_correlate(volt.ctypes.data, sample_bits, n_inputs, n_chan, n_time,
                                  out.ctypes.data, out64.ctypes.data if want64 else None,
                                  n_threads or threads())
    if rc == ERR_OVERFLOW:
        raise OverflowError("visibility outside the int32 range", out64)
    if rc:
        raise RuntimeError(f"oracle_correlate failed ({rc})")
    return (out, out64) if want64 else out


def n_baselines(n_inputs: int) -> int:
    return int(_load().oracle_n_baselines(n_inputs))


def baseline_index(i: int, j: int) -> int:
    return int(_load().oracle_baseline_index(i, j))


def _c128_as_pairs(a) -> np.ndarray:
    a = np.ascontiguousarray(a, np.complex128)
    return a.view(np.float64)


def calib_loss(V, M, g) -> float:
    """FP64 loss.  V, M: complex [n_chan, N(N+1)/2]; g: complex [N]."""
    V = np.ascontiguousarray(V, np.complex128)
    M = np.ascontiguousarray(M, np.complex128)
    g = np.ascontiguousarray(g, np.complex128)
    C, B = V.shape
    N = g.shape[0]
    assert B == N * (N + 1) // 2 and M.shape == V.shape
    return float(_load().oracle_calib_loss(V.ctypes.data, M.ctypes.data, g.ctypes.data, N, C))


def calib_grad(V, M, g, n_threads: int | None = None) -> np.ndarray:
    """FP64 gradient 2 dL/d conj(g), complex [N]."""
    V = np.ascontiguousarray(V, np.complex128)
    M = np.ascontiguousarray(M, np.complex128)
    g = np.ascontiguousarray(g, np.complex128)
    C, B = V.shape
    N = g.shape[0]
    assert B == N * (N + 1) // 2 and M.shape == V.shape
    out = np.zeros(N, np.complex128)
    rc = _load().oracle_calib_grad(V.ctypes.data, M.ctypes.data, g.ctypes.data, N, C,
                                   out.ctypes.data, n_threads or threads())
    if rc:
        raise RuntimeError("oracle_calib_grad failed")
    return out


def calib_als_target(V, M, g, n_threads: int | None = None) -> np.ndarray:
    """FP64 alternating least-squares target h, complex [N]: h_k minimises the
    loss over g_k with every other gain fixed at g (h_k = g_k where the
    normal equation is empty)."""
    V = np.ascontiguousarray(V, np.complex128)
    M = np.ascontiguousarray(M, np.complex128)
    g = np.ascontiguousarray(g, np.complex128)
    C, B = V.shape
    N = g.shape[0]
    assert B == N * (N + 1) // 2 and M.shape == V.shape
    out = np.zeros(N, np.complex128)
    rc = _load().oracle_calib_als_target(V.ctypes.data, M.ctypes.data, g.ctypes.data, N, C,
                                         out.ctypes.data, n_threads or threads())
    if rc:
        raise RuntimeError("oracle_calib_als_target failed")
    return out


def calib_solve(V, M, g0, n_iter: int, n_threads: int | None = None):
    """FP64 gain solve: ``n_iter`` alternating least-squares sweeps from g0.

    Sweep t (t = 1, 2, ...) computes the target h from the current gains for
    every input at once and then sets g = h when t is odd and g = (g + h) / 2
    when t is even; the averaging on every second sweep is the damping of
    Salvini & Wijnholds (2014), which stops the simultaneous update from
    oscillating between two points.  Returns (g, losses) with losses[t] the
    loss of the gains entering sweep t + 1."""
    g = np.array(g0, np.complex128)
    losses = []
    for t in range(1, n_iter + 1):
        losses.append(calib_loss(V, M, g))
        h = calib_als_target(V, M, g, n_threads)
        g = h if t % 2 == 1 else 0.5 * (g + h)
    return g, np.array(losses)


# ---- per-channel gains ----------------------------------------------------
# The same fit with one complex gain per input AND channel: g_k(nu).  The
# channels then decouple, so the definition is the single-channel problem
# above applied to every channel with that channel's gains:
#     L(G) = sum_nu L_nu(G[nu]),  L_nu the loss above over channel nu alone,
# and the gradient and the alternating least-squares target of channel nu
# are those of L_nu.  G, gradients and targets are complex [n_chan, N].
def _chan_args(V, M, G):
    V = np.ascontiguousarray(V, np.complex128)
    M = np.ascontiguousarray(M, np.complex128)
    G = np.ascontiguousarray(G, np.complex128)
    C, B = V.shape
    N = G.shape[1]
    assert G.shape == (C, N) and B == N * (N + 1) // 2 and M.shape == V.shape
    return V, M, G, C


def calib_chan_loss(V, M, G) -> float:
    """FP64 loss with per-channel gains G [n_chan, N]."""
    V, M, G, C = _chan_args(V, M, G)
    return float(sum(calib_loss(V[c:c + 1], M[c:c + 1], G[c]) for c in range(C)))


def calib_chan_grad(V, M, G, n_threads: int | None = None) -> np.ndarray:
    """FP64 gradient 2 dL/d conj(G), complex [n_chan, N]."""
    V, M, G, C = _chan_args(V, M, G)
    return np.stack([calib_grad(V[c:c + 1], M[c:c + 1], G[c], n_threads) for c in range(C)])


def calib_chan_als_target(V, M, G, n_threads: int | None = None) -> np.ndarray:
    """FP64 alternating least-squares target per channel, complex [n_chan, N]."""
    V, M, G, C = _chan_args(V, M, G)
    return np.stack([calib_als_target(V[c:c + 1], M[c:c + 1], G[c], n_threads)
                     for c in range(C)])


def calib_chan_solve(V, M, G0, n_iter: int, n_threads: int | None = None):
    """FP64 per-channel gain solve: the sweeps of ``calib_solve`` (plain
    target on odd sweeps, average with the previous gains on even ones) with
    the per-channel target.  Returns (G, losses), losses[t] the total loss of
    the gains entering sweep t + 1."""
    G = np.array(G0, np.complex128)
    losses = []
    for t in range(1, n_iter + 1):
        losses.append(calib_chan_loss(V, M, G))
        H = calib_chan_als_target(V, M, G, n_threads)
        G = H if t % 2 == 1 else 0.5 * (G + H)
    return G, np.array(losses)


# ---- full 2x2 Jones matrices per tile ---------------------------------------
# Inputs 2a and 2a + 1 are the two polarisations of tile a.  With one 2x2
# complex Jones matrix J_a per tile (frequency independent), the measurement
# of tile pair a > b is the 2x2 block V_ab[p][q] = V_{2a+p, 2b+q} (all four
# entries in the stored lower triangle), modelled as J_a M_ab J_b^H:
#     R_ab = J_a M_ab J_b^H - V_ab,   L = sum_nu sum_{a>b} ||R_ab||_F^2
# (blocks of a tile with itself, which hold the autocorrelations, are left
# out).  Gradient (2 dL/d conj(J_a), the PyTorch convention):
#     grad_a = 2 [ sum_{b<a} R_ab J_b M_ab^H + sum_{c>a} R_ca^H J_c M_ca ].
# Alternating least squares: with the other matrices fixed, L is a linear
# least-squares problem in J_a, sum_k ||J_a B_k - W_k||^2 with
# (B, W) = (M_ab J_b^H, V_ab) for b < a and (M_ca^H J_c^H, V_ca^H) for c > a,
# minimised by H_a = (sum W B^H)(sum B B^H)^-1 (H_a = J_a where sum B B^H is
# singular).  J, gradients and targets are complex [n_tiles, 2, 2].
def _jones_blocks(n_tiles):
    """(a, b, idx): tile pairs a > b and the baseline index of block entry (p, q)."""
    a, b = np.tril_indices(n_tiles, -1)
    i = 2 * a[:, None, None] + np.arange(2)[None, :, None]
    j = 2 * b[:, None, None] + np.arange(2)[None, None, :]
    return a, b, i * (i + 1) // 2 + j


def _jones_args(V, M, J):
    V = np.asarray(V, np.complex128)
    M = np.asarray(M, np.complex128)
    J = np.ascontiguousarray(J, np.complex128)
    n_tiles = J.shape[0]
    N = 2 * n_tiles
    assert J.shape == (n_tiles, 2, 2) and V.shape[1] == N * (N + 1) // 2 and M.shape == V.shape
    return V, M, J


def _herm(X):
    return np.conj(np.swapaxes(X, -1, -2))


def calib_jones_loss(V, M, J) -> float:
    """FP64 loss of per-tile Jones matrices J [n_tiles, 2, 2]."""
    V, M, J = _jones_args(V, M, J)
    a, b, idx = _jones_blocks(J.shape[0])
    L = 0.0
    for c in range(V.shape[0]):
        R = J[a] @ M[c][idx] @ _herm(J[b]) - V[c][idx]
        L += float(np.sum(np.abs(R) ** 2))
    return L


def calib_jones_grad(V, M, J) -> np.ndarray:
    """FP64 gradient 2 dL/d conj(J), complex [n_tiles, 2, 2]."""
    V, M, J = _jones_args(V, M, J)
    a, b, idx = _jones_blocks(J.shape[0])
    G = np.zeros_like(J)
    for c in range(V.shape[0]):
        Mb = M[c][idx]
        R = J[a] @ Mb @ _herm(J[b]) - V[c][idx]
        np.add.at(G, a, R @ J[b] @ _herm(Mb))
        np.add.at(G, b, _herm(R) @ J[a] @ Mb)
    return 2.0 * G


def calib_jones_als_target(V, M, J) -> np.ndarray:
    """FP64 alternating least-squares target H, complex [n_tiles, 2, 2]."""
    V, M, J = _jones_args(V, M, J)
    a, b, idx = _jones_blocks(J.shape[0])
    num = np.zeros_like(J)
    den = np.zeros_like(J)
    for c in range(V.shape[0]):
        Mb, Vb = M[c][idx], V[c][idx]
        Bl = Mb @ _herm(J[b])            # J_a B - V_ab, for tile a
        Bh = _herm(Mb) @ _herm(J[a])     # J_b B - V_ab^H, for tile b
        np.add.at(num, a, Vb @ _herm(Bl))
        np.add.at(den, a, Bl @ _herm(Bl))
        np.add.at(num, b, _herm(Vb) @ _herm(Bh))
        np.add.at(den, b, Bh @ _herm(Bh))
    H = J.copy()
    for t in range(J.shape[0]):
        if abs(np.linalg.det(den[t])) > 0.0:
            H[t] = num[t] @ np.linalg.inv(den[t])
    return H


def calib_jones_solve(V, M, J0, n_iter: int):
    """FP64 Jones solve: the sweeps of ``calib_solve`` (plain target on odd
    sweeps, average with the previous matrices on even ones) with the Jones
    target.  Returns (J, losses), losses[t] the loss entering sweep t + 1."""
    J = np.array(J0, np.complex128)
    losses = []
    for t in range(1, n_iter + 1):
        losses.append(calib_jones_loss(V, M, J))
        H = calib_jones_als_target(V, M, J)
        J = H if t % 2 == 1 else 0.5 * (J + H)
    return J, np.array(losses)


def _grid_args(tile_xy, vis):
    tile_xy = np.ascontiguousarray(tile_xy, np.float64)
    vis = np.ascontiguousarray(vis, np.int32)
    n_tiles = tile_xy.shape[0]
    N = 2 * n_tiles
    assert tile_xy.shape == (n_tiles, 2) and vis.ndim == 3 and vis.shape[1:] == (N * (N + 1) // 2, 2)
    return tile_xy, vis, n_tiles, vis.shape[0]


def grid(tile_xy, vis, f0, df, Ng, du, W, sigma) -> np.ndarray:
    """FP64 gridding of correlator output onto four polarisation grids,
    complex128 [4, Ng, Ng] (index 2p + q for product p, q; 0 = X, 1 = Y).
    tile_xy: [n_tiles, 2] metres; vis: int32 [n_chan, N(N+1)/2, 2], N = 2 n_tiles."""
    tile_xy, vis, n_tiles, n_chan = _grid_args(tile_xy, vis)
    out = np.zeros((4, Ng, Ng, 2), np.float64)
    _load().oracle_grid(tile_xy.ctypes.data, n_tiles, n_chan, f0, df, Ng, du, W, sigma,
                        vis.ctypes.data, out.ctypes.data)
    return out[..., 0] + 1j * out[..., 1]


def grid_cell(tile_xy, vis, f0, df, Ng, du, W, sigma, pol, r, s) -> complex:
    """One cell of grid ``pol`` computed from every point directly."""
    tile_xy, vis, n_tiles, n_chan = _grid_args(tile_xy, vis)
    val = np.zeros(2, np.float64)
    _load().oracle_grid_cell(tile_xy.ctypes.data, n_tiles, n_chan, f0, df, Ng, du, W, sigma,
                             vis.ctypes.data, pol, r, s, val.ctypes.data)
    return complex(val[0], val[1])


def stokes(inst, dl, chi, pixels=None):
    """FP64 Stokes conversion of four instrumental-polarisation images.

    Paper Sec. 2.1: the instrumental polarisation images are turned into
    Stokes I, Q, U, V by a 4x4 matrix that depends on time and sky position
    and is computed for every pixel.  Definition used (the paper gives no
    beam model): pixel (r, c) of an n x n slant-orthographic image has
    direction cosines l = (c - n/2) dl, m = (r - n/2) dl; with
    rho = sqrt(l^2 + m^2) < 1, cos(theta) = sqrt(1 - rho^2) and
    phi = atan2(m, l) + chi (chi: the parallactic rotation at the time), the
    ideal crossed-dipole response is
        J = [[cos(theta) cos(phi), -sin(phi)],
             [cos(theta) sin(phi),  cos(phi)]]
    (rows X, Y dipole; columns theta, phi sky components).  The instrumental
    coherency C = [[XX, XY], [YX, YY]] gives the sky brightness
    B = J^-1 C J^-H, and I = B00 + B11, Q = B00 - B11, U = B01 + B10,
    V = -i (B01 - B10).  Pixels with rho >= 1 (horizon and below) are zero.

    inst: complex [4, n, n] (XX, XY, YX, YY); returns complex [4, n, n]
    (I, Q, U, V).  With ``pixels`` (a list of (r, c)) only those pixels are
    converted (the others stay zero)."""
    inst = np.asarray(inst, np.complex128)
    n = inst.shape[-1]
    assert inst.shape == (4, n, n)
    idx = np.arange(n) - n / 2
    l = idx[None, :] * dl
    m = idx[:, None] * dl
    l, m = np.broadcast_arrays(l, m)
    rho = np.sqrt(l * l + m * m)
    up = rho < 1.0
    out = np.zeros_like(inst)
    todo = zip(*np.nonzero(up)) if pixels is None else [(r, c) for r, c in pixels if up[r, c]]
    for r, c in todo:
        ct = np.sqrt(1.0 - rho[r, c] ** 2)
        ph = np.arctan2(m[r, c], l[r, c]) + chi
        J = np.array([[ct * np.cos(ph), -np.sin(ph)], [ct * np.sin(ph), np.cos(ph)]])
        Ji = np.linalg.inv(J)
        C = np.array([[inst[0, r, c], inst[1, r, c]], [inst[2, r, c], inst[3, r, c]]])
        Bm = Ji @ C @ Ji.conj().T
        out[:, r, c] = [Bm[0, 0] + Bm[1, 1], Bm[0, 0] - Bm[1, 1], Bm[0, 1] + Bm[1, 0],
                        -1j * (Bm[0, 1] - Bm[1, 0])]
    return out
