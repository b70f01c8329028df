"""GB300-native MWA X-engine correlator: thin Python binding of libmwax.so.

The work is the X-engine of the real-time system described in "GPUs for data
processing in the MWA" (Sec. 2): every pair of channelised antenna inputs is
cross-correlated per fine channel and integrated, V_ij = sum_t x_i conj(x_j),
followed by the gain-calibration loss that consumes the visibilities.  Every
step runs in the library's CUDA kernels; this module only marshals
arguments (device pointers from torch tensors, the current CUDA stream) and
raises on a non-OK status.  There is no CPU fallback: without the built
library every call raises.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

LIB_PATH = _build.LIB

MWAX_OK = 0
STATUS = {0: "MWAX_OK", 1: "MWAX_ERR_INVALID_ARG", 2: "MWAX_ERR_SHAPE_MISMATCH",
          3: "MWAX_ERR_OVERFLOW_BOUND", 4: "MWAX_ERR_UNSUPPORTED", 5: "MWAX_ERR_OOM",
          6: "MWAX_ERR_CUDA", 7: "MWAX_ERR_TIMEOUT"}
STATUS_BY_NAME = {v: k for k, v in STATUS.items()}
KIND_EXACT, KIND_FP16 = 0, 1
ENGINE_TENSOR, ENGINE_PLAIN = 0, 1


class MwaxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_status_string(status)})")


class Job(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int32), ("n_chan", ctypes.c_int32),
                ("n_time", ctypes.c_int32), ("sample_bits", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("flush_blocks", ctypes.c_int32), ("chan_group", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("prefetch", ctypes.c_int32),
                ("mma_shape", ctypes.c_int32), ("pipeline", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("test_fault", ctypes.c_int32),
                ("unpack_sms", ctypes.c_int32), ("k_split", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_jobs", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("samples_per_block", ctypes.c_int32), ("flush_blocks", ctypes.c_int32),
                ("chan_group", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("prefetch", ctypes.c_int32),
                ("mma_shape", ctypes.c_int32), ("pipeline", ctypes.c_int32),
                ("scratch_bytes", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("checked_segment", ctypes.c_int32), ("k_split", ctypes.c_int32)]


class Timing(ctypes.Structure):
    _fields_ = [("unpack_ms", ctypes.c_double), ("correlate_ms", ctypes.c_double),
                ("unpack_launches", ctypes.c_int64), ("correlate_launches", ctypes.c_int64),
                ("h2d_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("h2d_copies", ctypes.c_int64), ("d2h_copies", ctypes.c_int64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64

# name -> (restype, argtypes); the exported C ABI of include/mwax.h
SIGNATURES = {
    "mwax_plan": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Job), _P]),
    "mwax_plan_batch": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Job), _I, _P]),
    "mwax_destroy": (_I, [_P]),
    "mwax_plan_get_info": (_I, [_P, ctypes.POINTER(PlanInfo)]),
    "mwax_plan_status": (_I, [_P]),
    "mwax_plan_recomputed_channels": (_I, [_P, ctypes.POINTER(_I64)]),
    "mwax_pair_work_list": (_I64, [_I, _I, _P, _I64]),
    "mwax_plan_set_timing": (_I, [_P, _I]),
    "mwax_plan_get_timing": (_I, [_P, ctypes.POINTER(Timing)]),
    "mwax_autotune": (_I, [ctypes.POINTER(Job), _P, _P, _P, ctypes.POINTER(TuneReport)]),
    "mwax_autotune_batch": (_I, [ctypes.POINTER(Job), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P,
                                 ctypes.POINTER(TuneReport)]),
    "mwax_correlate": (_I, [_P, _P, _I, _I, _I, _P]),
    "mwax_correlate_batch": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "mwax_correlate_host": (_I, [_P, _P, _I, _I, _I, _P]),
    "mwax_n_baselines": (_I64, [_I]),
    "mwax_baseline_index": (_I64, [_I, _I]),
    "mwax_baseline_pair": (_I, [_I64, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mwax_max_n_time": (_I64, [_I]),
    "mwax_status_string": (ctypes.c_char_p, [_I]),
    "mwax_calib_workspace_bytes": (_I64, [_I, _I]),
    "mwax_calib_loss": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    "mwax_calib_grad": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    "mwax_calib_loss_grad": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "mwax_calib_solve_workspace_bytes": (_I64, [_I, _I]),
    "mwax_calib_solve": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "mwax_calib_chan_workspace_bytes": (_I64, [_I, _I]),
    "mwax_calib_chan_solve_workspace_bytes": (_I64, [_I, _I]),
    "mwax_calib_chan_loss_grad": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "mwax_calib_chan_solve": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "mwax_calib_jones_workspace_bytes": (_I64, [_I, _I]),
    "mwax_calib_jones_loss_grad": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "mwax_calib_jones_solve": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "mwax_grid_plan": (_I, [_P, _P, _I, _I, ctypes.c_double, ctypes.c_double, _I, ctypes.c_double,
                            _I, ctypes.c_double, _P]),
    "mwax_grid": (_I, [_P, _P, _P]),
    "mwax_grid_plan_points": (_I64, [_P]),
    "mwax_grid_plan_entries": (_I64, [_P]),
    "mwax_grid_destroy": (_I, [_P]),
    "mwax_stokes": (_I, [_P, _I, ctypes.c_double, ctypes.c_double, _P, _P]),
    "mwax_calib_static_workspace_bytes": (_I64, []),
    "mwax_calib_loss_grad_static": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
}


def ensure_built() -> str:
    """Build libmwax.so for sm_103a if it is missing or stale."""
    return _build.build()


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built "
                               "(paper_0902_0915_gb300.ensure_built()); there is no fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _status_string(s: int) -> str:
    try:
        return lib().mwax_status_string(s).decode()
    except Exception:
        return "?"


def _check(status: int, where: str) -> None:
    if status != MWAX_OK:
        raise MwaxError(status, where)


# ---- baseline helpers --------------------------------------------------------
def n_baselines(n_inputs: int) -> int:
    return int(lib().mwax_n_baselines(n_inputs))


def baseline_index(i: int, j: int) -> int:
    return int(lib().mwax_baseline_index(i, j))


def baseline_pair(b: int):
    i, j = _I(), _I()
    _check(lib().mwax_baseline_pair(b, ctypes.byref(i), ctypes.byref(j)), "mwax_baseline_pair")
    return i.value, j.value


def max_n_time(sample_bits: int) -> int:
    return int(lib().mwax_max_n_time(sample_bits))


def pair_work_list(n_tiles: int, n_chan: int):
    """The pair-mode work list of one job (host only): rows (type, c0, I0, J0,
    c1, I1, J1), see mwax_pair_work_list."""
    import numpy as np

    n = int(lib().mwax_pair_work_list(n_tiles, n_chan, None, 0))
    if n < 0:
        raise ValueError("bad work-list shape")
    out = np.zeros((max(n, 1), 7), np.int32)
    lib().mwax_pair_work_list(n_tiles, n_chan, out.ctypes.data, n)
    return out[:n]


# ---- torch plumbing ---------------------------------------------------------------
def _torch():
    import torch

    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _job(n_inputs, n_chan, n_time, sample_bits, kind=KIND_EXACT, engine=ENGINE_TENSOR,
         flush_blocks=0, chan_group=0, stages=0, prefetch=0, mma_shape=0, pipeline=0,
         timeout_ms=0, test_fault=0, unpack_sms=0, k_split=0) -> Job:
    j = Job()
    j.n_inputs, j.n_chan, j.n_time, j.sample_bits = n_inputs, n_chan, n_time, sample_bits
    j.kind, j.engine, j.flush_blocks, j.chan_group = kind, engine, flush_blocks, chan_group
    j.stages, j.prefetch, j.mma_shape, j.pipeline = stages, prefetch, mma_shape, pipeline
    j.timeout_ms, j.test_fault, j.unpack_sms, j.k_split = timeout_ms, test_fault, unpack_sms, k_split
    return j


class Plan:
    """A correlation plan for one job (see include/mwax.h: mwax_plan).

    voltages: CUDA uint8 tensor holding [n_chan][n_time][n_inputs] packed
    samples (1 byte per complex sample for 4-bit, 2 bytes for 8-bit).
    Output: int32 (exact) or float32 (FP16 kind) tensor
    [n_chan, N(N+1)/2, 2] (re, im)."""

    def __init__(self, n_inputs, n_chan, n_time, sample_bits, kind=KIND_EXACT,
                 engine=ENGINE_TENSOR, flush_blocks=0, chan_group=0, stages=0, prefetch=0,
                 mma_shape=0, pipeline=0, timeout_ms=0, test_fault=0, unpack_sms=0,
                 k_split=0, stream=None):
        self.job = _job(n_inputs, n_chan, n_time, sample_bits, kind, engine, flush_blocks,
                        chan_group, stages, prefetch, mma_shape, pipeline, timeout_ms, test_fault,
                        unpack_sms, k_split)
        self.shape = (n_inputs, n_chan, n_time)
        self.sample_bits, self.kind, self.engine = sample_bits, kind, engine
        self._h = _P()
        self.stream = stream if stream is not None else _torch().cuda.current_stream()
        _check(lib().mwax_plan(ctypes.byref(self._h), ctypes.byref(self.job), self.stream.cuda_stream),
               "mwax_plan")

    @property
    def n_bl(self) -> int:
        return self.shape[0] * (self.shape[0] + 1) // 2

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(lib().mwax_plan_get_info(self._h, ctypes.byref(inf)), "mwax_plan_get_info")
        return inf

    def empty_out(self, device=None):
        torch = _torch()
        dt = torch.int32 if self.kind == KIND_EXACT else torch.float32
        return torch.empty((self.shape[1], self.n_bl, 2), dtype=dt,
                           device=device or torch.device("cuda", torch.cuda.current_device()))

    def correlate(self, voltages, out=None):
        """Asynchronous on the plan's stream; returns ``out``."""
        torch = _torch()
        n, c, t = self.shape
        bps = 1 if self.sample_bits == 4 else 2
        if voltages.dtype != torch.uint8 or not voltages.is_cuda or not voltages.is_contiguous():
            raise ValueError("voltages must be a contiguous CUDA uint8 tensor")
        if voltages.numel() != n * c * t * bps:
            raise ValueError("voltages size does not match the plan shape")
        if out is None:
            out = self.empty_out(voltages.device)
        _check(lib().mwax_correlate(self._h, voltages.data_ptr(), n, c, t, out.data_ptr()),
               "mwax_correlate")
        return out

    def correlate_host(self, voltages_host, out_host):
        """Host buffers (numpy or CPU tensors, ideally pinned); synchronous."""
        n, c, t = self.shape
        vp = voltages_host.ctypes.data if hasattr(voltages_host, "ctypes") else voltages_host.data_ptr()
        op = out_host.ctypes.data if hasattr(out_host, "ctypes") else out_host.data_ptr()
        _check(lib().mwax_correlate_host(self._h, vp, n, c, t, op), "mwax_correlate_host")
        return out_host

    def status(self) -> int:
        """Device status word of the last calls (synchronises the stream)."""
        return int(lib().mwax_plan_status(self._h))

    def recomputed_channels(self) -> int:
        """Channels recomputed with exact segments since the last read (plans
        with a checked single segment; synchronises the stream)."""
        n = ctypes.c_int64(0)
        _check(lib().mwax_plan_recomputed_channels(self._h, ctypes.byref(n)),
               "mwax_plan_recomputed_channels")
        return int(n.value)

    def set_timing(self, on: bool = True) -> None:
        _check(lib().mwax_plan_set_timing(self._h, 1 if on else 0), "mwax_plan_set_timing")

    def timing(self) -> Timing:
        t = Timing()
        _check(lib().mwax_plan_get_timing(self._h, ctypes.byref(t)), "mwax_plan_get_timing")
        return t

    def close(self):
        if self._h:
            lib().mwax_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GridPlan:
    """Gridding of correlator output onto four polarisation uv grids
    (mwax_grid_plan / mwax_grid).  tile_xy: [n_tiles, 2] metres."""

    def __init__(self, tile_xy, n_chan: int, f0: float, df: float, Ng: int, du: float, W: int = 7,
                 sigma: float = 1.0, stream=None):
        import numpy as np

        torch = _torch()
        xy = np.ascontiguousarray(tile_xy, np.float64)
        if xy.ndim != 2 or xy.shape[1] != 2:
            raise ValueError("tile_xy must be [n_tiles, 2]")
        self.n_tiles, self.n_chan, self.Ng = xy.shape[0], n_chan, Ng
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib().mwax_grid_plan(ctypes.byref(h), xy.ctypes.data, self.n_tiles, n_chan, f0, df, Ng,
                                    du, W, sigma, self._stream.cuda_stream), "mwax_grid_plan")
        self._h = h.value

    @property
    def n_points(self) -> int:
        return int(lib().mwax_grid_plan_points(self._h))

    @property
    def n_entries(self) -> int:
        """Stored weight factors (4 bytes each: 12 per patch candidate)."""
        return int(lib().mwax_grid_plan_entries(self._h))

    def empty_grids(self):
        torch = _torch()
        return torch.empty((4, self.Ng, self.Ng), dtype=torch.complex64, device="cuda")

    def grid(self, vis, grids=None):
        """vis: int32 CUDA tensor [n_chan, N(N+1)/2, 2] (N = 2 n_tiles), the
        correlator's output; returns complex64 [4, Ng, Ng] (index 2p + q)."""
        torch = _torch()
        N = 2 * self.n_tiles
        if not vis.is_cuda or vis.dtype != torch.int32 or vis.shape != (self.n_chan, N * (N + 1) // 2, 2):
            raise ValueError("vis must be int32 CUDA [n_chan, N(N+1)/2, 2] with N = 2 n_tiles")
        vis = vis.contiguous()
        if grids is None:
            grids = self.empty_grids()
        _check(lib().mwax_grid(self._h, vis.data_ptr(), torch.view_as_real(grids).data_ptr()),
               "mwax_grid")
        return grids

    def close(self):
        if getattr(self, "_h", None):
            lib().mwax_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stokes(inst, dl: float, chi: float, out=None):
    """Per-pixel Stokes conversion (mwax_stokes): inst complex64 CUDA
    [4, n, n] (XX, XY, YX, YY) -> complex64 [4, n, n] (I, Q, U, V)."""
    torch = _torch()
    if not inst.is_cuda or inst.dtype != torch.complex64 or inst.ndim != 3 or inst.shape[0] != 4 \
            or inst.shape[1] != inst.shape[2]:
        raise ValueError("inst must be complex64 CUDA [4, n, n]")
    inst = inst.contiguous()
    n = inst.shape[1]
    if out is None:
        out = torch.empty_like(inst)
    _check(lib().mwax_stokes(torch.view_as_real(inst).data_ptr(), n, dl, chi,
                             torch.view_as_real(out).data_ptr(), _stream_handle()), "mwax_stokes")
    return out


class BatchPlan:
    """Several uneven jobs correlated by one persistent launch per call,
    replayed from a CUDA graph (see include/mwax.h: mwax_plan_batch)."""

    def __init__(self, jobs, sample_bits=4, kind=KIND_EXACT, stream=None, mma_shape=0, stages=0,
                 prefetch=0, k_split=None):
        """jobs: (n_inputs, n_chan, n_time) per job; k_split: None (every job
        automatic) or one value per job (see mwax_job.k_split)."""
        self.shapes = [tuple(j) for j in jobs]
        self.sample_bits, self.kind = sample_bits, kind
        ks = [0] * len(jobs) if k_split is None else list(k_split)
        if len(ks) != len(jobs):
            raise ValueError("k_split needs one value per job")
        arr = (Job * len(jobs))(*[_job(n, c, t, sample_bits, kind, mma_shape=mma_shape,
                                       stages=stages, prefetch=prefetch, k_split=k)
                                  for (n, c, t), k in zip(jobs, ks)])
        self._h = _P()
        self.stream = stream if stream is not None else _torch().cuda.current_stream()
        _check(lib().mwax_plan_batch(ctypes.byref(self._h), arr, len(jobs), self.stream.cuda_stream),
               "mwax_plan_batch")

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(lib().mwax_plan_get_info(self._h, ctypes.byref(inf)), "mwax_plan_get_info")
        return inf

    def empty_outs(self, device=None):
        torch = _torch()
        dt = torch.int32 if self.kind == KIND_EXACT else torch.float32
        dev = device or torch.device("cuda", torch.cuda.current_device())
        return [torch.empty((c, n * (n + 1) // 2, 2), dtype=dt, device=dev) for (n, c, t) in self.shapes]

    def correlate(self, voltages, outs=None):
        if outs is None:
            outs = self.empty_outs(voltages[0].device)
        k = len(self.shapes)
        vin = (_P * k)(*[v.data_ptr() for v in voltages])
        vout = (_P * k)(*[o.data_ptr() for o in outs])
        _check(lib().mwax_correlate_batch(self._h, vin, vout), "mwax_correlate_batch")
        return outs

    def status(self) -> int:
        return int(lib().mwax_plan_status(self._h))

    def set_timing(self, on: bool = True) -> None:
        _check(lib().mwax_plan_set_timing(self._h, 1 if on else 0), "mwax_plan_set_timing")

    def timing(self) -> Timing:
        t = Timing()
        _check(lib().mwax_plan_get_timing(self._h, ctypes.byref(t)), "mwax_plan_get_timing")
        return t

    def close(self):
        if self._h:
            lib().mwax_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TUNE_FIELDS = ("mma_shape", "stages", "prefetch", "pipeline", "chan_group", "k_split")


def autotune(voltages, out, n_inputs, n_chan, n_time, sample_bits, kind=KIND_EXACT, stream=None):
    """Time candidate configurations on these device buffers; returns
    (dict of tuning fields, TuneReport).  See include/mwax.h: mwax_autotune."""
    j = _job(n_inputs, n_chan, n_time, sample_bits, kind)
    rep = TuneReport()
    _check(lib().mwax_autotune(ctypes.byref(j), voltages.data_ptr(), out.data_ptr(),
                               _stream_handle(stream), ctypes.byref(rep)), "mwax_autotune")
    return {k: getattr(j, k) for k in TUNE_FIELDS}, rep


def autotune_batch(jobs, voltages, outs, sample_bits=4, kind=KIND_EXACT, stream=None):
    """Batch variant: one (mma_shape, stages, prefetch) for the launch, then
    each job's k_split; returns the BatchPlan keyword arguments and the report."""
    k = len(jobs)
    arr = (Job * k)(*[_job(n, c, t, sample_bits, kind) for (n, c, t) in jobs])
    vin = (_P * k)(*[v.data_ptr() for v in voltages])
    vout = (_P * k)(*[o.data_ptr() for o in outs])
    rep = TuneReport()
    _check(lib().mwax_autotune_batch(arr, k, vin, vout, _stream_handle(stream), ctypes.byref(rep)),
           "mwax_autotune_batch")
    fields = {f: getattr(arr[0], f) for f in ("mma_shape", "stages", "prefetch")}
    fields["k_split"] = [arr[i].k_split for i in range(k)]
    return fields, rep


def correlate(voltages, n_inputs, n_chan, n_time, sample_bits, kind=KIND_EXACT,
              engine=ENGINE_TENSOR):
    """One-shot convenience: plan, correlate, destroy (synchronises)."""
    p = Plan(n_inputs, n_chan, n_time, sample_bits, kind, engine)
    out = p.correlate(voltages)
    st = p.status()
    p.close()
    _check(st, "correlate (device status)")
    return out


# ---- calibration ------------------------------------------------------------------
def calib_workspace(n_inputs: int, n_chan: int, device=None):
    torch = _torch()
    nb = int(lib().mwax_calib_workspace_bytes(n_inputs, n_chan))
    if nb < 0:
        raise ValueError("invalid calibration shape")
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


def _f32_pairs(t):
    """complex64 (or float32 [..., 2]) CUDA tensor -> contiguous float32 pairs."""
    torch = _torch()
    if not t.is_cuda:
        raise ValueError("calibration tensors must be CUDA tensors")
    t = t.contiguous()
    if t.dtype == torch.complex64:
        t = torch.view_as_real(t)
    if t.dtype != torch.float32 or t.shape[-1] != 2:
        raise ValueError("calibration tensors must be complex64 or float32 (re, im) pairs")
    return t


def calib_loss_grad(V, M, g, workspace=None, want_loss=True, want_grad=True):
    """(loss float32 scalar tensor or None, grad complex64 [N] or None).
    V, M: complex64 [n_chan, N(N+1)/2]; g: complex64 [N]."""
    torch = _torch()
    Vr, Mr, gr = _f32_pairs(V), _f32_pairs(M), _f32_pairs(g)
    n = gr.shape[0]
    c = Vr.shape[0]
    if Vr.shape != (c, n * (n + 1) // 2, 2) or Mr.shape != Vr.shape:
        raise ValueError("V, M must be [n_chan, N(N+1)/2] for N = len(g)")
    ws = workspace if workspace is not None else calib_workspace(n, c, V.device)
    loss = torch.empty((), dtype=torch.float32, device=V.device) if want_loss else None
    grad = torch.empty((n, 2), dtype=torch.float32, device=V.device) if want_grad else None
    _check(lib().mwax_calib_loss_grad(Vr.data_ptr(), Mr.data_ptr(), gr.data_ptr(), n, c,
                                      ws.data_ptr(), loss.data_ptr() if want_loss else None,
                                      grad.data_ptr() if want_grad else None,
                                      _stream_handle()), "mwax_calib_loss_grad")
    return loss, (torch.view_as_complex(grad) if want_grad else None)


def calib_solve(V, M, g0, n_iter: int, workspace=None, loss_history: bool = True):
    """Gain solve: ``n_iter`` alternating least-squares sweeps from ``g0``
    (complex64 [N], not modified).  Returns (g complex64 [N], losses float32
    [n_iter] or None) with losses[t] the loss of the gains entering sweep t+1."""
    torch = _torch()
    Vr, Mr = _f32_pairs(V), _f32_pairs(M)
    g = _f32_pairs(g0).clone()
    n = g.shape[0]
    c = Vr.shape[0]
    if Vr.shape != (c, n * (n + 1) // 2, 2) or Mr.shape != Vr.shape:
        raise ValueError("V, M must be [n_chan, N(N+1)/2] for N = len(g0)")
    if n_iter < 0:
        raise ValueError("n_iter must be >= 0")
    if workspace is None:
        nb = int(lib().mwax_calib_solve_workspace_bytes(n, c))
        if nb < 0:
            raise ValueError("invalid calibration shape")
        workspace = torch.empty(nb, dtype=torch.uint8, device=V.device)
    hist = (torch.empty(max(n_iter, 1), dtype=torch.float32, device=V.device)
            if loss_history else None)
    _check(lib().mwax_calib_solve(Vr.data_ptr(), Mr.data_ptr(), g.data_ptr(), n, c, n_iter,
                                  workspace.data_ptr(), hist.data_ptr() if hist is not None else None,
                                  _stream_handle()), "mwax_calib_solve")
    return torch.view_as_complex(g), (hist[:n_iter] if hist is not None else None)


def _chan_shapes(Vr, Mr, Gr):
    if Gr.dim() != 3:
        raise ValueError("per-channel gains must be [n_chan, N]")
    c, n = Gr.shape[0], Gr.shape[1]
    if Vr.shape != (c, n * (n + 1) // 2, 2) or Mr.shape != Vr.shape:
        raise ValueError("V, M must be [n_chan, N(N+1)/2] for G of shape [n_chan, N]")
    return n, c


def calib_chan_loss_grad(V, M, G, workspace=None, want_loss=True, want_grad=True):
    """Per-channel gains: (loss float32 scalar tensor or None, grad complex64
    [n_chan, N] or None).  V, M: complex64 [n_chan, N(N+1)/2]; G: complex64
    [n_chan, N]."""
    torch = _torch()
    Vr, Mr, Gr = _f32_pairs(V), _f32_pairs(M), _f32_pairs(G)
    n, c = _chan_shapes(Vr, Mr, Gr)
    if workspace is None:
        nb = int(lib().mwax_calib_chan_workspace_bytes(n, c))
        if nb < 0:
            raise ValueError("invalid calibration shape")
        workspace = torch.empty(nb, dtype=torch.uint8, device=V.device)
    loss = torch.empty((), dtype=torch.float32, device=V.device) if want_loss else None
    grad = torch.empty((c, n, 2), dtype=torch.float32, device=V.device) if want_grad else None
    _check(lib().mwax_calib_chan_loss_grad(Vr.data_ptr(), Mr.data_ptr(), Gr.data_ptr(), n, c,
                                           workspace.data_ptr(),
                                           loss.data_ptr() if want_loss else None,
                                           grad.data_ptr() if want_grad else None,
                                           _stream_handle()), "mwax_calib_chan_loss_grad")
    return loss, (torch.view_as_complex(grad) if want_grad else None)


def calib_chan_solve(V, M, G0, n_iter: int, workspace=None, loss_history: bool = True):
    """Per-channel gain solve: ``n_iter`` sweeps from ``G0`` (complex64
    [n_chan, N], not modified).  Returns (G complex64 [n_chan, N], losses
    float32 [n_iter] or None)."""
    torch = _torch()
    Vr, Mr = _f32_pairs(V), _f32_pairs(M)
    G = _f32_pairs(G0).clone()
    n, c = _chan_shapes(Vr, Mr, G)
    if n_iter < 0:
        raise ValueError("n_iter must be >= 0")
    if workspace is None:
        nb = int(lib().mwax_calib_chan_solve_workspace_bytes(n, c))
        if nb < 0:
            raise ValueError("invalid calibration shape")
        workspace = torch.empty(nb, dtype=torch.uint8, device=V.device)
    hist = (torch.empty(max(n_iter, 1), dtype=torch.float32, device=V.device)
            if loss_history else None)
    _check(lib().mwax_calib_chan_solve(Vr.data_ptr(), Mr.data_ptr(), G.data_ptr(), n, c, n_iter,
                                       workspace.data_ptr(),
                                       hist.data_ptr() if hist is not None else None,
                                       _stream_handle()), "mwax_calib_chan_solve")
    return torch.view_as_complex(G), (hist[:n_iter] if hist is not None else None)


def _jones_shapes(Vr, Mr, Jr):
    if Jr.dim() != 4 or Jr.shape[1:3] != (2, 2):
        raise ValueError("Jones matrices must be [n_tiles, 2, 2]")
    n = 2 * Jr.shape[0]
    c = Vr.shape[0]
    if Vr.shape != (c, n * (n + 1) // 2, 2) or Mr.shape != Vr.shape:
        raise ValueError("V, M must be [n_chan, N(N+1)/2] for N = 2 n_tiles")
    return n, c


def _jones_workspace(n, c, device):
    torch = _torch()
    nb = int(lib().mwax_calib_jones_workspace_bytes(n, c))
    if nb < 0:
        raise ValueError("invalid calibration shape")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def calib_jones_loss_grad(V, M, J, workspace=None, want_loss=True, want_grad=True):
    """Per-tile 2x2 Jones matrices: (loss float32 scalar tensor or None, grad
    complex64 [n_tiles, 2, 2] or None).  V, M: complex64 [n_chan, N(N+1)/2]
    with N = 2 n_tiles; J: complex64 [n_tiles, 2, 2]."""
    torch = _torch()
    Vr, Mr, Jr = _f32_pairs(V), _f32_pairs(M), _f32_pairs(J)
    n, c = _jones_shapes(Vr, Mr, Jr)
    ws = workspace if workspace is not None else _jones_workspace(n, c, V.device)
    loss = torch.empty((), dtype=torch.float32, device=V.device) if want_loss else None
    grad = torch.empty(Jr.shape, dtype=torch.float32, device=V.device) if want_grad else None
    _check(lib().mwax_calib_jones_loss_grad(Vr.data_ptr(), Mr.data_ptr(), Jr.data_ptr(), n, c,
                                            ws.data_ptr(), loss.data_ptr() if want_loss else None,
                                            grad.data_ptr() if want_grad else None,
                                            _stream_handle()), "mwax_calib_jones_loss_grad")
    return loss, (torch.view_as_complex(grad) if want_grad else None)


def calib_jones_solve(V, M, J0, n_iter: int, workspace=None, loss_history: bool = True):
    """Jones solve: ``n_iter`` alternating least-squares sweeps from ``J0``
    (complex64 [n_tiles, 2, 2], not modified).  Returns (J, losses float32
    [n_iter] or None)."""
    torch = _torch()
    Vr, Mr = _f32_pairs(V), _f32_pairs(M)
    Jr = _f32_pairs(J0).clone()
    n, c = _jones_shapes(Vr, Mr, Jr)
    if n_iter < 0:
        raise ValueError("n_iter must be >= 0")
    ws = workspace if workspace is not None else _jones_workspace(n, c, V.device)
    hist = (torch.empty(max(n_iter, 1), dtype=torch.float32, device=V.device)
            if loss_history else None)
    _check(lib().mwax_calib_jones_solve(Vr.data_ptr(), Mr.data_ptr(), Jr.data_ptr(), n, c, n_iter,
                                        ws.data_ptr(), hist.data_ptr() if hist is not None else None,
                                        _stream_handle()), "mwax_calib_jones_solve")
    return torch.view_as_complex(Jr), (hist[:n_iter] if hist is not None else None)


def _make_calib_function():
    torch = _torch()

    class CalibLoss(torch.autograd.Function):
        """L(g) = sum_nu sum_{i>j} |g_i conj(g_j) M_ij - V_ij|^2 with the
        hand-written forward and adjoint kernels; the gradient returned for
        g is PyTorch's complex convention dL/dRe g + i dL/dIm g.  One kernel
        pass computes both, the gradient is kept for backward.  The loss is
        differentiable in g only: V and M requiring a gradient is an error
        (their gradient would otherwise be silently dropped)."""

        @staticmethod
        def forward(ctx, g, V, M):
            if V.requires_grad or M.requires_grad:
                raise ValueError("calib_loss is differentiable in g only; "
                                 "detach V and M (their gradient is not computed)")
            # g [N]: one gain per input; g [n_chan, N]: per-channel gains
            fn = calib_chan_loss_grad if g.dim() == 2 else calib_loss_grad
            loss, grad = fn(V, M, g.detach().contiguous(), want_grad=g.requires_grad)
            ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=g.device))
            return loss

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return grad * gout, None, None

    return CalibLoss


_calib_cls = None


def calib_loss(g, V, M):
    """Differentiable calibration loss (torch.autograd.Function); g complex64
    [N] (one gain per input) or [n_chan, N] (per-channel gains)."""
    global _calib_cls
    if _calib_cls is None:
        _calib_cls = _make_calib_function()
    return _calib_cls.apply(g, V, M)
