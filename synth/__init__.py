"""Seeded synthetic channelised voltages: the input generator shared by the
oracle side and the CUDA side.

This module holds no correlation, integration or calibration arithmetic.  It
produces packed complex samples ``voltages[chan][time][input]`` (4+4-bit: one
byte, low nibble re / high nibble im; 8+8-bit: two int8 bytes re, im) from a
counter-based generator (Philox4x64-10) so that any subset of channels can be
regenerated on the host bit-identically to a multi-GB device fill.

Workload recipes follow the shapes of the MWA correlator the paper sizes
(512 antennas, 768 channels, 4 polarisation products; Sec. 2): see
``WORKLOADS``.  Where the paper is silent (noise level, tone, sources,
geometry) the recipe is this module's choice and is stated with it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
HOST_LIB = os.path.join(_LIBDIR, "libsynth_host.so")
CUDA_LIB = os.path.join(_LIBDIR, "libsynth_cuda.so")

SYNTH_NOISE_TONE, SYNTH_SOURCES, SYNTH_CONST, SYNTH_BIGSMALL, SYNTH_RANDMAX, SYNTH_QUARTER = range(6)
TABLE_SIZE = 4096
C_LIGHT = 299792458.0


# --------------------------------------------------------------------------
# build
# --------------------------------------------------------------------------
def build_commands(arch: str = "sm_103a"):
    """Compiler command lines for the two generator libraries."""
    os.makedirs(_LIBDIR, exist_ok=True)
    host = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall",
            os.path.join(_HERE, "synth_host.c"), "-o", HOST_LIB]
    comp = arch.replace("sm_", "compute_")
    cuda = ["nvcc", "-O3", "-gencode", f"arch={comp},code={arch}", "-Xcompiler", "-fPIC",
            "-shared", os.path.join(_HERE, "synth_cuda.cu"), "-o", CUDA_LIB]
    return [host, cuda]


def build(verbose: bool = False) -> None:
    cmds = build_commands()
    with ThreadPoolExecutor(len(cmds)) as ex:
        res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds))
    for c, r in zip(cmds, res):
        if r.returncode != 0:
            raise RuntimeError(f"synth build failed: {' '.join(c)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)


# --------------------------------------------------------------------------
# parameter block (mirrors synth_params in synth.h)
# --------------------------------------------------------------------------
class SynthParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("kind", ctypes.c_int32),
        ("sample_bits", ctypes.c_int32),
        ("n_inputs", ctypes.c_int32),
        ("n_time", ctypes.c_int32),
        ("sigma", ctypes.c_int32),
        ("tone_amp_q16", ctypes.c_int32),
        ("n_src", ctypes.c_int32),
        ("chan_base", ctypes.c_int32),
        ("c_re", ctypes.c_int32),
        ("c_im", ctypes.c_int32),
        ("t_split", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("cos_q16", ctypes.c_void_p),
        ("src_amp_q16", ctypes.c_void_p),
        ("src_rate", ctypes.c_void_p),
        ("ci", ctypes.c_void_p),
        ("gain_q16", ctypes.c_void_p),
    ]


def cos_table_q16() -> np.ndarray:
    """round(65536 * cos(2 pi k / 4096)), k = 0..4095 (int32)."""
    k = np.arange(TABLE_SIZE, dtype=np.float64)
    return np.round(65536.0 * np.cos(2.0 * np.pi * k / TABLE_SIZE)).astype(np.int32)


@dataclass
class Spec:
    """One synthetic voltage set: shape plus generation recipe."""
    name: str
    n_inputs: int
    n_chan: int
    n_time: int
    sample_bits: int
    seed: int
    kind: int = SYNTH_NOISE_TONE
    sigma: int = 2
    tone_amp: float = 0.0          # sample units
    n_src: int = 0
    src_amp: tuple = ()            # sample units, len n_src
    chan_base: int = 0
    c_re: int = 0
    c_im: int = 0
    t_split: int = 0
    ci: np.ndarray | None = None   # SYNTH_QUARTER [n_inputs, 2]
    gains: np.ndarray | None = None  # complex128 [n_inputs], applied to the source sum
    src_rate: np.ndarray | None = None  # uint32 [n_inputs, n_src]
    src_flux: np.ndarray | None = None  # float64 [n_src] (calibration model)
    chan_width_hz: float = 40e3
    meta: dict = field(default_factory=dict)

    @property
    def vmax(self) -> int:
        return 7 if self.sample_bits == 4 else 127

    @property
    def bytes_per_sample(self) -> int:
        return 1 if self.sample_bits == 4 else 2

    def tables(self) -> dict:
        """Host arrays referenced by the parameter block."""
        t = {"cos_q16": cos_table_q16()}
        if self.kind == SYNTH_SOURCES:
            t["src_amp_q16"] = np.round(np.asarray(self.src_amp, np.float64) * 65536.0).astype(np.int32)
            t["src_rate"] = np.ascontiguousarray(self.src_rate, dtype=np.uint32)
            if self.gains is not None:
                g = np.asarray(self.gains, np.complex128)
                gq = np.stack([np.round(g.real * 65536.0), np.round(g.imag * 65536.0)], axis=1)
                t["gain_q16"] = np.ascontiguousarray(gq.astype(np.int32))
        if self.kind == SYNTH_QUARTER:
            t["ci"] = np.ascontiguousarray(np.asarray(self.ci, np.int32).reshape(self.n_inputs, 2))
        return t

    def params(self, tables: dict, ptr) -> SynthParams:
        """Parameter block whose table pointers come from ptr(array)."""
        p = SynthParams()
        p.seed = self.seed
        p.kind = self.kind
        p.sample_bits = self.sample_bits
        p.n_inputs = self.n_inputs
        p.n_time = self.n_time
        p.sigma = self.sigma
        p.tone_amp_q16 = int(round(self.tone_amp * 65536.0))
        p.n_src = self.n_src
        p.chan_base = self.chan_base
        p.c_re, p.c_im, p.t_split = self.c_re, self.c_im, self.t_split
        for k in ("cos_q16", "src_amp_q16", "src_rate", "ci", "gain_q16"):
            setattr(p, k, ptr(tables[k]) if k in tables else None)
        return p

    def with_(self, **kw) -> "Spec":
        d = dict(self.__dict__)
        d.update(kw)
        return Spec(**d)


# --------------------------------------------------------------------------
# geometry for point sources (Sec. 2: antenna gains and source positions)
# --------------------------------------------------------------------------
def source_geometry(n_inputs: int, n_src: int, seed: int, chan_width_hz: float,
                    radius_m: float = 750.0, lm_radius: float = 0.5):
    """Seeded tile positions (uniform in a disc of radius ``radius_m``; the
    two polarisations of a tile share its position) and source direction
    cosines (uniform in a disc of radius ``lm_radius``).  Returns the phase
    advance per channel step, uint32 turns, [n_inputs, n_src]:
    rate = frac((u l + v m) / c * chan_width) * 2^32."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    n_tiles = (n_inputs + 1) // 2

    def disc(n, r):
        out = np.empty((0, 2))
        while len(out) < n:
            p = rng.uniform(-1.0, 1.0, size=(2 * n, 2))
            p = p[(p ** 2).sum(1) <= 1.0]
            out = np.concatenate([out, p])
        return out[:n] * r

    uv = disc(n_tiles, radius_m)
    lm = disc(n_src, lm_radius)
    tau = (uv @ lm.T) / C_LIGHT  # seconds [tiles, src]
    turns = tau * chan_width_hz
    frac = turns - np.floor(turns)
    rate_tile = np.floor(frac * 2.0 ** 32).astype(np.uint64) % (2 ** 32)
    rate = np.repeat(rate_tile, 2, axis=0)[:n_inputs].astype(np.uint32)
    return np.ascontiguousarray(rate), uv, lm


def grid_geometry_c1():
    """Inputs of the gridding workload that consumes the c1 correlation: the
    c1 tile positions (metres, [128, 2]), the first channel's frequency and the
    channel width (Hz): 768 channels of 40 kHz from 167.04 MHz (30.72 MHz, the
    MWA's high band), and the grid: 2048 x 2048 cells of 1 wavelength (every
    baseline of the 1.5 km array fits), support 7 cells, Gaussian width 1 cell."""
    _, uv, _ = source_geometry(256, 5, 1, 40e3)
    return {"tile_xy": np.ascontiguousarray(uv, np.float64), "f0": 167.04e6, "df": 40e3,
            "Ng": 2048, "du": 1.0, "W": 7, "sigma": 1.0}


# --------------------------------------------------------------------------
# workloads (shapes of the MWA correlator, Sec. 2)
# --------------------------------------------------------------------------
def spec_c0() -> Spec:
    """64 inputs x 64 channels x T=1000, 4+4-bit, sigma 2 + 0.3-amplitude
    common tone."""
    return Spec("c0", 64, 64, 1000, 4, seed=0, sigma=2, tone_amp=0.3, chan_width_hz=480e3)


def spec_c1() -> Spec:
    """256 inputs x 768 channels (40 kHz) x T=20000 (0.5 s), 4+4-bit, sigma 2
    plus 5 point sources with per-input phase gradients."""
    n_in, n_src, seed = 256, 5, 1
    rate, _, _ = source_geometry(n_in, n_src, seed, 40e3)
    rng = np.random.default_rng(np.random.PCG64(1000 + seed))
    amp = tuple(float(a) for a in rng.uniform(0.3, 1.0, n_src) * 2.0)
    return Spec("c1", n_in, 768, 20000, 4, seed=seed, kind=SYNTH_SOURCES, sigma=2,
                n_src=n_src, src_amp=amp, src_rate=rate, chan_base=3366, chan_width_hz=40e3)


def spec_c2() -> Spec:
    """1024 inputs x 3072 channels (10 kHz, 30.72 MHz) x T=10000 (1 s),
    8+8-bit, sigma 20."""
    return Spec("c2", 1024, 3072, 10000, 8, seed=2, sigma=20, chan_width_hz=10e3)


C3_JOBS = ((48, 256, 2000), (128, 768, 5000), (300, 1536, 10000), (1024, 3072, 20000))


def spec_c3(job: int) -> Spec:
    """Batched sub-array job ``job`` (0..3), 4+4-bit, sigma 2 + 0.3 tone."""
    n, c, t = C3_JOBS[job]
    return Spec(f"c3j{job}", n, c, t, 4, seed=3 + job, sigma=2, tone_amp=0.3,
                chan_width_hz=30.72e6 / c)


def spec_c4() -> Spec:
    """Calibration workload voltages: 1024 inputs x 768 channels x T=10000,
    8+8-bit.  x_i = g_i * sum_s sqrt(S_s) n_s(t) exp(i phi_is) * scale + noise,
    20 sources with flux S ~ log-uniform[0.1, 10], |g| ~ U(0.8, 1.2) with
    uniform phase, scale 3, noise sigma 10."""
    n_in, n_src, seed, scale = 1024, 20, 4, 3.0
    rate, _, _ = source_geometry(n_in, n_src, seed, 40e3)
    rng = np.random.default_rng(np.random.PCG64(1000 + seed))
    flux = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_src))
    gabs = rng.uniform(0.8, 1.2, n_in)
    gph = rng.uniform(0.0, 2.0 * np.pi, n_in)
    gains = gabs * np.exp(1j * gph)
    amp = tuple(float(a) for a in np.sqrt(flux) * scale)
    return Spec("c4", n_in, 768, 10000, 8, seed=seed, kind=SYNTH_SOURCES, sigma=10,
                n_src=n_src, src_amp=amp, src_rate=rate, gains=gains, src_flux=flux,
                chan_base=3366, chan_width_hz=40e3, meta={"scale": scale})


def model_visibilities_host(spec: Spec, chans) -> np.ndarray:
    """The calibration sky model of a point-source workload (the input the
    gain fit is made against, not part of the correlation): for channel c,
    M_ij(c) = sum_s S_s exp(i (phi_is - phi_js)) with phi_is = 2 pi
    frac(rate_is (c + chan_base) / 2^32), the same phase the generator
    applies to source s on input i.  FP64, returned as complex128
    [len(chans), N(N+1)/2] in the lower-triangle baseline order."""
    if spec.src_rate is None or spec.src_flux is None:
        raise ValueError("not a point-source workload with a flux model")
    N = spec.n_inputs
    ii, jj = np.tril_indices(N)
    rate = np.asarray(spec.src_rate, np.uint64)  # [N, S]
    flux = np.asarray(spec.src_flux, np.float64)
    out = np.empty((len(chans), ii.size), np.complex128)
    for k, c in enumerate(chans):
        turns = (rate * np.uint64(c + spec.chan_base)) % np.uint64(2 ** 32)
        e = np.exp(2j * np.pi * (turns.astype(np.float64) / 2.0 ** 32))  # [N, S]
        full = (e * flux) @ e.conj().T
        out[k] = full[ii, jj]
    return out


WORKLOADS = {"c0": spec_c0, "c1": spec_c1, "c2": spec_c2, "c4": spec_c4}


# --------------------------------------------------------------------------
# host fill
# --------------------------------------------------------------------------
_host = None
_cuda = None


def _load_host():
    global _host
    if _host is None:
        if not os.path.exists(HOST_LIB):
            raise RuntimeError(f"{HOST_LIB} missing: run synth.build()")
        lib = ctypes.CDLL(HOST_LIB)
        lib.synth_fill_host.restype = ctypes.c_int
        lib.synth_fill_host.argtypes = [ctypes.POINTER(SynthParams), ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
        lib.synth_philox_host.argtypes = [ctypes.c_void_p] * 3
        lib.synth_sample_host.argtypes = [ctypes.POINTER(SynthParams), ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        _host = lib
    return _host


def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block computed by the C generator."""
    lib = _load_host()
    c = np.ascontiguousarray(ctr, np.uint64)
    k = np.ascontiguousarray(key, np.uint64)
    o = np.zeros(4, np.uint64)
    lib.synth_philox_host(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def default_threads() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def fill_host(spec: Spec, chans=None, t0: int = 0, n_time: int | None = None,
              threads: int | None = None) -> np.ndarray:
    """Packed voltages for channels ``chans`` (default all):
    uint8 [len(chans), n_time, n_inputs * bytes_per_sample]."""
    lib = _load_host()
    if chans is None:
        chans = np.arange(spec.n_chan)
    ch = np.ascontiguousarray(chans, np.int64)
    nt = spec.n_time - t0 if n_time is None else n_time
    tabs = spec.tables()
    p = spec.params(tabs, lambda a: a.ctypes.data)
    out = np.empty((len(ch), nt, spec.n_inputs * spec.bytes_per_sample), np.uint8)
    rc = lib.synth_fill_host(ctypes.byref(p), ch.ctypes.data, len(ch), t0, nt, out.ctypes.data,
                             threads or default_threads())
    if rc != 0:
        raise RuntimeError(f"synth_fill_host failed ({rc})")
    return out


def sample_values(spec: Spec, chan: int, t: int, inp: int):
    """Unpacked (re, im) of one sample, for statistics tests."""
    lib = _load_host()
    tabs = spec.tables()
    p = spec.params(tabs, lambda a: a.ctypes.data)
    re = ctypes.c_int32()
    im = ctypes.c_int32()
    lib.synth_sample_host(ctypes.byref(p), chan, t, inp, ctypes.byref(re), ctypes.byref(im))
    return re.value, im.value


# --------------------------------------------------------------------------
# device fill (torch supplies the device memory and stream)
# --------------------------------------------------------------------------
def _load_cuda():
    global _cuda
    if _cuda is None:
        if not os.path.exists(CUDA_LIB):
            raise RuntimeError(f"{CUDA_LIB} missing: run synth.build()")
        lib = ctypes.CDLL(CUDA_LIB)
        lib.synth_fill_device.restype = ctypes.c_int
        lib.synth_fill_device.argtypes = [ctypes.POINTER(SynthParams), ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p]
        _cuda = lib
    return _cuda


def fill_device(spec: Spec, out, chan0: int = 0, n_chan: int | None = None, stream=None):
    """Fill the CUDA uint8 tensor ``out`` (>= n_chan*n_time*n_inputs*bps bytes)
    with channels chan0 .. chan0+n_chan-1.  Asynchronous on ``stream``."""
    import torch

    lib = _load_cuda()
    n_chan = spec.n_chan - chan0 if n_chan is None else n_chan
    need = n_chan * spec.n_time * spec.n_inputs * spec.bytes_per_sample
    if out.device.type != "cuda" or out.dtype != torch.uint8 or out.numel() < need:
        raise ValueError("out must be a CUDA uint8 tensor large enough for the fill")
    tabs = {k: torch.from_numpy(v).to(out.device) for k, v in spec.tables().items()}
    p = spec.params(tabs, lambda t: t.data_ptr())
    s = stream if stream is not None else torch.cuda.current_stream(out.device)
    rc = lib.synth_fill_device(ctypes.byref(p), chan0, n_chan, out.data_ptr(), s.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"synth_fill_device failed (cudaError {rc})")
    # keep the device tables alive until the fill has run
    s.synchronize()
    return out
