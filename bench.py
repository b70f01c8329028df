#!/usr/bin/env python
"""X-engine benchmark: tera complex-MAC/s and real-time factor of the
GB300 tensor-core correlator on seeded synthetic channelised voltages.

One step = one integration of the whole workload through the C ABI
(unpack + tcgen05 correlate + integration dump for every channel), inputs
resident in HBM.  Default workload: 1024 inputs (512 tiles x 2 pols) x 3072
fine channels (10 kHz, 30.72 MHz) x T = 10000 samples (1 s of sky),
8+8-bit samples, exact int32 visibilities.

Printed as one JSON line by rank 0.  ``--impl reference`` times the CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "X-engine tera complex-MAC/s & real-time factor, batched TC vs plain, bit-exact"
FULL_BAND_HZ = 30.72e6


# ---------------------------------------------------------------------------
def workloads():
    import synth

    return {
        "c2": (synth.spec_c2, "1024 inputs (512 tiles x 2 pol) x 3072 ch (10 kHz) x T=10000 (1 s), 8+8-bit"),
        "c1": (synth.spec_c1, "256 inputs x 768 ch (40 kHz) x T=20000 (0.5 s), 4+4-bit, 5 sources"),
        "c0": (synth.spec_c0, "64 inputs x 64 ch x T=1000, 4+4-bit"),
    }


def cmacs(spec) -> float:
    return spec.n_inputs * (spec.n_inputs + 1) / 2 * spec.n_chan * spec.n_time


def sky_seconds(spec) -> float:
    """T / chan_width: seconds of sampled sky per integration."""
    return spec.n_time / spec.chan_width_hz


def traffic_entry(kernel_key: str):
    """The committed ncu traffic record for a kernel and shape
    (profiles/traffic.json), or None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    return d.get(kernel_key)


def measured_traffic(kernel_key: str, channels_per_launch: int):
    """DRAM bytes per launch from the committed ncu capture, scaled by channels
    (traffic grows in proportion), or None."""
    e = traffic_entry(kernel_key)
    return None if e is None else e["bytes_per_channel"] * channels_per_launch


def unpack_bytes_per_channel(spec) -> float:
    """Algorithmic bytes the unpack moves per channel: packed samples read plus
    operand rows written ([time block][row][128 B], rows padded to 128)."""
    per_block = 32 if spec.sample_bits == 8 else 64
    kb = -(-spec.n_time // per_block)
    n_rows = -(-spec.n_inputs // 128) * 128
    packed = spec.n_inputs * spec.n_time * (2 if spec.sample_bits == 8 else 1)
    return float(packed + n_rows * kb * 128)


def unpack_kernel_name(spec) -> str:
    """The unpack kernel the plan picks for this shape: for 8-bit samples the
    TMA tile kernel where the raw rows are whole 16-byte units, else the
    fallbacks; for 4-bit samples the MN-major streaming kernel (one form,
    templated on the vector width the row length allows)."""
    n = spec.n_inputs
    if spec.sample_bits == 4:
        return f"unpack4_mn_kernel<{16 if n % 16 == 0 else 4 if n % 4 == 0 else 1}>"
    if os.environ.get("MWAX_UNPACK") is None and n % 2 == 0:
        return "unpack8_tile_kernel"
    return "unpack8_kernel"


def unpack_roofline(spec, info, tim, steps, peaks, peak_src):
    """HBM roofline of the unpack kernel (the second kernel of a step)."""
    per_ch = unpack_bytes_per_channel(spec)
    achieved = per_ch * spec.n_chan * steps / (tim.unpack_ms / 1e3) / 1e9
    peak = float(peaks["hbm_gbs"])
    traffic = measured_traffic(f"{unpack_kernel_name(spec)}|N{spec.n_inputs}|T{spec.n_time}",
                               info.chan_group)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "algorithmic_bytes_per_launch": per_ch * info.chan_group,
            "kernel": unpack_kernel_name(spec),
            "peak_source": f"HBM copy ({peak_src})",
            "ms_per_launch": tim.unpack_ms / max(1, tim.unpack_launches)}


def tensor_peak_at_clock(sample_bits: int, clk, sms: int):
    """Context for the tensor roofline: the dense MMA rate at the SM clock
    sampled during the timed region (8,192 FLOP per SM per cycle for
    kind::f16, twice that for kind::f8f6f4 E4M3), beside the measured cuBLAS
    figure, which was taken at a lower, power-capped clock."""
    if not clk or not clk.get("sm_mhz"):
        return None
    per_sm = 8192 if sample_bits == 8 else 16384
    return per_sm * sms * clk["sm_mhz"] * 1e6 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
def nvsmi_gpu_id(dev: int) -> str:
    """The id nvidia-smi knows the CUDA device `dev` by.  nvidia-smi numbers
    GPUs physically and ignores CUDA_VISIBLE_DEVICES, so a CUDA ordinal would
    name another GPU whenever the visible set is not the first GPUs of the
    machine: use the device's UUID, else the CUDA_VISIBLE_DEVICES entry."""
    try:
        import torch

        if torch.cuda.is_available():
            u = str(torch.cuda.get_device_properties(dev).uuid).strip()
            if u:
                return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
    if vis:
        entries = [x.strip() for x in vis.split(",") if x.strip()]
        if 0 <= dev < len(entries):
            return entries[dev]
    return str(dev)


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.gpu_id = nvsmi_gpu_id(index)
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self, first_sample_s: float = 3.0):
        """Start sampling; wait (up to first_sample_s) for the first sample, so
        that even a timed region shorter than the 200 ms period is bracketed
        by a sample taken just before it."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
            return
        t_end = time.monotonic() + first_sample_s
        while time.monotonic() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            self.f.close()
            os.unlink(self.f.name)
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def dist_init():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def meminfo_gb(key="MemAvailable") -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith(key + ":"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


# ---------------------------------------------------------------------------
def cpu_baseline(spec, budget_s: float):
    """The oracle, as it stands, on a bounded sample of channels."""
    import oracle
    import synth

    t_total, n_done, chans = 0.0, 0, []
    c = 0
    while t_total < budget_s and c < spec.n_chan:
        v = synth.fill_host(spec, chans=[c])
        t0 = time.perf_counter()
        oracle.correlate(v, spec.sample_bits, spec.n_inputs, 1, spec.n_time)
        t_total += time.perf_counter() - t0
        n_done += 1
        chans.append(c)
        c += max(1, spec.n_chan // 16)
    units = cmacs(spec) / spec.n_chan * n_done
    # the same oracle on one thread, one channel (the first of the sample)
    v = synth.fill_host(spec, chans=[0])
    t0 = time.perf_counter()
    oracle.correlate(v, spec.sample_bits, spec.n_inputs, 1, spec.n_time, n_threads=1)
    t1 = time.perf_counter() - t0
    return {"value": units / t_total / 1e12, "unit": "TCMAC/s", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{n_done} of {spec.n_chan} channels ({chans[0]}..{chans[-1]} step "
                      f"{max(1, spec.n_chan // 16)}), full N and T; {units:.3g} CMAC in {t_total:.1f} s",
            "one_thread": {"value": cmacs(spec) / spec.n_chan / t1 / 1e12, "unit": "TCMAC/s",
                           "cores": 1, "sample": f"channel 0, full N and T, {t1:.1f} s"}}


def run_reference(args, spec, desc, world, rank):
    """--impl reference: the CPU oracle timed on the host cores."""
    if rank != 0:
        return
    import oracle
    import synth

    # each step: one channel of the workload (bounded sample), oracle as it stands
    sample_chans = [(k * max(1, spec.n_chan // 16)) % spec.n_chan for k in range(args.steps + args.warmup)]
    vols = {}
    times = []
    for k, c in enumerate(sample_chans):
        if c not in vols:
            vols[c] = synth.fill_host(spec, chans=[c])
        t0 = time.perf_counter()
        oracle.correlate(vols[c], spec.sample_bits, spec.n_inputs, 1, spec.n_time)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    units = cmacs(spec) / spec.n_chan
    tot = sum(times)
    value = units * len(times) / tot / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TCMAC/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "step": "one channel per step"},
        "cpu_baseline": {"value": value, "unit": "TCMAC/s", "cores": oracle.threads(),
                         "kind": "oracle", "sample": f"1 of {spec.n_chan} channels per step"},
        "e2e": {"value": value, "unit": "TCMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def fp16_variant(mw, spec, vol, stream, args):
    import numpy as np
    import torch

    import oracle
    import synth

    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8, kind=mw.KIND_FP16, stream=stream)
    fout = p.empty_out()
    p.correlate(vol, fout)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    reps = 3
    for _ in range(reps):
        p.correlate(vol, fout)
    b.record(stream)
    b.synchronize()
    if p.status() != 0:
        raise RuntimeError("FP16 variant: device status not OK")
    ms = a.elapsed_time(b) / reps
    chans = [0, spec.n_chan - 1]
    got = fout[chans].double().cpu().numpy()
    p.close()
    _, ref = oracle.correlate(synth.fill_host(spec, chans=chans), 8, spec.n_inputs, len(chans),
                              spec.n_time, want64=True)
    ref = ref.astype(np.float64)
    N = spec.n_inputs
    ii, jj = np.tril_indices(N)
    autos = ref[:, [i * (i + 1) // 2 + i for i in range(N)], 0]
    norm = np.sqrt(autos[:, ii] * autos[:, jj])
    err = np.abs(got - ref).max(axis=2)
    big = np.abs(ref).max(axis=2) >= 0.01 * norm
    rep = {"value": cmacs(spec) / (ms / 1e3) / 1e12, "unit": "TCMAC/s", "ms_per_step": ms,
           "max_rel_err_autos_normalised": float((err / norm).max()),
           "max_abs_err": float(err.max()),
           "max_rel_err_where_abs_ge_1pct_of_autos": float((err[big] / np.abs(ref).max(axis=2)[big]).max()),
           "fp32_bound_2T_eps": 2 * spec.n_time * 2.0 ** -24,
           "channels_checked": chans, "reference": "int64 oracle (exact, equal to FP64)"}
    if np.all(err == 0):
        rep["note"] = ("every sum of this input stays below 2^24, where FP32 accumulation is exact; "
                       "see full_scale for an input where it rounds")
    rep["full_scale"] = fp16_full_scale(mw, spec, stream)
    return rep


def fp16_full_scale(mw, spec, stream, n_chan=8):
    """The FP16 variant on full-scale input (every component +-127) of the
    workload's shape, a few channels: the autos reach 2 * 127^2 * T, far above
    2^24, so the FP32 sums round; errors against the exact oracle."""
    import numpy as np
    import torch

    import oracle
    import synth

    fs = synth.Spec("full-scale", spec.n_inputs, n_chan, spec.n_time, 8, seed=spec.seed + 100,
                    kind=synth.SYNTH_RANDMAX)
    vol = torch.empty(n_chan * fs.n_time * fs.n_inputs * 2, dtype=torch.uint8, device="cuda")
    synth.fill_device(fs, vol)
    p = mw.Plan(fs.n_inputs, n_chan, fs.n_time, 8, kind=mw.KIND_FP16, stream=stream)
    out = p.correlate(vol)
    if p.status() != 0:
        raise RuntimeError("FP16 variant (full scale): device status not OK")
    p.close()
    chans = [0, n_chan - 1]
    got = out[chans].double().cpu().numpy()
    del vol, out
    _, ref = oracle.correlate(synth.fill_host(fs, chans=chans), 8, fs.n_inputs, len(chans),
                              fs.n_time, want64=True)
    ref = ref.astype(np.float64)
    N = fs.n_inputs
    ii, jj = np.tril_indices(N)
    autos = ref[:, [i * (i + 1) // 2 + i for i in range(N)], 0]
    norm = np.sqrt(autos[:, ii] * autos[:, jj])
    err = np.abs(got - ref).max(axis=2)
    ia = np.array([i * (i + 1) // 2 + i for i in range(N)])
    return {"input": f"{N} inputs x {n_chan} ch x T={fs.n_time}, every component +-127",
            "max_rel_err_autos_normalised": float((err / norm).max()),
            "max_abs_err": float(err.max()),
            "max_rel_err_autos": float((err[:, ia] / autos).max()),
            "fp32_bound_2T_eps": 2 * fs.n_time * 2.0 ** -24,
            "channels_checked": chans, "reference": "int64 oracle (exact, equal to FP64)"}


def run_batch(args):
    """c3: four uneven sub-array jobs in one persistent launch per call,
    replayed from a CUDA graph, against the plain per-channel form."""
    import numpy as np
    import torch

    import oracle
    import synth
    import paper_0902_0915_gb300 as mw

    if int(os.environ.get("RANK", "0")) != 0:
        return
    specs = [synth.spec_c3(j) for j in range(4)]
    desc = "batched jobs " + ", ".join(f"({s.n_inputs} in, {s.n_chan} ch, T={s.n_time})" for s in specs) + ", 4+4-bit"
    units = sum(cmacs(s) for s in specs)
    if args.impl == "reference":
        times, done = [], 0.0
        for k in range(args.steps + args.warmup):
            s = specs[k % 4]
            c = (k * 7) % s.n_chan
            v = synth.fill_host(s, chans=[c])
            t0 = time.perf_counter()
            oracle.correlate(v, 4, s.n_inputs, 1, s.n_time)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                times.append(dt)
                done += cmacs(s) / s.n_chan
        value = done / sum(times) / 1e12
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "TCMAC/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": sum(times) / len(times) * 1e3, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                          "config": {"workload": f"c3: {desc}", "step": "one channel of one job per step"},
                          "cpu_baseline": {"value": value, "unit": "TCMAC/s", "cores": oracle.threads(),
                                           "kind": "oracle", "sample": "one channel per step, jobs in turn"},
                          "e2e": {"value": value, "unit": "TCMAC/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    mw.ensure_built()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    vols = []
    for s in specs:
        v = torch.empty(s.n_chan * s.n_time * s.n_inputs, dtype=torch.uint8, device="cuda")
        synth.fill_device(s, v)
        vols.append(v)
    jobs = [(s.n_inputs, s.n_chan, s.n_time) for s in specs]
    outs = [torch.empty((s.n_chan, s.n_inputs * (s.n_inputs + 1) // 2, 2), dtype=torch.int32,
                        device="cuda") for s in specs]
    tune, rep = {}, None
    if args.tune:
        tune, rep = mw.autotune_batch(jobs, vols, outs, sample_bits=4, stream=stream)
    bp = mw.BatchPlan(jobs, sample_bits=4, stream=stream, **tune)
    for _ in range(args.warmup):
        bp.correlate(vols, outs)
    assert bp.status() == 0
    bp.set_timing(True)
    clocks = Clocks(0)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clocks.start()
    a.record(stream)
    for _ in range(args.steps):
        bp.correlate(vols, outs)
    b.record(stream)
    b.synchronize()
    clk = clocks.stop()
    tim = bp.timing()
    assert bp.status() == 0
    ms = a.elapsed_time(b) / args.steps
    peaks, src = load_peaks()
    peak = 2.0 * float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    achieved = 8.0 * units * args.steps / (tim.correlate_ms / 1e3) / 1e12 if tim.correlate_ms else None
    line = {"metric": METRIC, "value": units / (ms / 1e3) / 1e12, "unit": "TCMAC/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "e4m3",
            "data": "synthetic (seeded Philox4x64-10 channelised voltages, generated in HBM)",
            "config": {"workload": f"c3: {desc}", "launch": "per call: 4 unpacks + 1 persistent correlate, one CUDA graph",
                       "tuning": tune, "exact": "int32 visibilities, bit-exact",
                       "l2": "inputs 68 GB > 129 MB L2"},
            "roofline": None if achieved is None else {
                "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "correlate_tc_kernel (batched launch)",
                "peak_source": f"2 x bf16 sustained ({src})",
                "kernel_ms_per_launch": tim.correlate_ms / max(1, tim.correlate_launches),
                "unpack_ms_per_step": tim.unpack_ms / args.steps},
            "gpu_launches": int(5 * args.steps), "clocks": clk}
    pk = tensor_peak_at_clock(4, clk, torch.cuda.get_device_properties(0).multi_processor_count)
    if line["roofline"] is not None and pk:
        line["roofline"]["peak_at_clock"] = {"tflops": pk, "frac": achieved / pk,
                                             "note": "dense E4M3 MMA rate at the median SM clock sampled"}
    if rep is not None:
        line["config"]["autotune"] = {"candidates": rep.candidates, "best_ms": rep.best_ms,
                                      "default_ms": rep.default_ms}
    bp.close()
    if not args.no_plain:
        total = 0.0
        per_job = []
        for s, v, o in zip(specs, vols, outs):
            p = mw.Plan(s.n_inputs, s.n_chan, s.n_time, 4, engine=mw.ENGINE_PLAIN, stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.correlate(v, o)
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            per_job.append(t)
            total += t
            p.close()
        line["plain"] = {"ms_per_step": total, "value": units / (total / 1e3) / 1e12, "unit": "TCMAC/s",
                         "per_job_ms": per_job, "launches_per_step": sum(s.n_chan for s in specs),
                         "batched_speedup": total / ms}
    if not args.no_cpu:
        t_total, n_done = 0.0, 0.0
        for k, s in enumerate(specs):
            v = synth.fill_host(s, chans=[0])
            t0 = time.perf_counter()
            oracle.correlate(v, 4, s.n_inputs, 1, s.n_time)
            t_total += time.perf_counter() - t0
            n_done += cmacs(s) / s.n_chan
        line["cpu_baseline"] = {"value": n_done / t_total / 1e12, "unit": "TCMAC/s", "cores": oracle.threads(),
                                "kind": "oracle", "sample": "channel 0 of each job"}
    print(json.dumps(line), flush=True)


def model_visibilities(spec, chans, device):
    """M_ij(c) = sum_s S_s exp(i (phi_is - phi_js)) for the source geometry of
    `spec`, lower triangle [len(chans), N(N+1)/2] complex64 (setup only)."""
    import numpy as np
    import torch

    N = spec.n_inputs
    ii, jj = np.tril_indices(N)
    ii = torch.from_numpy(ii).to(device)
    jj = torch.from_numpy(jj).to(device)
    rate = torch.from_numpy(spec.src_rate.astype(np.float64)).to(device)  # [N, S] uint32 turns per channel
    flux = torch.from_numpy(np.asarray(spec.src_flux, np.float64)).to(device)
    out = torch.empty((len(chans), ii.numel()), dtype=torch.complex64, device=device)
    for k, c in enumerate(chans):
        turns = torch.remainder(rate * float(c + spec.chan_base), 2.0 ** 32) / 2.0 ** 32
        e = torch.exp(2j * np.pi * turns)  # [N, S]
        full = (e * flux) @ e.conj().T
        out[k] = full[ii, jj].to(torch.complex64)
    return out


def run_grid(args):
    """c5: gridding of the c1 correlation (128 tiles x 2 pol, 768 channels)
    onto four 2048 x 2048 polarisation grids."""
    import numpy as np
    import torch

    import oracle
    import synth
    import paper_0902_0915_gb300 as mw

    if int(os.environ.get("RANK", "0")) != 0:
        return
    spec = synth.spec_c1()
    geo = synth.grid_geometry_c1()
    N, C, T = spec.n_inputs, spec.n_chan, spec.n_time
    n_tiles = N // 2
    mw.ensure_built()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    vol = torch.empty(C * T * N, dtype=torch.uint8, device=dev)
    synth.fill_device(spec, vol)
    plan = mw.Plan(N, C, T, 4, stream=stream)
    vis = plan.correlate(vol)
    assert plan.status() == 0
    plan.close()
    del vol
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    gp = mw.GridPlan(geo["tile_xy"], C, geo["f0"], geo["df"], geo["Ng"], geo["du"], geo["W"],
                     geo["sigma"], stream=stream)
    plan_s = time.perf_counter() - t0
    grids = gp.empty_grids()
    for _ in range(args.warmup):
        gp.grid(vis, grids)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    a.record(stream)
    for _ in range(args.steps):
        gp.grid(vis, grids)
    b.record(stream)
    b.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b) / args.steps
    n_pts = gp.n_points
    n_entries = gp.n_entries
    W = geo["W"]
    Ng = geo["Ng"]
    # one grid call streams the stored weight factors (12 x 4 B per patch
    # candidate), gathers 4 int32 pairs per point (32 B), writes
    # and reads back the points' FP32 values (2 x 32 B), and writes the 4
    # grids (8 B per cell)
    bytes_call = 4.0 * n_entries + 96.0 * n_pts + 32.0 * Ng * Ng
    peaks, src = load_peaks()
    achieved = bytes_call / (ms / 1e3) / 1e9
    # context: every gridded point adds 4 complex values times a weight to the
    # W x W cells of its support, 8 FMA (16 flops) per cell
    tflops = n_pts * W * W * 16.0 / (ms / 1e3) / 1e12
    desc = (f"gridding of the c1 correlation ({n_tiles} tiles x 2 pol, {C} ch from "
            f"{geo['f0'] / 1e6:.2f} MHz) onto 4 x {geo['Ng']}^2 cells of {geo['du']} wavelength, "
            f"Gaussian support {W}")
    line = {"metric": "gridding throughput (visibility points x 4 polarisations / s), FP32",
            "value": n_pts * 4 / (ms / 1e3) / 1e9, "unit": "G samples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (the c1 correlation of seeded voltages; seeded tile positions)",
            "config": {"workload": f"c5: {desc}", "points": n_pts, "operator_entries": n_entries,
                       "l2": f"weight factors {4 * n_entries / 1e9:.2f} GB + grids {32 * Ng * Ng / 1e9:.2f} GB > L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s", "frac": achieved / float(peaks["hbm_gbs"]), "traffic": None,
                         "kernel": "grid_values_kernel + grid_apply_heavy_kernel + grid_apply_kernel (one grid call)",
                         "algorithmic_bytes": bytes_call, "fp32_tflops": tflops,
                         "peak_source": src},
            "plan_s": plan_s, "gpu_launches": 3 * args.steps, "clocks": clk}
    gp.close()
    if not args.no_cpu:
        sub = 8
        rng = np.random.default_rng(5)
        vh = rng.integers(-2 ** 20, 2 ** 20, (sub, N * (N + 1) // 2, 2)).astype(np.int32)
        t0 = time.perf_counter()
        oracle.grid(geo["tile_xy"], vh, geo["f0"], geo["df"], geo["Ng"], geo["du"], W, geo["sigma"])
        dt = time.perf_counter() - t0
        pts = n_tiles * (n_tiles - 1) * sub
        line["cpu_baseline"] = {"value": pts * 4 / dt / 1e9, "unit": "G samples/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"{sub} of {C} channels (seeded values of the same shape), FP64"}
    print(json.dumps(line), flush=True)


def run_stokes(args):
    """c6: per-pixel Stokes conversion of four 4096 x 4096 instrumental
    images covering the whole sky hemisphere (dl = 2/n)."""
    import numpy as np
    import torch

    import oracle
    import paper_0902_0915_gb300 as mw

    if int(os.environ.get("RANK", "0")) != 0:
        return
    n, chi = 4096, 0.3
    dl = 2.0 / n
    mw.ensure_built()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev)
    gen.manual_seed(6)
    inst = torch.randn((4, n, n), dtype=torch.complex64, device=dev, generator=gen)
    out = torch.empty_like(inst)
    for _ in range(args.warmup):
        mw.stokes(inst, dl, chi, out)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    a.record(stream)
    for _ in range(args.steps):
        mw.stokes(inst, dl, chi, out)
    b.record(stream)
    b.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b) / args.steps
    # 4 complex64 written per pixel; 4 read only above the horizon
    idx = (np.arange(n) - n / 2) * dl
    up = int(((idx[:, None] ** 2 + idx[None, :] ** 2) < 1.0).sum())
    bytes_step = 32.0 * n * n + 32.0 * up
    peaks, src = load_peaks()
    achieved = bytes_step / (ms / 1e3) / 1e9
    line = {"metric": "Stokes conversion throughput (pixels/s), FP32", "value": n * n / (ms / 1e3) / 1e9,
            "unit": "G pixels/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded complex Gaussian instrumental images)",
            "config": {"workload": f"c6: Stokes conversion of 4 x {n}^2 instrumental images, whole hemisphere, chi = {chi}",
                       "pixels_above_horizon": up,
                       "l2": f"{bytes_step / 1e9:.2f} GB per call > L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s", "frac": achieved / float(peaks["hbm_gbs"]),
                         "traffic": measured_traffic("stokes_kernel|4096", 1) if n == 4096 else None,
                         "kernel": "stokes_kernel", "peak_source": src},
            "gpu_launches": args.steps, "clocks": clk}
    if not args.no_cpu:
        rng = np.random.default_rng(6)
        sub = 128
        small = rng.standard_normal((4, sub, sub)) + 1j * rng.standard_normal((4, sub, sub))
        t0 = time.perf_counter()
        oracle.stokes(small, 2.0 / sub, chi)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sub * sub / dt / 1e9, "unit": "G pixels/s", "cores": 1,
                                "kind": "oracle", "sample": f"one {sub} x {sub} image set (FP64)"}
    print(json.dumps(line), flush=True)


def run_calib(args):
    """c4: calibration loss and adjoint (one pass) on correlator output."""
    import numpy as np
    import torch

    import oracle
    import synth
    import paper_0902_0915_gb300 as mw

    if int(os.environ.get("RANK", "0")) != 0:
        return
    spec = synth.spec_c4()
    if args.chan:
        spec = spec.with_(n_chan=args.chan)
    N, C, T = spec.n_inputs, spec.n_chan, spec.n_time
    B = N * (N + 1) // 2
    desc = f"calibration loss+adjoint, {N} inputs x {C} ch, V from T={T} 8-bit correlation, 20-source model"
    metric = "calibration loss+gradient throughput (baseline-channel terms/s), FP32"
    mw.ensure_built()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    vol = torch.empty(C * T * N * 2, dtype=torch.uint8, device=dev)
    synth.fill_device(spec, vol)
    plan = mw.Plan(N, C, T, 8, stream=stream)
    vis = plan.correlate(vol)
    assert plan.status() == 0
    plan.close()
    del vol
    scale2 = 2.0 * spec.meta["scale"] ** 2
    # element-wise IEEE division by a device scalar (the oracle side divides the same way)
    sdev = torch.tensor(np.float32(T * scale2), dtype=torch.float32, device=dev)
    V = torch.complex(vis[..., 0].float() / sdev, vis[..., 1].float() / sdev)
    del vis
    M = model_visibilities(spec, list(range(C)), dev)
    g_true = torch.from_numpy(np.asarray(spec.gains, np.complex64)).to(dev)
    rng = np.random.default_rng(4)
    g = (g_true * torch.from_numpy((1 + 0.05 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))).astype(np.complex64)).to(dev)).contiguous()
    ws = mw.calib_workspace(N, C, dev)
    for _ in range(args.warmup):
        loss, grad = mw.calib_loss_grad(V, M, g, ws)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    a.record(stream)
    for _ in range(args.steps):
        loss, grad = mw.calib_loss_grad(V, M, g, ws)
    b.record(stream)
    b.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b) / args.steps
    terms = B * C
    bytes_step = 2 * 8 * B * C + 16 * N
    peaks, src = load_peaks()
    achieved = bytes_step / (ms / 1e3) / 1e9
    line = {"metric": metric, "value": terms / (ms / 1e3) / 1e9, "unit": "Gterms/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (V from correlating seeded c4-style voltages; point-source model)",
            "config": {"workload": f"c4: {desc}", "l2": f"V + M {2 * 8 * B * C / 1e9:.1f} GB > L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s", "frac": achieved / float(peaks["hbm_gbs"]),
                         "traffic": measured_traffic("calib_step|N1024", C) if N == 1024 else None,
                         "kernel": "calib_tile_kernel + calib_gather_kernel (one step)",
                         "peak_source": src},
            "loss": float(loss), "gpu_launches": 2 * args.steps, "clocks": clk}
    # gain solve: alternating least-squares sweeps from the same starting gains
    n_sweeps = 10
    ws_solve = torch.empty(int(mw.lib().mwax_calib_solve_workspace_bytes(N, C)), dtype=torch.uint8,
                           device=dev)
    mw.calib_solve(V, M, g, 1, ws_solve)  # warm-up
    torch.cuda.synchronize()
    a.record(stream)
    g_sol, hist = mw.calib_solve(V, M, g, n_sweeps, ws_solve)
    b.record(stream)
    b.synchronize()
    ms_sweep = a.elapsed_time(b) / n_sweeps
    loss_final, _ = mw.calib_loss_grad(V, M, g_sol, ws, want_grad=False)
    achieved_s = bytes_step / (ms_sweep / 1e3) / 1e9
    line["solve"] = {"sweeps": n_sweeps, "ms_per_sweep": ms_sweep,
                     "value": terms / (ms_sweep / 1e3) / 1e9, "unit": "Gterms/s per sweep",
                     "loss_start": float(hist[0]), "loss_after": float(loss_final),
                     "roofline": {"bound": "hbm", "achieved": achieved_s, "peak": float(peaks["hbm_gbs"]),
                                  "unit": "GB/s", "frac": achieved_s / float(peaks["hbm_gbs"]),
                                  "traffic": (measured_traffic("calib_sweep|N1024", C)
                                              if N == 1024 else None),
                                  "kernel": "calib_tile_kernel<den> + calib_gather_kernel<solve> (one sweep)",
                                  "peak_source": src},
                     "gpu_launches": 2 * n_sweeps}
    # per-channel gains g_k(nu): the same pass with one gain per input and channel
    G = (g[None, :] * torch.from_numpy(
        (1 + 0.02 * (rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N))))
        .astype(np.complex64)).to(dev)).contiguous()
    ws_c = torch.empty(int(mw.lib().mwax_calib_chan_solve_workspace_bytes(N, C)), dtype=torch.uint8,
                       device=dev)
    for _ in range(args.warmup):
        mw.calib_chan_loss_grad(V, M, G, ws_c)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        loss_c, _ = mw.calib_chan_loss_grad(V, M, G, ws_c)
    b.record(stream)
    b.synchronize()
    ms_c = a.elapsed_time(b) / args.steps
    bytes_c = 2 * 8 * B * C + 2 * 8 * N * C  # V, M; G in, gradient out
    ach_c = bytes_c / (ms_c / 1e3) / 1e9
    mw.calib_chan_solve(V, M, G, 1, ws_c)  # warm-up
    torch.cuda.synchronize()
    a.record(stream)
    G_sol, hist_c = mw.calib_chan_solve(V, M, G, n_sweeps, ws_c)
    b.record(stream)
    b.synchronize()
    ms_cs = a.elapsed_time(b) / n_sweeps
    loss_c_final, _ = mw.calib_chan_loss_grad(V, M, G_sol, ws_c, want_grad=False)
    line["per_channel_gains"] = {
        "ms_per_step": ms_c, "value": terms / (ms_c / 1e3) / 1e9, "unit": "Gterms/s",
        "loss": float(loss_c),
        "roofline": {"bound": "hbm", "achieved": ach_c, "peak": float(peaks["hbm_gbs"]),
                     "unit": "GB/s", "frac": ach_c / float(peaks["hbm_gbs"]), "traffic": None,
                     "kernel": "calib_chan_tile_kernel + calib_chan_gather_kernel (one step)",
                     "peak_source": src},
        "solve": {"sweeps": n_sweeps, "ms_per_sweep": ms_cs,
                  "value": terms / (ms_cs / 1e3) / 1e9, "unit": "Gterms/s per sweep",
                  "loss_start": float(hist_c[0]), "loss_after": float(loss_c_final),
                  "hbm_frac": bytes_c / (ms_cs / 1e3) / 1e9 / float(peaks["hbm_gbs"])},
        "gpu_launches": 2 * args.steps + 2 * n_sweeps}
    # full 2x2 Jones matrices per tile (leakage terms), from diagonal gains plus 5 % leakage
    n_t = N // 2
    Jm = torch.zeros((n_t, 2, 2), dtype=torch.complex64, device=dev)
    Jm[:, 0, 0], Jm[:, 1, 1] = g[0::2], g[1::2]
    Jm[:, 0, 1] = torch.from_numpy((0.05 * (rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t))).astype(np.complex64)).to(dev)
    Jm[:, 1, 0] = torch.from_numpy((0.05 * (rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t))).astype(np.complex64)).to(dev)
    ws_j = torch.empty(int(mw.lib().mwax_calib_jones_workspace_bytes(N, C)), dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        mw.calib_jones_loss_grad(V, M, Jm, ws_j)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        loss_j, _ = mw.calib_jones_loss_grad(V, M, Jm, ws_j)
    b.record(stream)
    b.synchronize()
    ms_j = a.elapsed_time(b) / args.steps
    terms_j = 4 * (n_t * (n_t - 1) // 2) * C  # baseline-channel terms inside cross-tile blocks
    bytes_j = 16 * terms_j + 2 * 32 * n_t
    ach_j = bytes_j / (ms_j / 1e3) / 1e9
    mw.calib_jones_solve(V, M, Jm, 1, ws_j)  # warm-up
    torch.cuda.synchronize()
    a.record(stream)
    J_sol, hist_j = mw.calib_jones_solve(V, M, Jm, n_sweeps, ws_j)
    b.record(stream)
    b.synchronize()
    ms_js = a.elapsed_time(b) / n_sweeps
    loss_j_final, _ = mw.calib_jones_loss_grad(V, M, J_sol, ws_j, want_grad=False)
    line["jones"] = {
        "ms_per_step": ms_j, "value": terms_j / (ms_j / 1e3) / 1e9, "unit": "Gterms/s",
        "loss": float(loss_j),
        "roofline": {"bound": "hbm", "achieved": ach_j, "peak": float(peaks["hbm_gbs"]),
                     "unit": "GB/s", "frac": ach_j / float(peaks["hbm_gbs"]), "traffic": None,
                     "kernel": "calib_jones_tile2_kernel + calib_jones_gather_kernel (one step)",
                     "peak_source": src},
        "solve": {"sweeps": n_sweeps, "ms_per_sweep": ms_js,
                  "value": terms_j / (ms_js / 1e3) / 1e9, "unit": "Gterms/s per sweep",
                  "loss_start": float(hist_j[0]), "loss_after": float(loss_j_final),
                  "hbm_frac": bytes_j / (ms_js / 1e3) / 1e9 / float(peaks["hbm_gbs"])},
        "gpu_launches": 2 * args.steps + 2 * n_sweeps}
    if not args.no_cpu:
        sub = list(range(0, C, C // 8))[:8]
        # the oracle's own correlation of these channels (bit-exact against the
        # GPU's, checked), turned into V by the same FP32 formula
        vis64 = oracle.correlate(synth.fill_host(spec, chans=sub), 8, N, len(sub), T)
        sc = np.float32(T * scale2)
        V_host = (vis64[..., 0].astype(np.float32) / sc
                  + 1j * (vis64[..., 1].astype(np.float32) / sc)).astype(np.complex64)
        V64 = V_host.astype(np.complex128)
        M64 = M[sub].cpu().numpy().astype(np.complex128)
        g64 = g.cpu().numpy().astype(np.complex128)
        t0 = time.perf_counter()
        L64 = oracle.calib_loss(V64, M64, g64)
        G64 = oracle.calib_grad(V64, M64, g64)
        dt = time.perf_counter() - t0
        subd = torch.tensor(sub, device=dev)
        Vs, Ms = V.index_select(0, subd), M.index_select(0, subd)
        ls, gs_ = mw.calib_loss_grad(Vs, Ms, g)
        gsn = gs_.cpu().numpy()
        line["check"] = {
            "channels": sub, "v_equal_to_oracle_v": bool(np.array_equal(
                Vs.cpu().numpy().view(np.uint32), V_host.view(np.uint32))),
            "loss_rel_err": abs(float(ls) - L64) / L64,
            "grad_max_rel_err": float(np.abs(gsn - G64).max() / np.abs(G64).max()),
            "tolerance": {"loss": 1e-5, "grad": 1e-4},
            "reference": "FP64 oracle on the oracle's correlation of the sampled channels"}
        line["cpu_baseline"] = {"value": B * len(sub) / dt / 1e9, "unit": "Gterms/s", "cores": oracle.threads(),
                                "kind": "oracle", "sample": f"{len(sub)} of {C} channels (FP64 loss + gradient)"}
        t0 = time.perf_counter()
        oracle.calib_solve(V64, M64, g64, 1)
        dt = time.perf_counter() - t0
        line["solve"]["cpu_baseline"] = {"value": B * len(sub) / dt / 1e9, "unit": "Gterms/s per sweep",
                                         "cores": oracle.threads(), "kind": "oracle",
                                         "sample": f"1 sweep on {len(sub)} of {C} channels (FP64)"}
        G64 = G[sub].cpu().numpy().astype(np.complex128)
        t0 = time.perf_counter()
        oracle.calib_chan_loss(V64, M64, G64)
        oracle.calib_chan_grad(V64, M64, G64)
        dt = time.perf_counter() - t0
        J64 = Jm.cpu().numpy().astype(np.complex128)
        t0 = time.perf_counter()
        oracle.calib_jones_loss(V64, M64, J64)
        oracle.calib_jones_grad(V64, M64, J64)
        dt = time.perf_counter() - t0
        line["jones"]["cpu_baseline"] = {
            "value": 4 * (n_t * (n_t - 1) // 2) * len(sub) / dt / 1e9, "unit": "Gterms/s",
            "cores": 1, "kind": "oracle", "sample": f"{len(sub)} of {C} channels (FP64 numpy loss + gradient)"}
        line["per_channel_gains"]["cpu_baseline"] = {
            "value": B * len(sub) / dt / 1e9, "unit": "Gterms/s", "cores": oracle.threads(),
            "kind": "oracle", "sample": f"{len(sub)} of {C} channels (FP64 loss + gradient)"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mwax", choices=["mwax", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c0", "c3", "c4", "c5", "c6"])
    ap.add_argument("--engine", default="tensor", choices=["tensor", "plain"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank correlates its own full workload; strong: the "
                         "workload's channels are split across ranks")
    ap.add_argument("--chan", type=int, default=0,
                    help="override the channel count (small cases for profiling)")
    ap.add_argument("--tune", action="store_true",
                    help="run the autotuner first (default: the plan's default configuration, "
                         "the one the committed ncu traffic figures were taken on)")
    ap.add_argument("--no-tune", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-variant report")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    import synth

    if args.workload == "c3":
        return run_batch(args)
    if args.workload == "c5":
        return run_grid(args)
    if args.workload == "c6":
        return run_stokes(args)
    if args.workload == "c4":
        return run_calib(args)

    mk, desc = workloads()[args.workload]
    spec = mk()
    if args.chan > 0:
        spec = spec.with_(n_chan=args.chan)
        desc = f"{desc}; channels reduced to {args.chan}"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, spec, desc, world, rank)
        return

    import torch

    import paper_0902_0915_gb300 as mw

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mw.ensure_built()
    if not os.path.exists(synth.CUDA_LIB):
        synth.build()
    from paper_0902_0915_gb300.shard import channel_range

    if args.scaling == "weak":
        # every rank correlates its own full workload (its own band)
        rspec = spec.with_(seed=spec.seed + 1000 * rank) if rank else spec
        chan0 = 0
    else:
        # the workload's channels split into contiguous ranges, no exchange
        chan0, chan1 = channel_range(spec.n_chan, rank, world)
        rspec = spec.with_(n_chan=chan1 - chan0)
    stream = torch.cuda.current_stream(dev)
    vol = torch.empty(rspec.n_chan * rspec.n_time * rspec.n_inputs * rspec.bytes_per_sample,
                      dtype=torch.uint8, device=dev)
    if args.scaling == "weak":
        synth.fill_device(rspec, vol)
    else:
        synth.fill_device(spec, vol, chan0=chan0, n_chan=rspec.n_chan)
    engine = mw.ENGINE_TENSOR if args.engine == "tensor" else mw.ENGINE_PLAIN
    n_bl = rspec.n_inputs * (rspec.n_inputs + 1) // 2
    out = torch.empty((rspec.n_chan, n_bl, 2), dtype=torch.int32, device=dev)
    tune, tune_rep = {}, None
    if engine == mw.ENGINE_TENSOR and args.tune:
        tune, tune_rep = mw.autotune(vol, out, rspec.n_inputs, rspec.n_chan, rspec.n_time,
                                     rspec.sample_bits, stream=stream)
    plan = mw.Plan(rspec.n_inputs, rspec.n_chan, rspec.n_time, rspec.sample_bits, engine=engine,
                   stream=stream, **tune)
    for _ in range(args.warmup):
        plan.correlate(vol, out)
    if plan.status() != 0:
        raise RuntimeError("device status not OK after warm-up")
    clocks = Clocks(local)
    clocks.start()  # waits for its first sample, so before the barrier
    plan.set_timing(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        plan.correlate(vol, out)
    ev1.record(stream)
    ev1.synchronize()
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(world)
    elapsed_ms = ev0.elapsed_time(ev1)
    tim = plan.timing()
    plan.set_timing(False)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"device status {st} in the timed region")
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    ms_per_step = elapsed_ms / args.steps
    units = cmacs(rspec)
    total_units = units * world if args.scaling == "weak" else cmacs(spec)
    value = total_units / (ms_per_step / 1e3) / 1e12
    rtf = sky_seconds(rspec) / (ms_per_step / 1e3)

    peaks, peak_src = load_peaks()
    if rspec.sample_bits == 8:
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        peak_note = f"bf16 sustained ({peak_src}); kind::f16 runs at the bf16 rate"
    else:
        peak = 2.0 * float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
        peak_note = f"2 x bf16 sustained ({peak_src}; nominal fp8/bf16 ratio 4.5/2.25)"
    info = plan.info()
    recomputed = plan.recomputed_channels() if engine == mw.ENGINE_TENSOR else 0
    if engine == mw.ENGINE_TENSOR and tim.correlate_ms > 0:
        achieved = 8.0 * units * args.steps / (tim.correlate_ms / 1e3) / 1e12
        tkey = (f"correlate_tc_kernel<{rspec.sample_bits},EXACT,"
                f"{ {1: 'narrow', 2: 'wide', 3: 'pair', 4: 'fused'}.get(info.mma_shape, 'narrow') }>"
                f"|N{rspec.n_inputs}|T{rspec.n_time}")
        tent = traffic_entry(tkey)
        traffic = tent["bytes_per_channel"] * info.chan_group if tent else None
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "traffic_note": (f"DRAM bytes per launch of chan_group channels, scaled from a "
                                     f"{tent['capture_channels']}-channel ncu capture "
                                     f"(profiles/traffic.json); algorithmic bytes per launch: "
                                     f"operands + visibilities = "
                                     f"{tent['algorithmic_bytes_per_channel'] * info.chan_group:.4g}"
                                     if tent else None),
                    "kernel": "correlate_tc_kernel", "peak_source": peak_note,
                    "kernel_ms_per_launch": tim.correlate_ms / max(1, tim.correlate_launches),
                    "unpack_ms_per_step": tim.unpack_ms / args.steps,
                    "correlate_ms_per_step": tim.correlate_ms / args.steps}
        if tim.unpack_ms > 0:
            roofline["unpack"] = unpack_roofline(rspec, info, tim, args.steps, peaks, peak_src)
        if info.mma_shape == 4:
            roofline["note"] = ("fused pair mode: the kernel also converts the packed samples into its "
                                "operand tiles (no unpack pass, no operand buffer), so its duration is the "
                                "whole step; the tensor pipe waits on that conversion")
            roofline["packed_samples_gbs"] = (rspec.n_chan * rspec.n_time * rspec.n_inputs * args.steps
                                              / (tim.correlate_ms / 1e3) / 1e9)
        pk = tensor_peak_at_clock(rspec.sample_bits, clk,
                                  torch.cuda.get_device_properties(dev).multi_processor_count)
        if pk:
            roofline["peak_at_clock"] = {"tflops": pk, "frac": achieved / pk,
                                         "note": "dense MMA rate at the median SM clock sampled"}
    else:
        roofline = None

    line = {
        "metric": METRIC, "value": value, "unit": "TCMAC/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": args.scaling, "vs_baseline": None,
        "dtype": "f16" if rspec.sample_bits == 8 else "e4m3",
        "data": "synthetic (seeded Philox4x64-10 channelised voltages, generated in HBM)",
        "config": {"workload": f"{args.workload}: {desc}", "n_inputs": rspec.n_inputs,
                   "n_chan": rspec.n_chan, "n_time": rspec.n_time, "sample_bits": rspec.sample_bits,
                   "engine": args.engine, "exact": "int32 visibilities, bit-exact",
                   "l2": f"inputs {vol.numel() / 1e9:.1f} GB > 129 MB L2 (no flush needed)",
                   "chan_group": info.chan_group, "flush_blocks": info.flush_blocks,
                   "mma_shape": info.mma_shape, "stages": info.stages, "prefetch": info.prefetch,
                   "k_split": info.k_split,
                   "pipeline": info.pipeline,
                   "checked_segment": None if not info.checked_segment else {
                       "recomputed_channels": recomputed,
                       "of": rspec.n_chan * (args.warmup + args.steps),
                       "note": "one FP32 segment per item; channels whose largest auto "
                               "reached 2^24 recomputed with exact segments"},
                   "autotune": None if tune_rep is None else {
                       "candidates": tune_rep.candidates, "from_cache": bool(tune_rep.from_cache),
                       "best_ms": tune_rep.best_ms, "default_ms": tune_rep.default_ms},
                   "parallelism": f"channels, {world} GPU(s), no collective"},
        "rtf": rtf,
        "roofline": roofline,
        # a checked-segment correlate launch is followed by the check kernel and
        # the (usually empty) recompute launch inside the same timed record
        "gpu_launches": int(tim.unpack_launches
                            + tim.correlate_launches * (3 if info.checked_segment else 1)),
        "clocks": clk,
    }

    # plain form on the same GPU (one CUDA-core launch per channel), one step
    if rank == 0 and not args.no_plain and engine == mw.ENGINE_TENSOR:
        pp = mw.Plan(rspec.n_inputs, rspec.n_chan, rspec.n_time, rspec.sample_bits,
                     engine=mw.ENGINE_PLAIN, stream=stream)
        pp.correlate(vol, out)  # warm-up
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pp.correlate(vol, out)
        b.record(stream)
        b.synchronize()
        pms = a.elapsed_time(b)
        line["plain"] = {"ms_per_step": pms, "value": units / (pms / 1e3) / 1e12, "unit": "TCMAC/s",
                         "launches_per_step": rspec.n_chan}
        pp.close()

    # FP16-in / FP32-accumulate variant (8-bit samples): time and error vs the
    # exact integer oracle (= FP64-exact) on two sampled channels
    if rank == 0 and not args.no_fp16 and engine == mw.ENGINE_TENSOR and rspec.sample_bits == 8:
        line["fp16_variant"] = fp16_variant(mw, rspec, vol, stream, args)

    # end to end through the public API with host buffers (pinned), N GPUs
    if not args.no_e2e:
        in_b = vol.numel()
        out_b = out.numel() * 4
        need_gb = (in_b + out_b) / 1e9 * 1.25
        if meminfo_gb() * 0.8 / max(1, world) < need_gb:
            line["e2e"] = None
            line["e2e_note"] = f"skipped: host MemAvailable {meminfo_gb():.0f} GB < {need_gb:.0f} GB per rank"
        else:
            hin = torch.empty(in_b, dtype=torch.uint8).pin_memory()
            hout = torch.empty(out.shape, dtype=out.dtype).pin_memory()
            hin.copy_(vol)
            del vol
            torch.cuda.empty_cache()
            plan.correlate_host(hin, hout)  # warm-up (allocates the staging ring)
            # each call is one step: H2D of every channel group, compute, D2H of
            # the visibilities.  The host link is shared with other tenants of
            # the machine, so the step time is the median of the timed calls.
            # The plan's timing hook records events around every copy on its
            # copy streams, so the link rate reported is the one these calls
            # achieved (bytes over the summed copy durations).
            n_e2e = max(3, min(args.steps, 7))
            times = []
            plan.timing()
            plan.set_timing(True)
            for _ in range(n_e2e):
                barrier(world)
                t0 = time.perf_counter()
                plan.correlate_host(hin, hout)
                times.append(max_over_ranks(time.perf_counter() - t0, world))
            tm = plan.timing()
            plan.set_timing(False)
            dt = statistics.median(times)
            link_h2d_gbs = tm.h2d_bytes / (tm.h2d_ms / 1e3) / 1e9 if tm.h2d_ms > 0 else None
            link_d2h_gbs = tm.d2h_bytes / (tm.d2h_ms / 1e3) / 1e9 if tm.d2h_ms > 0 else None
            line["e2e"] = {"value": total_units / dt / 1e12, "unit": "TCMAC/s",
                           "h2d_bytes_per_step": in_b, "d2h_bytes_per_step": out_b,
                           "ms_per_step": dt * 1e3, "steps": n_e2e, "statistic": "median",
                           "ms_min": min(times) * 1e3, "ms_max": max(times) * 1e3,
                           "link_h2d_gbs": link_h2d_gbs, "link_d2h_gbs": link_d2h_gbs,
                           "h2d_ms_per_step": tm.h2d_ms / n_e2e,
                           "link_note": "rates of the host path's own copies in these calls "
                                        "(events on its copy streams)",
                           "link_bound_value": (total_units / (in_b / (link_h2d_gbs * 1e9)) / 1e12
                                                if link_h2d_gbs else None)}

    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(spec, args.cpu_budget)

    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
