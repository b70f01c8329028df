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


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
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
    return {"value": units / t_total / 1e12, "unit": "TCMAC/s", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{n_done} of {spec.n_chan} channels ({chans[0]}..{chans[-1]} step "
                      f"{max(1, spec.n_chan // 16)}), full N and T; {units:.3g} CMAC in {t_total:.1f} s"}


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
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mwax", choices=["mwax", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c0"])
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
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    import synth

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
    plan = mw.Plan(rspec.n_inputs, rspec.n_chan, rspec.n_time, rspec.sample_bits, engine=engine,
                   stream=stream)
    out = plan.empty_out(dev)
    for _ in range(args.warmup):
        plan.correlate(vol, out)
    if plan.status() != 0:
        raise RuntimeError("device status not OK after warm-up")
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    plan.set_timing(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
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
    if engine == mw.ENGINE_TENSOR and tim.correlate_ms > 0:
        achieved = 8.0 * units * args.steps / (tim.correlate_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "correlate_tc_kernel", "peak_source": peak_note,
                    "kernel_ms_per_launch": tim.correlate_ms / max(1, tim.correlate_launches),
                    "unpack_ms_per_step": tim.unpack_ms / args.steps,
                    "correlate_ms_per_step": tim.correlate_ms / args.steps}
    else:
        roofline = None

    info = plan.info()
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
                   "parallelism": f"channels, {world} GPU(s), no collective"},
        "rtf": rtf,
        "roofline": roofline,
        "gpu_launches": int(tim.unpack_launches + tim.correlate_launches),
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
            barrier(world)
            t0 = time.perf_counter()
            n_e2e = max(1, min(args.steps, 5))
            for _ in range(n_e2e):
                plan.correlate_host(hin, hout)
            dt = (time.perf_counter() - t0) / n_e2e
            dt = max_over_ranks(dt, world)
            line["e2e"] = {"value": total_units / dt / 1e12, "unit": "TCMAC/s",
                           "h2d_bytes_per_step": in_b, "d2h_bytes_per_step": out_b,
                           "ms_per_step": dt * 1e3, "steps": n_e2e}

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
