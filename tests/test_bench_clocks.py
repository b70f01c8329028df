"""The bench's clock sampler (CPU, with a stand-in for nvidia-smi on PATH):
it waits for a first sample before the timed region, takes the median SM
clock, and reports every active throttle reason by name."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/bin/sh
# prints one CSV sample every 0.2 s, as nvidia-smi -lms 200 does
sleep 0.3
i=0
while true; do
  if [ $i -lt 2 ]; then sm=2070; else sm=1800; fi
  echo "0, $sm, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active"
  i=$((i+1))
  sleep 0.2
done
"""


def test_clock_sampler_waits_and_summarises(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    c = bench.Clocks(0)
    t0 = time.monotonic()
    c.start()
    waited = time.monotonic() - t0
    assert 0.2 <= waited < 3.0  # returned once the first sample was there
    r = c.stop()  # a timed region far shorter than the sampling period
    assert r is not None and r["samples"] >= 1
    assert r["sm_max_mhz"] == 2070.0 and r["reasons"] == ["sw_power_cap"]
    c = bench.Clocks(0)
    c.start()
    time.sleep(1.6)
    r = c.stop()
    assert r["samples"] >= 3
    if r["samples"] >= 5:  # 2070, 2070, then 1800s: the median is 1800
        assert r["sm_mhz"] == 1800.0


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    c = bench.Clocks(0)
    name = c.f.name
    c.start()
    assert c.stop() is None
    assert not os.path.exists(name)  # the sample file is removed either way


ARGS_FAKE = """#!/bin/sh
# records its arguments, then prints one sample
echo "$@" > "$(dirname "$0")/args.txt"
echo "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
sleep 5
"""


def test_clock_sampler_names_the_visible_gpu(tmp_path, monkeypatch):
    """Under CUDA_VISIBLE_DEVICES=3 CUDA device 0 is physical GPU 3: the sampler
    must ask nvidia-smi (which ignores the variable) about GPU 3, not GPU 0."""
    exe = tmp_path / "nvidia-smi"
    exe.write_text(ARGS_FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3")
    import torch

    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)  # the CPU-side fallback
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    c = bench.Clocks(0)
    assert c.gpu_id == "3"
    c.start()
    c.stop()
    args = (tmp_path / "args.txt").read_text().split()
    assert args[args.index("-i") + 1] == "3"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-0c1d2e3f, GPU-aabbccdd")
    assert bench.Clocks(1).gpu_id == "GPU-aabbccdd"
