"""Failure detection on the GPU without faulting it: a bounded device wait is
made to run out on purpose (the epilogue withholds one accumulator release),
the kernel reports MWAX_ERR_TIMEOUT through the plan's status word, frees its
tensor memory and returns, and the device keeps working."""
import time

import pytest

import synth
from gpu_util import assert_exact, device_volt, oracle_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mw(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return mwax_lib


@pytest.mark.parametrize("shape", [1, 2])
def test_withheld_release_times_out_and_device_recovers(mw, shape):
    import torch

    spec = synth.Spec("ff", 130, 4, 600, 8, seed=3, sigma=30)
    v = device_volt(spec)
    # flush_blocks=1: one accumulator segment per K-block, so every CTA needs
    # to reuse its first accumulator buffer; 150 ms per wait
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8, flush_blocks=1, timeout_ms=150,
                test_fault=1, mma_shape=shape)
    t0 = time.time()
    p.correlate(v)
    st = p.status()
    dt = time.time() - t0
    assert st == mw.STATUS_BY_NAME["MWAX_ERR_TIMEOUT"]
    assert dt < 30.0
    p.close()
    # the context is intact: the same correlation without the fault is exact
    q = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8, flush_blocks=1, mma_shape=shape)
    out = q.correlate(v)
    assert q.status() == 0
    assert_exact(out.cpu().numpy(), oracle_for(spec, range(spec.n_chan)), "after timeout")
    q.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("shape", [3, 4])
def test_withheld_release_times_out_pair_mode(mw, shape):
    """The same in pair mode and in the fused pair mode (one accumulator
    buffer per CTA, released per work item): CTA 0 withholds the release of
    its first item, so the MMA warp's wait before its second item runs out
    (and the fused mode's converter warps, waiting for a free stage, end on
    the abort flag)."""
    import torch

    spec = synth.Spec("ffp", 256, 400, 600, 4, seed=5, sigma=2)
    v = device_volt(spec)
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 4, timeout_ms=150, test_fault=1,
                mma_shape=shape)
    assert p.info().work_items > 2 * 152
    t0 = time.time()
    p.correlate(v)
    st = p.status()
    assert st == mw.STATUS_BY_NAME["MWAX_ERR_TIMEOUT"]
    assert time.time() - t0 < 30.0
    p.close()
    q = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 4, mma_shape=shape)
    out = q.correlate(v)
    assert q.status() == 0
    chans = [0, 1, 199, 398, 399]
    assert_exact(out[chans].cpu().numpy(), oracle_for(spec, chans), "after timeout (pair)")
    q.close()
    torch.cuda.synchronize()


def test_status_word_clears_after_read(mw):
    spec = synth.Spec("ff2", 64, 2, 200, 8, seed=4, sigma=30)
    v = device_volt(spec)
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8, flush_blocks=1, timeout_ms=100,
                test_fault=1)
    p.correlate(v)
    assert p.status() == mw.STATUS_BY_NAME["MWAX_ERR_TIMEOUT"]
    assert p.status() == 0  # read-and-clear
    p.close()


def test_allocation_failure_is_reported(mw, monkeypatch):
    """Host-side injected fault: with the allocation test hook set, plan
    creation returns MWAX_ERR_OOM (no abort, nothing leaked), and the next
    plan without it works."""
    import torch

    monkeypatch.setenv("MWAX_TEST_FAIL_ALLOC", "1")
    for make in (lambda: mw.Plan(64, 4, 100, 4),
                 lambda: mw.BatchPlan([(48, 2, 100), (64, 3, 200)], sample_bits=4)):
        with pytest.raises(mw.MwaxError) as ei:
            make()
        assert ei.value.status == mw.STATUS_BY_NAME["MWAX_ERR_OOM"]
    monkeypatch.delenv("MWAX_TEST_FAIL_ALLOC")
    p = mw.Plan(64, 4, 100, 4)
    out = p.correlate(torch.zeros(64 * 4 * 100, dtype=torch.uint8, device="cuda"))
    assert p.status() == 0 and int(out.abs().sum().item()) == 0
    p.close()
