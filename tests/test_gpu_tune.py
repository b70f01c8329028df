"""Autotuner and pipeline options: every tuning choice keeps the result
bit-exact; the tuner's choice is cached and re-applied."""
import numpy as np
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


def test_autotune_choice_is_exact_and_cached(mw, tmp_path, monkeypatch):
    import torch

    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("MWAX_TUNE_CACHE", str(cache))
    spec = synth.Spec("t", 300, 9, 700, 8, seed=5, sigma=40)
    v = device_volt(spec)
    out = torch.empty((spec.n_chan, spec.n_inputs * (spec.n_inputs + 1) // 2, 2), dtype=torch.int32,
                      device="cuda")
    fields, rep = mw.autotune(v, out, spec.n_inputs, spec.n_chan, spec.n_time, 8)
    assert rep.candidates >= 4 and rep.from_cache == 0 and rep.best_ms > 0
    # candidate 0 is the plan's own default: tuning never picks a slower setting
    assert rep.default_ms > 0 and rep.best_ms <= rep.default_ms * 1.0001
    assert cache.read_text().strip()
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8, **fields)
    got = p.correlate(v)
    assert p.status() == 0
    assert_exact(got.cpu().numpy(), oracle_for(spec, range(spec.n_chan)), "tuned")
    p.close()
    fields2, rep2 = mw.autotune(v, out, spec.n_inputs, spec.n_chan, spec.n_time, 8)
    assert rep2.from_cache == 1 and fields2 == fields
    # an all-auto plan picks the cached choice up
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8)
    inf = p.info()
    assert inf.mma_shape == fields["mma_shape"] and inf.stages == fields["stages"]
    p.close()


@pytest.mark.parametrize("N,bits", [(260, 8), (256, 8), (256, 4)])
@pytest.mark.parametrize("shape", [1, 2])
def test_overlapped_pipeline_is_exact(mw, shape, N, bits):
    """Unpack of the next channel group on a few SMs (second stream, second
    scratch buffer) beside the correlation of the current one; N = 256 takes
    the TMA-staged unpack, N = 260 the register-staged one."""
    spec = synth.Spec("o", N, 7, 300, bits, seed=8, sigma=50 if bits == 8 else 2)
    v = device_volt(spec)
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, bits, chan_group=2, pipeline=2,
                mma_shape=shape, unpack_sms=12)
    assert p.info().pipeline == 2
    out = p.correlate(v)
    out = p.correlate(v, out)
    assert p.status() == 0
    assert_exact(out.cpu().numpy(), oracle_for(spec, range(spec.n_chan)), "overlap")
    p.close()


def test_batch_autotune_and_graph_timing(mw):
    import torch

    jobs = [(64, 5, 300), (200, 3, 400)]
    specs = [synth.Spec(f"bt{k}", n, c, t, 4, seed=60 + k, sigma=2) for k, (n, c, t) in enumerate(jobs)]
    vs = [device_volt(s) for s in specs]
    outs = [torch.empty((c, n * (n + 1) // 2, 2), dtype=torch.int32, device="cuda") for (n, c, t) in jobs]
    fields, rep = mw.autotune_batch(jobs, vs, outs)
    assert rep.candidates >= 3 and rep.best_ms > 0
    assert rep.default_ms > 0 and rep.best_ms <= rep.default_ms * 1.0001
    assert len(fields["k_split"]) == len(jobs) and all(0 <= k <= 8 for k in fields["k_split"])
    bp = mw.BatchPlan(jobs, **fields)
    bp.set_timing(True)
    outs = bp.correlate(vs, outs)
    t = bp.timing()
    assert t.correlate_launches == 1 and t.unpack_launches == 1 and t.correlate_ms > 0 and t.unpack_ms > 0
    assert bp.status() == 0
    for s, o in zip(specs, outs):
        assert_exact(o.cpu().numpy(), oracle_for(s, range(s.n_chan)), s.name)
    bp.close()


def test_autotune_4bit_with_fused_candidates(mw, tmp_path, monkeypatch):
    """A 4-bit job of two tiles: the candidates include the fused pair mode
    (mma_shape 4) with and without time ranges; the plan's default is
    candidate 0, the choice is never slower than it, and it stays exact."""
    import torch

    monkeypatch.setenv("MWAX_TUNE_CACHE", str(tmp_path / "tune4.txt"))
    spec = synth.Spec("t4", 256, 6, 2000, 4, seed=9, sigma=2, tone_amp=0.3)
    v = device_volt(spec)
    out = torch.empty((spec.n_chan, spec.n_inputs * (spec.n_inputs + 1) // 2, 2), dtype=torch.int32,
                      device="cuda")
    fields, rep = mw.autotune(v, out, spec.n_inputs, spec.n_chan, spec.n_time, 4)
    assert rep.candidates >= 8 and rep.from_cache == 0
    assert rep.default_ms > 0 and rep.best_ms <= rep.default_ms * 1.0001
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 4, **fields)
    assert p.info().mma_shape in (1, 2, 3, 4)
    got = p.correlate(v)
    assert p.status() == 0
    assert_exact(got.cpu().numpy(), oracle_for(spec, range(spec.n_chan)), "tuned 4-bit")
    p.close()
