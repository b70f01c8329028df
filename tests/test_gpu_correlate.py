"""GPU parity of the correlator against the CPU oracle, through the C ABI.

Integer visibilities must match the oracle bit for bit.  Inputs are filled
on the device by the shared generator and regenerated on the host for the
oracle (never copied back from the GPU)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_exact, device_volt, oracle_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mw(mwax_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return mwax_lib


def run(mw, spec, engine, **kw):
    import torch

    v = device_volt(spec)
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, spec.sample_bits, engine=engine, **kw)
    out = p.correlate(v)
    st = p.status()
    torch.cuda.synchronize()
    assert st == 0, f"device status {st}"
    res = out.cpu().numpy()
    p.close()
    return res


# ---------------------------------------------------------------------------
def test_device_generator_matches_host(mw):
    import torch

    for spec, chans in ((synth.spec_c0(), None), (synth.spec_c1().with_(n_time=300), (0, 767)),
                        (synth.spec_c2().with_(n_time=100), (5, 3071))):
        if chans is None:
            d = device_volt(spec).cpu().numpy()
            h = synth.fill_host(spec).ravel()
            np.testing.assert_array_equal(d, h)
        else:
            for c in chans:
                d = device_volt(spec, chan0=c, n_chan=1).cpu().numpy()
                h = synth.fill_host(spec, chans=[c]).ravel()
                np.testing.assert_array_equal(d, h)
    torch.cuda.synchronize()


SMALL = [(1, 1, 1), (2, 7, 1), (3, 8, 3), (17, 33, 2), (64, 100, 3), (129, 65, 2), (130, 64, 1),
         (257, 40, 1)]


@pytest.mark.parametrize("bits", [4, 8])
@pytest.mark.parametrize("N,T,C", SMALL)
def test_plain_small(mw, bits, N, T, C):
    spec = synth.Spec("s", N, C, T, bits, seed=N * 131 + T, sigma=2 if bits == 4 else 40,
                      tone_amp=0.3)
    assert_exact(run(mw, spec, mw.ENGINE_PLAIN), oracle_for(spec, range(C)), f"plain {N},{T},{C}")


SHAPES = [1, 2]  # M128xN128 (Re, Im separately) and M128xN256 ([Re | Im] per MMA)
# plus 3: two tile pairs per work item, for integrations that are one exact segment
SHAPES_ONE_SEGMENT = [1, 2, 3]


@pytest.mark.parametrize("shape", SHAPES_ONE_SEGMENT)
@pytest.mark.parametrize("bits", [4, 8])
@pytest.mark.parametrize("N,T,C", SMALL)
def test_tensor_small(mw, bits, N, T, C, shape):
    spec = synth.Spec("s", N, C, T, bits, seed=N * 131 + T + 7, sigma=2 if bits == 4 else 40,
                      tone_amp=0.3)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, mma_shape=shape), oracle_for(spec, range(C)),
                 f"tc {N},{T},{C}")


@pytest.mark.parametrize("bits", [4, 8])
@pytest.mark.parametrize("N,T,C", [(16, 33, 3), (48, 1000, 2), (120, 64, 3), (272, 97, 2),
                                   (1024, 70, 1), (1000, 45, 2), (256, 130, 3), (128, 64, 2),
                                   (304, 200, 2)])
def test_tensor_tma_unpack_shapes(mw, bits, N, T, C):
    """Shapes the TMA tile unpack takes (N a multiple of 8 for 8-bit and of 16
    for 4-bit samples; inputs past N in the last tile read as zeros) and shapes
    that fall back to the other kernels, with ragged last time blocks."""
    spec = synth.Spec("tma", N, C, T, bits, seed=N + T + bits, sigma=2 if bits == 4 else 40,
                      tone_amp=0.3)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR), oracle_for(spec, range(C)), f"tma {N},{T},{C}")


@pytest.mark.parametrize("bits,N,T,C", [(8, 130, 1000, 3), (8, 202, 77, 4), (8, 1002, 45, 2),
                                        (4, 300, 1000, 3), (4, 52, 130, 5), (4, 1004, 65, 2),
                                        (4, 132, 20000, 1)])
def test_tile_unpack_thread_loaded_rows(mw, bits, N, T, C):
    """Sample rows that are whole 4-byte but not 16-byte units (2N bytes for
    8-bit, N for 4-bit samples): the tile unpack loads its raw box with the
    threads instead of TMA; inputs past N and samples past T read as zero."""
    spec = synth.Spec("tl", N, C, T, bits, seed=N + T, sigma=2 if bits == 4 else 40,
                      tone_amp=0.3)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR), oracle_for(spec, range(C)), f"tile {bits},{N},{T}")


@pytest.mark.parametrize("bits,N,T,C,G", [(8, 256, 1000, 12, 5), (8, 200, 77, 7, 3),
                                          (8, 1024, 100, 4, 1), (8, 136, 33, 5, 2),
                                          (4, 256, 1000, 12, 5), (4, 208, 77, 7, 3),
                                          (4, 144, 33, 5, 2)])
def test_overlapped_coresident_unpack(mw, bits, N, T, C, G):
    """pipeline 2 with the small unpack CTA beside the correlate on every SM:
    several channel groups (ragged last group), N not a multiple of 128 (the
    raw box reads past N as zeros), ragged last time block."""
    spec = synth.Spec("ov", N, C, T, bits, seed=N + T + C, sigma=40 if bits == 8 else 2,
                      tone_amp=0.3)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, pipeline=2, chan_group=G),
                 oracle_for(spec, range(C)), f"overlap {N},{T},{C},{G}")


def test_c0_both_engines(mw):
    spec = synth.spec_c0()
    ref = oracle_for(spec, range(spec.n_chan))
    assert_exact(run(mw, spec, mw.ENGINE_PLAIN), ref, "plain c0")
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR), ref, "tensor c0")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bits,flush", [(8, 1), (8, 2), (8, 5), (4, 1), (4, 3)])
def test_tensor_flush_segments(mw, bits, flush, shape):
    """Short FP32 segments: many int32 flushes per item, ragged last segment."""
    spec = synth.Spec("f", 200, 2, 1000, bits, seed=flush + bits, sigma=2 if bits == 4 else 60)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, flush_blocks=flush, mma_shape=shape),
                 oracle_for(spec, range(2)), f"flush {flush}")


def test_tensor_multiple_channel_groups(mw):
    spec = synth.Spec("g", 140, 7, 130, 4, seed=3, sigma=2)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, chan_group=3), oracle_for(spec, range(7)), "groups")


@pytest.mark.parametrize("bits,N,T,C,G", [
    (4, 48, 100, 5, 0), (4, 136, 333, 4, 0), (4, 256, 2000, 5, 2), (4, 300, 1000, 3, 0),
    (4, 520, 130, 3, 2), (4, 640, 64, 3, 0), (4, 1024, 64, 2, 0), (4, 1100, 70, 1, 0),
    (4, 256, 65, 1, 0), (8, 200, 512, 3, 0), (8, 384, 100, 4, 3), (8, 1000, 33, 2, 0)])
def test_pair_mode_shapes(mw, bits, N, T, C, G):
    """Two tile pairs per work item: 1 to 9 tiles (shared items (I; J, J+1)
    with and without the diagonal tile, diagonal leftovers paired across
    channels, a last single item), odd and even channel counts, channel
    groups with a ragged last group (its own work list), ragged N and T."""
    spec = synth.Spec("pm", N, C, T, bits, seed=N + 3 * T + C, sigma=2 if bits == 4 else 40,
                      tone_amp=0.3)
    kw = {"chan_group": G} if G else {}
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, mma_shape=3, **kw), oracle_for(spec, range(C)),
                 f"pair {bits},{N},{T},{C},{G}")


def test_pair_mode_choice(mw):
    """Auto takes the fused pair mode for 4-bit exact jobs of at most two
    tiles with whole 16-input sample rows, the pair mode where the
    integration is one exact segment, and the checked single segment for
    longer exact jobs; explicit segments or shapes are kept; a pair or fused
    pair request that cannot be served is refused."""
    def info(*a, **kw):
        p = mw.Plan(*a, **kw)
        i = p.info()
        p.close()
        return i.mma_shape, i.checked_segment

    assert info(256, 2, 20000, 4) == (4, 0)
    assert info(64, 2, 1000, 4) == (4, 0)
    assert info(384, 2, 2000, 4) == (3, 0)  # three tiles
    assert info(200, 2, 2000, 4) == (3, 0)  # sample rows not whole 16-byte units
    assert info(256, 2, 2000, 4, mma_shape=3) == (3, 0)
    assert info(1024, 2, 2000, 4, mma_shape=4) == (4, 0)
    assert info(256, 2, 200000, 4) == (3, 1)  # longer than one exact segment: checked
    for bad in [dict(n=256, t=2000, bits=8), dict(n=200, t=2000, bits=4),
                dict(n=256, t=200000, bits=4)]:
        with pytest.raises(mw.MwaxError):
            mw.Plan(bad["n"], 2, bad["t"], bad["bits"], mma_shape=4)
    with pytest.raises(mw.MwaxError):
        mw.BatchPlan([(256, 2, 2000), (200, 2, 2000)], sample_bits=4, mma_shape=4)
    assert info(256, 2, 512, 8) == (3, 0)  # exactly one segment (16 blocks)
    assert info(256, 2, 20000, 8) == (3, 1)  # 8-bit, 16 blocks per exact segment
    assert info(256, 2, 513, 8, mma_shape=3) == (3, 1)
    assert info(256, 2, 20000, 8, mma_shape=1) == (1, 0)
    assert info(256, 2, 20000, 8, flush_blocks=16) == (1, 0)
    assert info(256, 2, 20000, 8, kind=mw.KIND_FP16) == (3, 0)
    with pytest.raises(mw.MwaxError):
        mw.Plan(256, 2, 2000, 4, mma_shape=3, flush_blocks=4)
    with pytest.raises(mw.MwaxError):
        mw.BatchPlan([(256, 2, 2000), (128, 2, 2000)], sample_bits=8, mma_shape=3)


# ---------------------------------------------------------------------------
# fused pair mode (mma_shape 4): converter warps write the operand tiles
# from the packed 4-bit samples, no unpack pass
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,T,C,G,ks", [
    (16, 33, 3, 0, 1), (48, 100, 5, 0, 1), (64, 1000, 5, 0, 0), (64, 1000, 3, 0, 8),
    (128, 64, 3, 0, 1), (144, 65, 2, 0, 1), (256, 2000, 5, 2, 1), (256, 640, 4, 3, 3),
    (272, 97, 2, 0, 1), (384, 333, 3, 2, 1), (512, 330, 2, 0, 2), (1024, 64, 2, 0, 1)])
def test_fused_pair_mode(mw, N, T, C, G, ks):
    """Every tile count from 1 to 8 (shared items with two and three tiles,
    diagonal leftovers paired across channels, a last single item), the last
    tile partly filled (N = 144, 272: inputs past N read as zero), ragged
    last time blocks (one sample in the last block at T = 65), channel groups
    with a ragged last group, time ranges per item (automatic at 64 inputs);
    bit-exact on the first call and on a second call into the same buffer."""
    spec = synth.Spec("fu", N, C, T, 4, seed=N + 7 * T + C, sigma=2, tone_amp=0.3)
    v = device_volt(spec)
    kw = {"chan_group": G} if G else {}
    if ks:
        kw["k_split"] = ks
    p = mw.Plan(N, C, T, 4, mma_shape=4, **kw)
    inf = p.info()
    assert inf.mma_shape == 4 and inf.scratch_bytes == 0
    if ks:
        assert inf.k_split == ks
    out = p.correlate(v)
    out = p.correlate(v, out)
    assert p.status() == 0
    assert_exact(out.cpu().numpy(), oracle_for(spec, range(C)), f"fused {N},{T},{C},{G},{ks}")
    p.close()


def test_fused_pair_batch(mw):
    """A batch of small 4-bit jobs (every job at most two tiles with whole
    16-input rows) takes the fused pair mode: one persistent launch reading
    every job's voltages, no unpack graph, no operand buffers; bit-exact per
    job, on the first call and again on new buffers (the graph is rebuilt)."""
    import torch

    jobs = [(48, 5, 300), (128, 3, 400), (256, 2, 700), (16, 4, 65)]
    specs = [synth.Spec(f"fb{k}", n, c, t, 4, seed=90 + k, sigma=2, tone_amp=0.3)
             for k, (n, c, t) in enumerate(jobs)]
    bp = mw.BatchPlan(jobs, sample_bits=4)
    inf = bp.info()
    assert inf.mma_shape == 4 and inf.scratch_bytes == 0
    for rep in range(2):
        vs = [device_volt(s) for s in specs]
        bp.set_timing(True)
        outs = bp.correlate(vs)
        t = bp.timing()
        assert bp.status() == 0
        assert t.unpack_launches == 0 and t.correlate_launches == 1
        for s, o in zip(specs, outs):
            assert_exact(o.cpu().numpy(), oracle_for(s, range(s.n_chan)), f"fused batch {s.name}")
    bp.close()
    torch.cuda.synchronize()


def test_fused_pair_largest_single_segment(mw):
    """All samples (7, 7) over the longest 4-bit integration that is one exact
    segment: V_ii = 98 T = 16,771,328, just below 2^24."""
    T = 2674 * 64
    spec = synth.Spec("fmax", 144, 1, T, 4, seed=0, kind=synth.SYNTH_CONST, c_re=7, c_im=7)
    out = run(mw, spec, mw.ENGINE_TENSOR, mma_shape=4)
    assert out[0, 0, 0] == 98 * T == 16_771_328 and out[0, 0, 1] == 0
    assert_exact(out, oracle_for(spec, [0]), "fused max")


def test_fused_pair_big_then_small(mw):
    spec = synth.Spec("fbs", 144, 2, 20000, 4, seed=11, kind=synth.SYNTH_BIGSMALL, t_split=19000)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, mma_shape=4), oracle_for(spec, range(2)),
                 "fused big-small")


def _volt8(arr):
    """[chan][time][input] complex integers -> packed 8+8-bit bytes (host)
    and a device copy of them."""
    import torch

    raw = np.empty(arr.shape + (2,), np.int8)
    raw[..., 0] = arr.real
    raw[..., 1] = arr.imag
    host = raw.view(np.uint8).ravel().copy()
    return host, torch.from_numpy(host.copy()).cuda()


def test_checked_segment_adapts_to_full_scale_input(mw):
    """Every channel at full scale: the first call recomputes them all; the
    plan then runs the narrow shape for the next 8 calls (nothing recomputed)
    and tries the one-segment pass again on the 10th.  Exact every time."""
    import torch

    N, C, T = 200, 8, 2000
    rng = np.random.default_rng(10)
    x = rng.choice([-127, 127], (C, T, N)) + 1j * rng.choice([-127, 127], (C, T, N))
    host, v = _volt8(x)
    ref = oracle.correlate(host, 8, N, C, T)
    p = mw.Plan(N, C, T, 8)
    counts = []
    for call in range(10):
        out = p.correlate(v)
        assert p.status() == 0  # (synchronises: the next call sees this one's count)
        counts.append(p.recomputed_channels())
        if call in (0, 1, 9):
            assert_exact(out.cpu().numpy(), ref, f"adaptive call {call}")
    assert counts == [C] + [0] * 8 + [C]
    p.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("group", [0, 2])
def test_checked_segment_recomputes_only_flagged_channels(mw, group):
    """8-bit, T = 2000 (125 blocks, 8 exact segments): channels 1 and 4 carry
    full-scale samples (Re V_ii = 2000 * 2 * 127^2 > 2^24), the others sigma
    20 noise.  The one-segment pass is inexact on channels 1 and 4 only; the
    check flags exactly those two and the narrow recompute makes the whole
    output bit-exact, also across channel groups."""
    import torch

    N, C, T = 200, 6, 2000
    rng = np.random.default_rng(9)
    x = np.clip(np.rint(rng.normal(0, 20, (C, T, N, 2))), -127, 127)
    x = x[..., 0] + 1j * x[..., 1]
    for c in (1, 4):
        x[c] = rng.choice([-127, 127], (T, N)) + 1j * rng.choice([-127, 127], (T, N))
    host, v = _volt8(x)
    kw = {"chan_group": group} if group else {}
    p = mw.Plan(N, C, T, 8, **kw)
    assert p.info().checked_segment == 1
    out = p.correlate(v)
    assert p.status() == 0
    assert p.recomputed_channels() == 2
    assert p.recomputed_channels() == 0  # read-and-clear
    assert_exact(out.cpu().numpy(), oracle.correlate(host, 8, N, C, T), "checked")
    p.close()
    torch.cuda.synchronize()


def test_pair_mode_largest_single_segment(mw):
    """4-bit samples all (7, 7) over the longest integration that is still one
    exact segment (2674 blocks of 64 samples): V_ii = 98 T = 16,771,328, just
    below 2^24, accumulated in FP32 tensor memory without any flush."""
    T = 2674 * 64
    spec = synth.Spec("pmax", 130, 1, T, 4, seed=0, kind=synth.SYNTH_CONST, c_re=7, c_im=7)
    out = run(mw, spec, mw.ENGINE_TENSOR, mma_shape=3)
    assert out[0, 0, 0] == 98 * T == 16_771_328 and out[0, 0, 1] == 0
    assert_exact(out, oracle_for(spec, [0]), "pair max")


@pytest.mark.parametrize("shape", SHAPES_ONE_SEGMENT)
@pytest.mark.parametrize("bits", [4, 8])
def test_exact_window_big_then_small(mw, bits, shape):
    """Accumulator near the top of its segment window, then +-1 addends: any
    loss of low-order bits in the tensor-core accumulation shows up."""
    T = 20000 if bits == 4 else 2000
    split = 19000 if bits == 4 else 500
    spec = synth.Spec("bs", 130, 2, T, bits, seed=11, kind=synth.SYNTH_BIGSMALL, t_split=split)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, mma_shape=shape), oracle_for(spec, range(2)),
                 "big-small")


@pytest.mark.parametrize("shape", SHAPES_ONE_SEGMENT)
def test_exact_random_max_magnitude(mw, shape):
    spec = synth.Spec("rm", 256, 2, 3000, 8, seed=12, kind=synth.SYNTH_RANDMAX)
    assert_exact(run(mw, spec, mw.ENGINE_TENSOR, mma_shape=shape), oracle_for(spec, range(2)),
                 "randmax")


@pytest.mark.parametrize("bits", [4, 8])
@pytest.mark.parametrize("N", [200, 300])
def test_plain_random_max_magnitude(mw, bits, N):
    """Plain engine (32- and 64-input tiles) on samples at the ends of the
    supported range (its byte dot products negate the imaginary parts of the
    column inputs); T = 5001 cuts each channel's integration into ranges
    added with integer atomics, and leaves a last sample without a partner."""
    spec = synth.Spec("rmp", N, 2, 5001, bits, seed=13 + N, kind=synth.SYNTH_RANDMAX)
    assert_exact(run(mw, spec, mw.ENGINE_PLAIN), oracle_for(spec, range(2)),
                 f"randmax plain {bits} {N}")


def test_int32_bound_at_max_integration(mw):
    """All samples (127, 127) at the largest allowed T: V_ii = 2,147,479,576."""
    T = mw.max_n_time(8)
    spec = synth.Spec("cmax", 3, 1, T, 8, seed=0, kind=synth.SYNTH_CONST, c_re=127, c_im=127)
    out = run(mw, spec, mw.ENGINE_TENSOR)
    assert out[0, 0, 0] == 2_147_479_576 and out[0, 0, 1] == 0
    assert_exact(out, oracle_for(spec, [0]), "bound")
    out = run(mw, spec, mw.ENGINE_PLAIN)
    assert out[0, 0, 0] == 2_147_479_576


def test_quarter_tone_closed_form(mw):
    N, T = 150, 999
    rng = np.random.default_rng(2)
    c = rng.integers(-7, 8, (N, 2))
    spec = synth.Spec("q", N, 1, T, 4, seed=0, kind=synth.SYNTH_QUARTER, ci=c)
    out = run(mw, spec, mw.ENGINE_TENSOR)[0]
    cc = c[:, 0] + 1j * c[:, 1]
    ii, jj = np.tril_indices(N)
    e = T * cc[ii] * np.conj(cc[jj])
    np.testing.assert_array_equal(out[:, 0], e.real.astype(np.int64))
    np.testing.assert_array_equal(out[:, 1], e.imag.astype(np.int64))


@pytest.mark.parametrize("shape", [0, 1, 3])
def test_fp16_variant_error(mw, shape):
    """FP16 inputs, FP32 accumulation without integer flushes: error against
    the exact (int64 = FP64-exact) oracle stays within the FP32 summation
    bound 2T * 2^-24 (autos-normalised).  Auto picks the pair mode (one
    segment); 1 forces the narrow shape."""
    import torch

    spec = synth.Spec("h", 300, 3, 10000, 8, seed=21, sigma=20)
    v = device_volt(spec)
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8, kind=mw.KIND_FP16, mma_shape=shape)
    assert p.info().mma_shape == (3 if shape == 0 else shape)
    out = p.correlate(v)
    assert p.status() == 0
    got = out.cpu().numpy().astype(np.float64)
    _, ref = oracle_for(spec, range(spec.n_chan), want64=True)
    N = spec.n_inputs
    ii, jj = np.tril_indices(N)
    auto = ref[:, [oracle.baseline_index(i, i) for i in range(N)], 0].astype(np.float64)
    norm = np.sqrt(auto[:, ii] * auto[:, jj])
    err = np.abs(got - ref).max(axis=2) / norm
    assert err.max() <= 2 * spec.n_time * 2.0**-24
    p.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("shape", [0, 1])
def test_fp16_variant_error_full_scale(mw, shape):
    """Full-scale 8-bit input (every component +-127) at T = 10000: the autos
    reach 2 * 127^2 * T = 3.2e8 > 2^24, so the FP32 sums do round.  The error
    against the exact oracle is non-zero and within the FP32 summation bound
    2T * 2^-24 (autos-normalised), and the exact kind on the same input is
    still bit-exact."""
    import torch

    spec = synth.Spec("hfs", 256, 2, 10000, 8, seed=23, kind=synth.SYNTH_RANDMAX)
    v = device_volt(spec)
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8, kind=mw.KIND_FP16, mma_shape=shape)
    out = p.correlate(v)
    assert p.status() == 0
    got = out.cpu().numpy().astype(np.float64)
    p.close()
    exact, ref = oracle_for(spec, range(spec.n_chan), want64=True)
    N = spec.n_inputs
    ii, jj = np.tril_indices(N)
    auto = ref[:, [oracle.baseline_index(i, i) for i in range(N)], 0].astype(np.float64)
    assert auto.min() == 2 * 127**2 * spec.n_time
    norm = np.sqrt(auto[:, ii] * auto[:, jj])
    abs_err = np.abs(got - ref).max(axis=2)
    err = abs_err / norm
    assert 0 < err.max() <= 2 * spec.n_time * 2.0**-24, err.max()
    assert abs_err.max() >= 1.0  # FP32 rounding really happened
    q = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 8)
    assert_exact(q.correlate(v).cpu().numpy(), exact, "exact kind, full scale")
    q.close()
    torch.cuda.synchronize()


def test_batch_uneven_jobs(mw):
    import torch

    jobs = [(48, 4, 200), (128, 3, 500), (300, 2, 1000), (130, 2, 70)]
    specs = [synth.Spec(f"b{k}", n, c, t, 4, seed=40 + k, sigma=2, tone_amp=0.3)
             for k, (n, c, t) in enumerate(jobs)]
    bp = mw.BatchPlan(jobs, sample_bits=4)
    vs = [device_volt(s) for s in specs]
    outs = bp.correlate(vs)
    outs = bp.correlate(vs, outs)  # graph replay
    assert bp.status() == 0
    for s, o in zip(specs, outs):
        assert_exact(o.cpu().numpy(), oracle_for(s, range(s.n_chan)), s.name)
    bp.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("engine", [0, 1])
def test_host_buffers(mw, engine):
    import torch

    spec = synth.spec_c0()
    h = torch.from_numpy(synth.fill_host(spec).ravel()).pin_memory()
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 4, engine=engine, chan_group=7)
    out = torch.empty((spec.n_chan, spec.n_inputs * (spec.n_inputs + 1) // 2, 2),
                      dtype=torch.int32).pin_memory()
    p.set_timing(True)
    p.correlate_host(h, out)
    tm = p.timing()
    assert p.status() == 0
    assert_exact(out.numpy(), oracle_for(spec, range(spec.n_chan)), "host path")
    # the timing hook saw every copy: 64 channels in groups of 7 -> 10 copies each way
    assert tm.h2d_copies == 10 and tm.d2h_copies == 10
    assert tm.h2d_bytes == h.numel() and tm.d2h_bytes == out.numel() * 4
    assert tm.h2d_ms > 0 and tm.d2h_ms > 0
    p.close()


def test_shape_mismatch_and_host_pointer_rejected(mw):
    import torch

    p = mw.Plan(8, 2, 10, 4)
    v = torch.zeros(8 * 2 * 10, dtype=torch.uint8, device="cuda")
    out = p.empty_out()
    assert mw.lib().mwax_correlate(p._h, v.data_ptr(), 8, 3, 10, out.data_ptr()) == 2
    hv = torch.zeros(8 * 2 * 10, dtype=torch.uint8)
    assert mw.lib().mwax_correlate(p._h, hv.data_ptr(), 8, 2, 10, out.data_ptr()) == 1
    p.close()


def test_unaligned_buffers_rejected(mw):
    """Device buffers that do not start on a 16-byte boundary are refused
    before any launch (the unpack and dump kernels use vector accesses)."""
    import torch

    p = mw.Plan(16, 2, 64, 4)
    v = torch.zeros(16 * 2 * 64 + 16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(p.empty_out().numel() + 4, dtype=torch.int32, device="cuda")
    L = mw.lib()
    assert L.mwax_correlate(p._h, v.data_ptr() + 1, 16, 2, 64, out.data_ptr()) == 1
    assert L.mwax_correlate(p._h, v.data_ptr(), 16, 2, 64, out.data_ptr() + 4) == 1
    assert L.mwax_correlate(p._h, v.data_ptr(), 16, 2, 64, out.data_ptr()) == 0
    assert p.status() == 0
    p.close()
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times,
# checked on sampled channels the oracle recomputes one by one
# ---------------------------------------------------------------------------
def _full_size(mw, spec, chans, **kw):
    import torch

    v = device_volt(spec)
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, spec.sample_bits, **kw)
    out = p.correlate(v)
    assert p.status() == 0
    del v
    got = out[list(chans)].cpu().numpy()
    del out
    p.close()
    torch.cuda.empty_cache()
    assert_exact(got, oracle_for(spec, chans), spec.name)


@pytest.mark.parametrize("shape", SHAPES_ONE_SEGMENT + [4])
def test_full_size_c1_sampled(mw, shape):
    spec = synth.spec_c1()
    _full_size(mw, spec, [0, 1, 383, 766, 767], mma_shape=shape)


def test_full_size_c2_overlapped_sampled(mw):
    spec = synth.spec_c2()
    _full_size(mw, spec, [0, 208, 209, 1500, 3071], pipeline=2)


@pytest.mark.parametrize("shape", [0] + SHAPES)
def test_full_size_c2_sampled(mw, shape):
    spec = synth.spec_c2()
    rng = np.random.default_rng(2)
    chans = sorted(set([0, spec.n_chan - 1] + rng.choice(spec.n_chan, 6, replace=False).tolist()))
    _full_size(mw, spec, chans, mma_shape=shape)


def test_full_size_c3_batched_sampled(mw):
    """The batched workload as the benchmark runs it: all four jobs (48, 128,
    300 and 1024 inputs; 256 .. 3072 channels; T up to 20000) in one batch
    plan (one graph of unpacks, one persistent correlate launch), checked on
    sampled channels of every job (first, last and one inside)."""
    import torch

    specs = [synth.spec_c3(j) for j in range(4)]
    torch.cuda.empty_cache()
    vs = [device_volt(s) for s in specs]
    bp = mw.BatchPlan([(s.n_inputs, s.n_chan, s.n_time) for s in specs], sample_bits=4)
    outs = bp.correlate(vs)
    assert bp.status() == 0
    picks = []
    for s, o in zip(specs, outs):
        chans = [0, s.n_chan // 3, s.n_chan - 1]
        picks.append((s, chans, o[chans].cpu().numpy()))
    bp.close()
    del vs, outs
    torch.cuda.empty_cache()
    for s, chans, got in picks:
        assert_exact(got, oracle_for(s, chans), s.name)


# ---------------------------------------------------------------------------
# time ranges per work item (k_split): partial sums added with int32 atomics
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bits,N,T,C,G,ks", [
    (4, 64, 1000, 5, 0, 2), (4, 64, 1000, 3, 0, 8), (4, 200, 333, 4, 3, 3), (4, 300, 640, 2, 0, 5),
    (8, 100, 500, 3, 0, 2), (8, 256, 2000, 3, 2, 4), (8, 130, 96, 2, 0, 1)])
def test_split_items_exact(mw, bits, N, T, C, G, ks):
    """Every pair-mode item cut into ks time ranges (ragged range lengths,
    channel groups with a ragged last group, the 8-bit checked segment at
    T = 2000): bit-exact, and a second call on the same output buffer too
    (the plan zeroes it before adding)."""
    import torch

    spec = synth.Spec("ks", N, C, T, bits, seed=N + T + ks, sigma=2 if bits == 4 else 40,
                      tone_amp=0.3)
    v = device_volt(spec)
    kw = {"chan_group": G} if G else {}
    p = mw.Plan(N, C, T, bits, mma_shape=3, k_split=ks, **kw)
    assert p.info().k_split == ks
    out = p.correlate(v)
    out = p.correlate(v, out)
    assert p.status() == 0
    assert_exact(out.cpu().numpy(), oracle_for(spec, range(C)), f"split {ks}")
    p.close()
    torch.cuda.synchronize()


def test_split_auto_for_small_jobs(mw):
    """A job whose items cannot fill the SMs gets time ranges automatically
    (c0: 32 two-diagonal items on 152 SMs -> 4 ranges); a large one does not;
    the host-buffer path with ranges is exact."""
    import torch

    spec = synth.spec_c0()
    p = mw.Plan(spec.n_inputs, spec.n_chan, spec.n_time, 4)
    ks = p.info().k_split
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ks > 1 and p.info().work_items * 1 <= sms * 8
    ref = oracle_for(spec, range(spec.n_chan))
    assert_exact(p.correlate(device_volt(spec)).cpu().numpy(), ref, "auto split")
    h = torch.from_numpy(synth.fill_host(spec).ravel()).pin_memory()
    out = torch.empty((spec.n_chan, spec.n_inputs * (spec.n_inputs + 1) // 2, 2),
                      dtype=torch.int32).pin_memory()
    p.correlate_host(h, out)
    assert p.status() == 0
    assert_exact(out.numpy(), ref, "auto split, host buffers")
    p.close()
    q = mw.Plan(1024, 64, 2000, 4)
    assert q.info().k_split == 1
    q.close()


def test_split_rejected_where_it_cannot_apply(mw):
    with pytest.raises(mw.MwaxError) as e:
        mw.Plan(100, 2, 1000, 8, kind=mw.KIND_FP16, k_split=2)  # float sums: no atomics
    assert e.value.status == mw.STATUS_BY_NAME["MWAX_ERR_UNSUPPORTED"]
    with pytest.raises(mw.MwaxError) as e:
        mw.Plan(100, 2, 100, 4, k_split=2)  # 2 time blocks: fewer than 2 per range
    assert e.value.status == mw.STATUS_BY_NAME["MWAX_ERR_UNSUPPORTED"]
    with pytest.raises(mw.MwaxError) as e:
        mw.Plan(100, 2, 1000, 4, mma_shape=1, k_split=2)  # narrow shape: not pair mode
    assert e.value.status == mw.STATUS_BY_NAME["MWAX_ERR_UNSUPPORTED"]
    with pytest.raises(mw.MwaxError) as e:
        mw.Plan(100, 2, 1000, 4, k_split=9)
    assert e.value.status == mw.STATUS_BY_NAME["MWAX_ERR_INVALID_ARG"]


def test_batch_per_job_split(mw):
    """One persistent launch in which the jobs take different time ranges per
    item (each job's own k_split): bit-exact for every job, twice."""
    import torch

    jobs = [(48, 6, 2000), (128, 3, 700), (300, 2, 1000)]
    specs = [synth.Spec(f"bk{k}", n, c, t, 4, seed=80 + k, sigma=2, tone_amp=0.3)
             for k, (n, c, t) in enumerate(jobs)]
    vs = [device_volt(s) for s in specs]
    bp = mw.BatchPlan(jobs, k_split=[4, 1, 3])
    assert bp.info().k_split == 4
    outs = bp.correlate(vs)
    outs = bp.correlate(vs, outs)
    assert bp.status() == 0
    for s, o in zip(specs, outs):
        assert_exact(o.cpu().numpy(), oracle_for(s, range(s.n_chan)), s.name)
    bp.close()
    torch.cuda.synchronize()
