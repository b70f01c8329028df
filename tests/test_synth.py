"""Input generator checks (host side): Philox known answers against numpy,
sample statistics, subset regeneration, packing."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("key,ctr", [((5, 7), (1, 2, 3, 4)), ((0, 0), (0, 0, 0, 0)),
                                     ((2**64 - 1, 12345), (2**64 - 2, 0, 2**63, 99))])
def test_philox_matches_numpy(key, ctr):
    """numpy.random.Philox is Philox4x64-10; it bumps the counter before
    producing its first block."""
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
    ref = bg.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    np.testing.assert_array_equal(synth.philox4x64_10(c, key), ref)


def _vals(spec, chans=(0,), n_time=None):
    v = synth.fill_host(spec, chans=list(chans), n_time=n_time)
    return oracle.decode(v, spec.sample_bits)


@pytest.mark.parametrize("bits,sigma", [(4, 2), (8, 20)])
def test_noise_statistics(bits, sigma):
    spec = synth.Spec("s", 64, 4, 2000, bits, seed=9, sigma=sigma)
    re, im = _vals(spec, chans=range(4))
    n = re.size
    for x in (re, im):
        x = x.astype(np.float64)
        # rounding adds 1/12 variance; clipping at +-7 removes a little at sigma 2
        var_ref = sigma**2 + 1.0 / 12.0
        assert abs(x.mean()) < 5 * sigma / np.sqrt(n)
        assert abs(x.var() - var_ref) < 0.03 * var_ref + 5 * np.sqrt(2.0 / n) * var_ref
    m = 7 if bits == 4 else 127
    assert re.min() >= -m and re.max() <= m and im.min() >= -m and im.max() <= m


def test_subset_regeneration_matches_full_fill():
    spec = synth.spec_c0()
    full = synth.fill_host(spec)
    sub = synth.fill_host(spec, chans=[5, 63, 0])
    np.testing.assert_array_equal(sub[0], full[5])
    np.testing.assert_array_equal(sub[1], full[63])
    np.testing.assert_array_equal(sub[2], full[0])
    part = synth.fill_host(spec, chans=[7], t0=100, n_time=50)
    np.testing.assert_array_equal(part[0], full[7, 100:150])


def test_threads_do_not_change_samples():
    spec = synth.spec_c1().with_(n_time=64)
    a = synth.fill_host(spec, chans=[0, 700], threads=1)
    b = synth.fill_host(spec, chans=[0, 700], threads=7)
    np.testing.assert_array_equal(a, b)


def test_sources_are_correlated_across_inputs():
    """With injected sources the cross-power between two inputs is nonzero
    while pure noise gives ~0."""
    spec = synth.spec_c1().with_(n_time=4000)
    re, im = _vals(spec)
    x = (re + 1j * im).reshape(4000, spec.n_inputs)
    c = np.mean(x[:, 10] * np.conj(x[:, 11]))
    assert abs(c) > 0.3  # sources add sum_s A_s^2 ~ several units of cross-power
    spec0 = synth.Spec("n", 16, 1, 4000, 4, seed=1, sigma=2)
    re0, im0 = _vals(spec0)
    x0 = (re0 + 1j * im0).reshape(4000, 16)
    assert abs(np.mean(x0[:, 3] * np.conj(x0[:, 4]))) < 0.4


def test_pattern_kinds():
    T = 10
    s = synth.Spec("k", 3, 1, T, 8, seed=0, kind=synth.SYNTH_CONST, c_re=-127, c_im=5)
    re, im = _vals(s)
    assert (re == -127).all() and (im == 5).all()
    s = synth.Spec("b", 3, 1, T, 4, seed=0, kind=synth.SYNTH_BIGSMALL, t_split=4)
    re, im = _vals(s)
    re = re.reshape(T, 3)
    assert (re[:4] == 7).all() and set(np.abs(re[4:]).ravel()) == {1}
    s = synth.Spec("r", 3, 1, 200, 8, seed=0, kind=synth.SYNTH_RANDMAX)
    re, im = _vals(s)
    assert set(re.tolist()) == {-127, 127}
