"""Helpers for the GPU parity tests: device-side input fill, oracle on the
host-regenerated channels, element-by-element comparison."""
import numpy as np

import oracle
import synth


def device_volt(spec, chan0=0, n_chan=None):
    import torch

    n_chan = spec.n_chan - chan0 if n_chan is None else n_chan
    buf = torch.empty(n_chan * spec.n_time * spec.n_inputs * spec.bytes_per_sample,
                      dtype=torch.uint8, device="cuda")
    synth.fill_device(spec, buf, chan0=chan0, n_chan=n_chan)
    return buf


def oracle_for(spec, chans, want64=False):
    """Oracle visibilities for channels ``chans`` of ``spec`` (host regeneration)."""
    v = synth.fill_host(spec, chans=list(chans))
    return oracle.correlate(v, spec.sample_bits, spec.n_inputs, len(chans), spec.n_time,
                            want64=want64)


def assert_exact(gpu_out, ref, what=""):
    g = np.asarray(gpu_out)
    if not np.array_equal(g, ref):
        bad = np.argwhere(g != ref)
        c, b, k = bad[0]
        raise AssertionError(f"{what}: {len(bad)} mismatches; first at chan {c} baseline {b} "
                             f"part {k}: gpu {g[c, b, k]} oracle {ref[c, b, k]}")
