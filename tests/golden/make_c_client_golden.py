"""Writes c_client_corr.txt: a small correlation case for the plain C client
(tests/c_client/abi_client.c) -- seeded 4+4-bit voltages from the shared input
generator and the visibilities the CPU oracle computes from them.

Run from the repository root:  python tests/golden/make_c_client_golden.py
Only the input generator (synth) and the oracle are called."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

N, C, T, BITS = 20, 2, 70, 4


def main():
    oracle.build()
    synth.build()
    spec = synth.Spec("c_client", N, C, T, BITS, seed=20, sigma=2, tone_amp=0.3)
    volt = synth.fill_host(spec)
    vis = oracle.correlate(volt, BITS, N, C, T)
    with open(os.path.join(HERE, "c_client_corr.txt"), "w") as f:
        f.write("# Plain-C client case: seeded 4+4-bit voltages [chan][time][input] (hex, one\n"
                "# byte per complex sample) and the oracle's int32 visibilities\n"
                "# [chan][b][re, im], b = i(i+1)/2 + j (paper Sec. 2: every pair of inputs\n"
                "# cross-correlated per channel, then integrated).  Written by\n"
                "# make_c_client_golden.py from the input generator and the CPU oracle.\n")
        f.write(f"{N} {C} {T} {BITS}\n")
        f.write(volt.tobytes().hex() + "\n")
        for c in range(C):
            f.write(" ".join(str(int(x)) for x in vis[c].ravel()) + "\n")


if __name__ == "__main__":
    main()
