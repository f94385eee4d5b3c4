"""Writes oracle_config0_sampled.txt: the CPU oracle's h+ and hx (Sec. 2.2, Eq. 3-6:
the SPA sum of every voice, conjugate partners implied) for the seeded 0.25-yr,
55-mode synthetic workload on 64 evenly spaced bins of its 2^15-bin grid.  Calls
only oracle/.  Rerun it (python -m tests.golden.make_oracle_regression) only with
a change to the oracle's arithmetic whose commit names the passage that justifies it."""
import os

import numpy as np

from oracle import oracle as O
from paper_2307_12585_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "oracle_config0_sampled.txt")


def sample():
    w = synth.small_config(0)
    idx = np.linspace(0, w.n_freqs - 1, 64).astype(np.int64)
    return w.with_freqs(w.freqs[idx])


def main():
    w = sample()
    hp, hc = O.sum_modes(w)
    with open(PATH, "w") as fh:
        fh.write("# CPU oracle, SPA sum (Sec. 2.2, Eq. 3-6), 0.25-yr 55-mode synthetic workload, seed 0,\n")
        fh.write("# 64 evenly spaced bins of the 2^15-bin grid; written by make_oracle_regression.py\n")
        fh.write("# f  Re h+  Im h+  Re hx  Im hx\n")
        for f, a, b in zip(w.freqs, hp, hc):
            fh.write("%.17g %.17g %.17g %.17g %.17g\n" % (f, a.real, a.imag, b.real, b.imag))


if __name__ == "__main__":
    main()
