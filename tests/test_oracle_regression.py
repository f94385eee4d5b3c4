"""The oracle against its stored output (tests/golden/oracle_config0_sampled.txt,
written by tests/golden/make_oracle_regression.py from the oracle alone): a change
of the oracle's arithmetic beyond summation order shows up here, so it is made on
purpose, with the fixture rewritten by that script."""
import numpy as np

from tests.golden import make_oracle_regression as G


def test_oracle_matches_its_stored_output(oracle):
    ref = np.loadtxt(G.PATH)
    w = G.sample()
    assert np.array_equal(ref[:, 0], w.freqs)
    hp, hc = oracle.sum_modes(w)
    got = np.stack([hp.real, hp.imag, hc.real, hc.imag], axis=1)
    assert np.linalg.norm(got - ref[:, 1:]) <= 1e-13 * np.linalg.norm(ref[:, 1:])
    assert np.array_equal(got == 0, ref[:, 1:] == 0)
