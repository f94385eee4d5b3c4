"""Pins of the oracle's time-domain voice sum (Eq. 2), the input of the TD
comparator and of the brute-force DFT checks: a linear-chirp voice (quadratic
phase, constant amplitude), which the not-a-knot spline reproduces exactly,
has the closed form h(t) = A Y_lm e^{-i Phi(t)} (plus its partner
(-1)^l conj(A) Y_{l,-m} e^{+i Phi(t)}); samples after the last knot are 0."""
import math

import numpy as np

from tests import _analytic as AN


def test_linear_chirp_samples(oracle):
    w, p = AN.linear_chirp()
    dt = 37.0
    N = int(np.floor((w.t[-1] - w.t[0]) / dt)) + 50
    for conj in (False, True):
        tj, hp, hc = oracle.td_samples(w, dt, N, conj_partners=conj)
        Phi = 2 * math.pi * (p["f0"] * tj + 0.5 * p["fd"] * tj ** 2) + p["P0"]
        A = w.amp[0, 0]
        l, m = int(w.l[0]), int(w.m[0])
        h = A * oracle.swsh_closed(l, m, w.theta, w.phi) * np.exp(-1j * Phi)
        if conj:
            h += (-1) ** l * np.conj(A) * oracle.swsh_closed(l, -m, w.theta, w.phi) * np.exp(1j * Phi)
        h[tj > w.t[-1]] = 0
        got = hp - 1j * hc
        # the phase knots carry their FP64 rounding (~1e-16 x 6e3 rad), the spline adds no error
        assert np.max(np.abs(got - h)) < 1e-10 * np.max(np.abs(h))
        assert np.all(got[tj > w.t[-1]] == 0) and np.count_nonzero(tj > w.t[-1]) > 0
