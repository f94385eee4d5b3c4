"""Closed-form pins of the oracle's SPA sum (Eq. 3 with the phase of Eq. 4;
standard-SPA limit of Eq. 10).  With conj_partners off and a voice whose
frequency stays positive, h+ - i hx = H(f) (h = h+ - i hx, Eq. 1), and
H(f) / Y_lm is the voice's stationary-phase transform.

The expected values carry the exact effect of the FP64 rounding of the phase
knots (the spline of the rounding errors), so what remains is the oracle's own
arithmetic.  Errors are measured against the largest |H| (at bins where the
two roots of a turning-point voice interfere, |H| itself is tiny)."""
import math

import numpy as np
import pytest

from tests import _analytic as AN

TOL = 1e-12


def _voice(oracle, w):
    hp, hc = oracle.sum_modes(w, conj_partners=False)
    Y = oracle.swsh_closed(int(w.l[0]), int(w.m[0]), w.theta, w.phi)
    return (hp - 1j * hc) / (Y * w.prefactor)


def test_linear_chirp(oracle):
    w, p = AN.linear_chirp()
    got = _voice(oracle, w) / w.amp[0, 0]
    exp = AN.linear_chirp_expected(w, p, w.freqs)
    assert np.count_nonzero(exp) > 1000
    assert np.array_equal(got != 0, exp != 0)          # the same bins are covered
    err = np.abs(got - exp) / np.abs(exp).max()
    assert err.max() < TOL


def test_quadratic_turning_point(oracle):
    w, p = AN.quadratic_voice()
    got = _voice(oracle, w) / w.amp[0, 0]
    exp = AN.quadratic_voice_expected(w, p, w.freqs)
    # Near the turnover F*, the FP64 rounding of F(t) - f (~1e-16 |F|) moves
    # the root by that over Fdot, and Fdot -> 0: the weight's relative error
    # grows like eps |F| Fddot / Fdot^2.  Bins within 1e-6 F* are excluded
    # (reported separately), bins within 1e-4 F* get the looser bound.
    dist = np.abs(w.freqs - p["Fs"]) / p["Fs"]
    far, near = dist > 1e-4, (dist > 1e-6) & (dist <= 1e-4)
    scale = np.abs(exp[dist > 1e-6]).max()
    assert np.count_nonzero(exp[far]) > 1000 and np.count_nonzero(exp[near]) >= 2
    assert np.array_equal((got != 0)[dist > 1e-6], (exp != 0)[dist > 1e-6])
    err = np.abs(got - exp) / scale
    assert err[far].max() < TOL
    assert err[near].max() < 1e-10
    # two roots (both branches) contribute below the turnover frequency
    two = (w.freqs < p["Fs"]) & (w.freqs > p["Fs"] - 0.5 * p["kappa"] * (p["T"] - p["ts"]) ** 2)
    assert np.count_nonzero(two) > 100


def test_power_law_chirp_converges(oracle):
    """configs' extra chirp voice: F = F0 (1 - t/tc)^(-3/8) sampled on K knots.
    The spline phase error is O(h^4) but the weight 1/sqrt|Fdot| uses the
    spline's derivative, which converges as O(h^3): the error must fall at
    least 8x per doubling of K, and reach < 3e-8 at K = 400."""
    from paper_2307_12585_gb300 import synth
    errs = []
    for K in (100, 200, 400):
        w, p = synth.chirp_config(K=K, n_bins=2 ** 12)
        sel = (w.freqs > 2.2e-4) & (w.freqs < 3.6e-4)
        w = w.with_freqs(w.freqs[sel])
        got = _voice(oracle, w)
        exp = AN.power_law_expected(p, w.freqs)
        errs.append(np.sqrt(np.sum(np.abs(got - exp) ** 2) / np.sum(np.abs(exp) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.5 < r1 < 45 and 7.5 < r2 < 45, errs
    assert errs[2] < 3e-8
