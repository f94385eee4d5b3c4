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


def test_linear_chirp_from_two_series(oracle):
    """A voice with m = 2, n = -1 whose fundamental phases are both quadratic:
    Phi_V = m Phi_phi + n Phi_r is a linear chirp's phase with f0 = m p1 + n q1 and
    Fdot = m p2 + n q2, so the closed form holds with the n Omega_r term of the
    frequency track and the n Phi_r term of the phase at full weight (the other
    closed forms have n = 0)."""
    import mpmath as mp
    from scipy.interpolate import CubicSpline
    from paper_2307_12585_gb300.synth import Waveform
    rng = np.random.default_rng(3)
    K, T = 41, 1e6
    t = np.concatenate([[0.0], np.sort(rng.uniform(0, T, K - 2)), [T]])
    m, n = 2, -1
    p1, p2, c1 = 0.8e-3, 0.7e-9, 0.2      # Phi_phi = 2 pi (p1 t + p2 t^2/2) + c1
    q1, q2, c2 = 0.6e-3, 0.4e-9, -0.1     # Phi_r   = 2 pi (q1 t + q2 t^2/2) + c2
    tp = 2 * math.pi
    pp, pr = tp * (p1 * t + p2 * t * t / 2) + c1, tp * (q1 * t + q2 * t * t / 2) + c2
    amp = 0.7 + 0.4j
    freqs = np.linspace(0.8e-3, 2.2e-3, 3000)
    w = Waveform(t, pp, pr, tp * (p1 + p2 * t), tp * (q1 + q2 * t), np.array([3], np.int32), np.array([m], np.int32),
                 np.array([n], np.int32), np.full((1, K), amp, np.complex128), 0.9, 0.4, 1.0, freqs)
    got = _voice(oracle, w) / amp
    # expected: the chirp's transform, with the spline of the combined phase knots' rounding
    mp.mp.dps = 40
    P = [mp.mpf(x) for x in (p1, p2, c1, q1, q2, c2)]
    f0, fd = m * P[0] + n * P[3], m * P[1] + n * P[4]
    P0 = m * P[2] + n * P[5]
    exact = lambda x: 2 * mp.pi * (f0 * x + fd * x * x / 2) + P0
    d = np.array([float(m * mp.mpf(float(pp[k])) + n * mp.mpf(float(pr[k])) - exact(mp.mpf(float(t[k])))) for k in range(K)])
    corr = CubicSpline(t, d, bc_type="not-a-knot")
    exp = np.zeros(freqs.shape, np.complex128)
    for i, fi in enumerate(freqs):
        x = mp.mpf(fi) - f0
        if not (0 <= x < fd * T):
            continue
        psi = mp.pi * x * x / fd - P0 - mp.pi / 4 - float(corr(float(x / fd)))
        exp[i] = complex(mp.cos(psi), mp.sin(psi)) / math.sqrt(float(fd))
    assert np.count_nonzero(exp) > 1000
    assert np.array_equal(got != 0, exp != 0)
    err = np.abs(got - exp) / np.abs(exp).max()
    assert err.max() < TOL


@pytest.mark.parametrize("uniform", [False, True])
def test_quadratic_turning_point(oracle, uniform):
    w, p = AN.quadratic_voice(K=40, uniform=True) if uniform else AN.quadratic_voice()
    # plus a dense cluster just below the turnover frequency; with uniform knots the
    # turnover is mid-segment, so both roots of these bins fall in the segment that
    # holds it (its split into monotone pieces is exercised)
    w = w.with_freqs(np.unique(np.concatenate([w.freqs, p["Fs"] * (1 - np.logspace(-5.9, -3.3, 160))])))
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
