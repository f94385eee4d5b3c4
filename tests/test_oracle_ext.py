"""Pins of the oracle's extended stationary-phase form (Sec. 2.2, Eq. 7-10).

Per root the extended form replaces the Fresnel value by
G = -(2/sqrt 3)(i Fdot/|Fddot|) e^z K_{1/3}(z), z = -2 pi i Fdot^3/(3 Fddot^2).
The oracle evaluates e^z K_{1/3}(z) by quadrature of an integral definition;
it is pinned here against an independent library routine (scipy's kv, AMOS),
against the standard SPA it must reduce to when Fddot -> 0, and, for a whole
sum, against the exact Fourier transform of a cubic-phase voice: its two
roots' extended contributions add up to an Airy function, at every bin below
the turnover, where the standard SPA diverges."""
import math

import numpy as np
import pytest

from tests import _analytic as AN


def _scipy_G(Fd, Fdd):
    from scipy.special import kv
    z = -2j * np.pi * Fd ** 3 / (3 * Fdd ** 2)
    return -(2 / np.sqrt(3)) * (1j * Fd / np.abs(Fdd)) * np.exp(z) * kv(1.0 / 3.0, z)


@pytest.mark.parametrize("Fdd", [1.0, -3e-18, 2.5e-15])
def test_factor_matches_library_bessel(oracle, Fdd):
    pytest.importorskip("scipy")
    X = np.concatenate([np.logspace(-9, 9, 181), -np.logspace(-9, 9, 181)])
    Fd = np.cbrt(3 * X * Fdd ** 2 / (2 * np.pi))
    got = oracle.ext_factor(Fd, np.full_like(Fd, Fdd))
    ref = _scipy_G(Fd, Fdd)
    assert np.max(np.abs(got / ref - 1)) < 1e-13


def test_factor_limits(oracle):
    pytest.importorskip("scipy")
    from scipy.special import airy, gamma
    # Fddot = 0: exactly the Fresnel value
    Fd = np.array([3e-9, -2e-11, 1.0])
    got = oracle.ext_factor(Fd, np.zeros(3))
    std = np.exp(-1j * np.sign(Fd) * np.pi / 4) / np.sqrt(np.abs(Fd))
    assert np.allclose(got, std, rtol=1e-15, atol=0)
    # |X| -> inf: 1 + a_1/z + a_2/z^2 + O(z^-3), a_k = prod_{j<=k} (4 nu^2 - (2j-1)^2)/(8j)
    # (Hankel's expansion): a_1 = -5/72, a_2 = 385/10368
    for X in (1e3, -1e3, 1e4, 1e7):
        Fdd = 1e-17
        Fd = np.cbrt(3 * X * Fdd ** 2 / (2 * np.pi))
        r = oracle.ext_factor(np.array([Fd]), np.array([Fdd]))[0] * np.sqrt(abs(Fd)) * np.exp(1j * np.sign(Fd) * np.pi / 4)
        z = -1j * X
        assert abs(r - (1 + (-5 / 72) / z + (385 / 10368) / z ** 2)) < 0.05 / abs(X) ** 3 + 2e-15
    # Fdot = 0 (a double root): the two-root limit 2 pi (pi |Fddot|)^{-1/3} Ai(0)
    for Fdd in (1.0, -4e-16):
        exp = 2 * np.pi * (np.pi * abs(Fdd)) ** (-1 / 3) * airy(0.0)[0]
        got = oracle.ext_factor(np.array([0.0]), np.array([Fdd]))[0]
        assert abs(got - exp) < 1e-14 * exp
        assert abs(exp - 2 * np.pi ** (2 / 3) / (3 ** (2 / 3) * gamma(2 / 3)) * abs(Fdd) ** (-1 / 3)) < 1e-14 * exp
    # mirror symmetry: G(-Fdot, Fddot) = conj G(Fdot, Fddot)
    Fd = np.array([2e-10]); Fdd = np.array([5e-18])
    gp, gm = oracle.ext_factor(Fd, Fdd)[0], oracle.ext_factor(-Fd, Fdd)[0]
    assert abs(gm - np.conj(gp)) < 1e-14 * abs(gp)
    # both zero: nothing
    assert oracle.ext_factor(np.array([0.0]), np.array([0.0]))[0] == 0


def _voice(oracle, w, spa):
    hp, hc = oracle.sum_modes(w, conj_partners=False, spa=spa)
    Y = oracle.swsh_closed(int(w.l[0]), int(w.m[0]), w.theta, w.phi)
    return (hp - 1j * hc) / (Y * w.prefactor) / w.amp[0, 0]


def airy_expected(p, f):
    """Exact Fourier transform of exp(-i Phi(t)), Phi = 2 pi [Fs tau - kappa tau^3/6] + Ps,
    tau = t - ts, over the whole line: e^{i(2 pi f ts - Ps)} 2 pi a Ai(-2 pi (Fs - f) a),
    a = (pi kappa)^{-1/3}."""
    from scipy.special import airy
    a = (math.pi * p["kappa"]) ** (-1.0 / 3.0)
    return np.exp(1j * (2 * math.pi * f * p["ts"] - p["Ps"])) * 2 * math.pi * a * airy(-2 * math.pi * (p["Fs"] - f) * a)[0]


def test_cubic_phase_voice_is_airy(oracle):
    """Both roots inside the trajectory (Fs - kappa (T - ts)^2/2 < f < Fs): the
    extended sum is the exact transform (to the knots' FP64 rounding, ~1e-12),
    including the bins next to the turnover.  Above Fs there is no root and
    the sum is 0 (the method sums over real roots only)."""
    pytest.importorskip("scipy")
    w, p = AN.quadratic_voice(nb=6000)
    f = np.concatenate([np.linspace(1.3e-3, 2.1e-3, 6000), p["Fs"] - np.logspace(-13, -6, 40)])
    f = np.unique(f)
    w = w.with_freqs(f)
    got = _voice(oracle, w, "extended")
    std = _voice(oracle, w, "standard")
    exp = airy_expected(p, f)
    lo = p["Fs"] - 0.5 * p["kappa"] * (p["T"] - p["ts"]) ** 2
    both = (f < p["Fs"]) & (f > lo * 1.0001)
    assert np.count_nonzero(both) > 2000
    scale = np.abs(exp[both]).max()
    err = np.abs(got[both] - exp[both]) / scale
    assert err.max() < 1e-11
    # within 1e-6 F* of the turnover the standard form is off by O(1); the extended one is not
    near = both & (np.abs(f - p["Fs"]) < 1e-6 * p["Fs"])
    assert np.count_nonzero(near) >= 20
    assert np.max(np.abs(std[near] - exp[near])) / scale > 0.1
    assert np.all(got[f > p["Fs"]] == 0)


def test_linear_chirp_unchanged(oracle):
    """Fddot = 0 in the trajectory's spline up to rounding: extended == standard."""
    w, p = AN.linear_chirp()
    a, b = _voice(oracle, w, "extended"), _voice(oracle, w, "standard")
    assert np.max(np.abs(a - b)) < 1e-12 * np.abs(b).max()


def test_extended_vs_standard_config(oracle):
    """On the 0.25-yr, 55-mode workload the two forms differ by O(1/X) away from
    turnovers and by O(1) next to them; conjugate-partner symmetry holds for
    both (sum with partners == sum of the listed modes + sum of the partners)."""
    from paper_2307_12585_gb300 import synth
    w = synth.small_config(0, n_bins=2 ** 12)
    he = oracle.sum_modes(w, spa="extended")
    hs = oracle.sum_modes(w, spa="standard")
    d = oracle.rel_l2(np.concatenate(he), np.concatenate(hs))
    assert 1e-9 < d < 1e-1
    # partners listed explicitly: (l, -m, -n) with (-1)^l conj(A)
    e = w.with_modes(np.arange(w.n_modes))
    sgn = np.where(w.l % 2 == 0, 1.0, -1.0)
    e.l = np.concatenate([w.l, w.l]).astype(np.int32)
    e.m = np.concatenate([w.m, -w.m]).astype(np.int32)
    e.n = np.concatenate([w.n, -w.n]).astype(np.int32)
    e.amp = np.concatenate([w.amp, sgn[:, None] * np.conj(w.amp)])
    hx = oracle.sum_modes(e, conj_partners=False, spa="extended")
    assert oracle.rel_l2(hx[0], he[0]) < 1e-13 and oracle.rel_l2(hx[1], he[1]) < 1e-13
