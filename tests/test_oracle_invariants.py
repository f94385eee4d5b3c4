"""Invariant pins of the oracle's SPA sum, each tied to a term of the method:
time shift (the 2 pi f t term, Eq. 3), azimuthal / radial phase offsets (the
m Phi_phi + n Phi_r voice phase, Eq. 1-2), the conjugate-partner voices and
the h = h+ - i hx split (Eq. 1), bin independence (Eq. 9 is evaluated per f),
and knot ownership (each crossing of a knot frequency counted once)."""
from fractions import Fraction
import math

import numpy as np
import pytest

from paper_2307_12585_gb300 import synth


def _rel(a, b):
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def _dyadic_config():
    """small config with knot times on multiples of 4096 s and phase knots on
    multiples of 2^-20 rad, so that shifts by dyadic amounts are exact"""
    w = synth.small_config(0, n_bins=2 ** 13)
    w.t = np.round(w.t / 4096.0) * 4096.0
    w.phi_phi = np.round(w.phi_phi * 2 ** 20) / 2 ** 20
    w.phi_r = np.round(w.phi_r * 2 ** 20) / 2 ** 20
    return w


def _exp_i2pi(x_frac):
    """e^{2 pi i x} for an exact rational x (reduced mod 1 exactly)"""
    r = x_frac - math.floor(x_frac)
    return complex(math.cos(2 * math.pi * float(r)), math.sin(2 * math.pi * float(r)))


def test_time_shift(oracle):
    w = _dyadic_config()
    hp, hc = oracle.sum_modes(w)
    tau0 = 3 * 2 ** 20
    w2 = synth.Waveform(**{k: getattr(w, k) for k in w.__dataclass_fields__})
    w2.t = w.t + tau0
    hp2, hc2 = oracle.sum_modes(w2)
    ph = np.array([_exp_i2pi(Fraction(float(f)) * tau0) for f in w.freqs])
    assert _rel(hp2, hp * ph) < 1e-12 and _rel(hc2, hc * ph) < 1e-12


@pytest.mark.parametrize("which", ["phi_phi", "phi_r"])
def test_phase_offset(oracle, which):
    w = _dyadic_config()
    delta = 0.25
    for j in range(w.n_modes):
        wj = w.with_modes([j])
        F = (wj.m[0] * wj.omega_phi + wj.n[0] * wj.omega_r)
        if not (np.all(F > 0) or np.all(F < 0)):
            continue
        hp, hc = oracle.sum_modes(wj)
        w2 = wj.with_freqs(wj.freqs)
        setattr(w2, which, getattr(wj, which) + delta)
        hp2, hc2 = oracle.sum_modes(w2)
        k = int(wj.m[0]) if which == "phi_phi" else int(wj.n[0])
        rot = np.exp(-1j * k * delta * np.sign(F[0]))
        if np.sum(np.abs(hp)) == 0:
            continue
        assert _rel(hp2, hp * rot) < 1e-12 and _rel(hc2, hc * rot) < 1e-12


def test_conj_partners_explicit(oracle):
    w = synth.small_config(0, n_bins=2 ** 13)
    hp, hc = oracle.sum_modes(w, conj_partners=True)
    e = w.with_modes(np.arange(w.n_modes))
    sgn = np.where(w.l % 2 == 0, 1.0, -1.0)
    e.l = np.concatenate([w.l, w.l]).astype(np.int32)
    e.m = np.concatenate([w.m, -w.m]).astype(np.int32)
    e.n = np.concatenate([w.n, -w.n]).astype(np.int32)
    e.amp = np.concatenate([w.amp, sgn[:, None] * np.conj(w.amp)])
    hp2, hc2 = oracle.sum_modes(e, conj_partners=False)
    assert _rel(hp2, hp) < 1e-14 and _rel(hc2, hc) < 1e-14


def test_bin_subset_is_exact(oracle):
    w = synth.small_config(0)
    hp, hc = oracle.sum_modes(w)
    rng = np.random.default_rng(5)
    sel = np.sort(rng.choice(w.n_freqs, 1000, replace=False))
    hp2, hc2 = oracle.sum_modes(w, freqs=w.freqs[sel])
    assert np.array_equal(hp2, hp[sel]) and np.array_equal(hc2, hc[sel])


def test_linearity_in_amplitude(oracle):
    w = synth.small_config(0, n_bins=2 ** 12)
    hp, hc = oracle.sum_modes(w, conj_partners=False)
    a = 0.3 - 1.7j
    w2 = w.with_freqs(w.freqs)
    w2.amp = w.amp * a
    hp2, hc2 = oracle.sum_modes(w2, conj_partners=False)
    H, H2 = hp - 1j * hc, hp2 - 1j * hc2          # = H(f) + 0 when no voice is negative
    Hm, Hm2 = hp + 1j * hc, hp2 + 1j * hc2        # = conj H(-f)
    assert _rel(H2, a * H) < 1e-14 and _rel(Hm2, np.conj(a) * Hm) < 1e-14


def test_knot_frequencies_owned_once(oracle):
    """bins placed exactly on the knot frequencies of one increasing voice:
    the half-open ownership counts each once, and the last knot not at all"""
    w = synth.small_config(0)
    j = int(np.nonzero((w.l == 2) & (w.m == 2) & (w.n == 0))[0][0])
    wj = w.with_modes([j])
    Fk = (2.0 * wj.omega_phi + 0.0 * wj.omega_r) / (2 * math.pi)
    assert np.all(np.diff(Fk) > 0)
    hp, hc, st = oracle.sum_modes(wj.with_freqs(Fk), conj_partners=False, return_stats=True)
    assert st["contributions"] == wj.K - 1
    assert np.all(np.abs(hp[:-1]) > 0) and hp[-1] == 0
