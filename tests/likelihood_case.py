"""Likelihood test inputs (Eq. 13-15): data = oracle waveform at slightly
offset parameters + Gaussian noise with Re, Im ~ N(0, S/(4 df)); the prefactor
is rescaled so that the injection's SNR (both channels, Eq. 13) is 78."""
import numpy as np

from paper_2307_12585_gb300 import synth


def make(oracle, w, seed=3, snr=78.0, df=None):
    df = df if df is not None else 1.0 / w.meta.get("T", w.t[-1] - w.t[0])
    S = synth.psd(w.freqs)
    hp, hc = oracle.sum_modes(w)
    rho = np.sqrt(oracle.inner(hp, hp, S, df) + oracle.inner(hc, hc, S, df))
    w = w.with_freqs(w.freqs)
    w.prefactor = float(w.prefactor * snr / rho)
    inj = w.with_freqs(w.freqs)
    inj.amp = w.amp * (1.0 + 0.01j)
    inj.phi_phi = w.phi_phi + 1e-3
    dp, dc = oracle.sum_modes(inj)
    rng = np.random.default_rng(seed)
    nz = lambda: synth.noise(rng, w.freqs, df)
    return w, dp + nz(), dc + nz(), S, df
