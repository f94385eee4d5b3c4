"""Brute-force pin of the oracle's SPA sum: the DFT of the time-domain voice
sum (Eq. 2) built from the same knots with an independent spline and Y_lm
implementation, sampled at dt = 10 s (Nyquist far above every voice, Sec. 2.3),
with the e^{+2 pi i f t} sign of Eq. 3.  The SPA is an approximation, so the
check is a match (overlap of Eq. 12-13 with a flat PSD) above 0.999, away
from each voice's end frequencies (truncation edges, Fig. 1 upper panel) and
turnovers."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import synth


def _match(a, b):
    return float(np.real(np.vdot(a, b)) / np.sqrt(np.real(np.vdot(a, a)) * np.real(np.vdot(b, b))))


def _edges(w, conj):
    """end and turnover frequencies (Hz, signed) of every voice"""
    out = []
    for j in range(w.n_modes):
        F = (w.m[j] * w.omega_phi + w.n[j] * w.omega_r) / (2 * np.pi)
        out += [F[0], F[-1]]
        dF = np.diff(F)
        out += list(F[1:-1][np.sign(dF[1:]) != np.sign(dF[:-1])])
    out = np.array(out)
    return np.concatenate([out, -out]) if conj else out


@pytest.mark.parametrize("modes", [[(2, 2, 0)], [(2, 1, -3)], [(2, 2, 0), (3, 3, 2), (2, 1, -3), (3, 1, 1)]])
def test_spa_matches_dft_of_time_domain(oracle, modes):
    base = synth.small_config(0)
    idx = [int(np.nonzero((base.l == l) & (base.m == m) & (base.n == n))[0][0]) for (l, m, n) in modes]
    w = base.with_modes(idx)
    fk, Hp, Hc = oracle.td_dft(w, dt=10.0, conj_partners=True)
    sel = (fk > 5e-5) & (fk < 6e-3)
    fk, Hp, Hc = fk[sel], Hp[sel], Hc[sel]
    hp, hc = oracle.sum_modes(w, freqs=fk, conj_partners=True)
    edges = _edges(w, True)
    clean = np.min(np.abs(fk[:, None] - edges[None, :]), axis=1) > 6e-5
    assert np.count_nonzero(clean & (np.abs(hp) > 0)) > 300
    for a, b in ((hp, Hp), (hc, Hc)):
        assert _match(a[clean], b[clean]) > 0.999
    # where the SPA has no voice, the DFT holds only leakage
    empty = clean & (np.abs(hp) == 0)
    if np.any(empty):
        assert np.sum(np.abs(Hp[empty]) ** 2) < 1e-2 * np.sum(np.abs(Hp[clean]) ** 2)


def test_turning_point_voice_matches_dft_away_from_turnover(oracle):
    base = synth.small_config(0)
    # (l, m, n) = (2, 1, -5): F = (Om_phi - 5 Om_r)/2pi < 0 with a minimum inside
    # the trajectory, so both the turnover and the conj H(-f) branch are used
    j = int(np.nonzero((base.l == 2) & (base.m == 1) & (base.n == -5))[0][0])
    w = base.with_modes([j])
    F = (w.omega_phi - 5 * w.omega_r) / (2 * np.pi)
    assert 0 < np.argmin(F) < w.K - 1 and np.all(F < 0)
    fk, Hp, Hc = oracle.td_dft(w, dt=10.0, conj_partners=True)
    sel = (fk > 5e-5) & (fk < 6e-3)
    fk, Hp, Hc = fk[sel], Hp[sel], Hc[sel]
    hp, hc = oracle.sum_modes(w, freqs=fk, conj_partners=True)
    edges = _edges(w, True)
    clean = np.min(np.abs(fk[:, None] - edges[None, :]), axis=1) > 3e-5
    assert np.count_nonzero(clean & (np.abs(hp) > 0)) > 300
    for a, b in ((hp, Hp), (hc, Hc)):
        assert _match(a[clean], b[clean]) > 0.99
