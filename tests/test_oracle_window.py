"""Pins of the frequency-domain Hann window (Sec. 2.3: the FD waveform is
convolved with the transform of the window applied to the TD waveform).

1. The three-term form is exact for the DFT: for any samples x_j and the
   periodic Hann window w_j = sin^2(pi j/N), DFT(w x)[k] = X[k]/2 - X[k-1]/4
   - X[k+1]/4 (checked on the brute-force TD voice sum, so the weights and the
   neighbour alignment are pinned by an independent computation).
2. Applied to the SPA sum it agrees with the DFT of the windowed TD signal
   (match > 0.999 away from voice edges), and, over the whole band, windowing
   brings the two closer than without it (the paper's leakage argument)."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import synth


def _match(a, b):
    return float(np.real(np.vdot(a, b)) / np.sqrt(np.real(np.vdot(a, a)) * np.real(np.vdot(b, b))))


def test_three_term_form_is_exact_on_dft(oracle):
    base = synth.small_config(0)
    w = base.with_modes([3, 17, 30])
    fk, Hp, Hc = oracle.td_dft(w, dt=20.0)
    fkw, Wp, Wc = oracle.td_dft(w, dt=20.0, window="hann")
    assert np.array_equal(fk, fkw)
    # interior bins: both neighbours are on the grid (k = 1..N/2-1 has them inside 0..N/2)
    for X, W in ((Hp, Wp), (Hc, Wc)):
        pred = oracle.hann_fd(X)
        err = np.abs(pred[1:-1] - W[1:-1]).max() / np.abs(W).max()
        assert err < 1e-11


def test_hann_fd_definition(oracle):
    O = oracle
    h = np.array([1 + 2j, -3.0, 0.5j, 4.0])
    got = O.hann_fd(h)
    exp = np.array([0.5 * h[0] - 0.25 * h[1], 0.5 * h[1] - 0.25 * (h[0] + h[2]),
                    0.5 * h[2] - 0.25 * (h[1] + h[3]), 0.5 * h[3] - 0.25 * h[2]])
    assert np.array_equal(got, exp)
    # linearity and the DC gain of the window (its mean is 1/2)
    assert np.allclose(O.hann_fd(np.ones(8))[1:-1], 0.0)
    assert np.sum(O.hann_td(64)) == pytest.approx(32.0, rel=1e-14)


@pytest.mark.parametrize("modes", [[(2, 2, 0)], [(2, 2, 0), (3, 3, 2), (2, 1, -3), (3, 1, 1)]])
def test_windowed_spa_matches_windowed_dft(oracle, modes):
    base = synth.small_config(0)
    idx = [int(np.nonzero((base.l == l) & (base.m == m) & (base.n == n))[0][0]) for (l, m, n) in modes]
    w = base.with_modes(idx)
    fk, Hp, Hc = oracle.td_dft(w, dt=10.0)
    _, Wp, Wc = oracle.td_dft(w, dt=10.0, window="hann")
    hp, hc = oracle.sum_modes(w, freqs=fk)
    wp, wc = oracle.hann_fd(hp), oracle.hann_fd(hc)
    band = (fk > 5e-5) & (fk < 6e-3)
    # away from every voice's end and turnover frequencies
    edges = []
    for j in range(w.n_modes):
        F = (w.m[j] * w.omega_phi + w.n[j] * w.omega_r) / (2 * np.pi)
        dF = np.diff(F)
        edges += [F[0], F[-1]] + list(F[1:-1][np.sign(dF[1:]) != np.sign(dF[:-1])])
    edges = np.abs(np.array(edges))
    clean = band & (np.min(np.abs(fk[:, None] - edges[None, :]), axis=1) > 6e-5)
    assert np.count_nonzero(clean & (np.abs(wp) > 0)) > 300
    for a, b in ((wp, Wp), (wc, Wc)):
        assert _match(a[clean], b[clean]) > 0.999
    # whole band, edges included: the window reduces the FD/TD disagreement
    for (a, b), (aw, bw) in (((hp, Hp), (wp, Wp)), ((hc, Hc), (wc, Wc))):
        assert 1 - _match(aw[band], bw[band]) < 0.5 * (1 - _match(a[band], b[band]))
