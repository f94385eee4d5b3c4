"""Pins of the oracle's Whittle log-likelihood gradient (Eq. 13-14).

L is piecewise smooth: a bin changes voice, branch or segment when a knot or
turnover frequency crosses it.  The gradient is the derivative with the bin
assignment fixed, so finite differences use a "safe" grid that keeps every
bin away from all knot, end and turnover frequencies by more than the step
can move them.  Two identities are exact: h is linear in the amplitude knots
(Euler: sum_k a_k dL/da_k = sum_alpha <d - h|h>_alpha), and a constant
offset delta of Phi_phi multiplies voice V by e^{-i m_V delta} (for a mode of
one frequency sign sigma, h_j -> e^{-i m_j sigma_j delta} h_j)."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import synth


def _setup(seed=0, n_modes=None, n_bins=3000):
    w = synth.small_config(seed, n_bins=8192)
    if n_modes:
        w = w.with_modes(np.arange(n_modes))
    return w


def _boundaries(w):
    out = []
    for j in range(w.n_modes):
        F = (w.m[j] * w.omega_phi + w.n[j] * w.omega_r) / (2 * np.pi)
        out += list(F)
        dF = np.diff(F)
        # turnover neighbourhoods: whole segments around a sign change of dF
        for k in np.nonzero(np.sign(dF[1:]) != np.sign(dF[:-1]))[0]:
            out += list(np.linspace(F[k], F[k + 2], 50))
    b = np.abs(np.array(out))
    return np.sort(b)


def safe_grid(w, n_bins=3000, margin=2e-6):
    f = np.linspace(1e-4, 6e-3, 40000)
    b = _boundaries(w)
    idx = np.searchsorted(b, f)
    lo = np.abs(f - b[np.clip(idx - 1, 0, len(b) - 1)])
    hi = np.abs(b[np.clip(idx, 0, len(b) - 1)] - f)
    ok = np.minimum(lo, hi) > margin * f
    f = f[ok]
    return f[:: max(1, len(f) // n_bins)]


def _data(oracle, w, seed=1):
    hp, hc = oracle.sum_modes(w)
    rng = np.random.default_rng(seed)
    s = np.abs(hp).max()
    # data = a rotated, rescaled copy plus noise, so that d - h is O(h)
    return (hp * 0.97 * np.exp(0.05j) + 0.02 * s * rng.normal(size=hp.shape),
            hc * 1.02 * np.exp(-0.04j) + 0.02 * s * rng.normal(size=hc.shape))


def _L(oracle, w, d, S, df):
    return oracle.loglike_grad(w, d[0], d[1], S, df, grad=False)


def test_loglike_definition(oracle):
    w = _setup()
    w = w.with_freqs(safe_grid(w))
    d = _data(oracle, w)
    S = synth.psd(w.freqs) / 1e-40
    df = 1e-7
    hp, hc = oracle.sum_modes(w)
    ref = -0.5 * (oracle.inner(d[0] - hp, d[0] - hp, S, df) + oracle.inner(d[1] - hc, d[1] - hc, S, df))
    assert abs(_L(oracle, w, d, S, df) - ref) <= 1e-12 * abs(ref)


def test_euler_identity_amplitudes(oracle):
    w = _setup()
    w = w.with_freqs(safe_grid(w))
    d = _data(oracle, w)
    S = synth.psd(w.freqs) / 1e-40
    df = 1e-7
    L, g = oracle.loglike_grad(w, d[0], d[1], S, df)
    lhs = np.sum(w.amp.real * g["amp"].real + w.amp.imag * g["amp"].imag)
    hp, hc = oracle.sum_modes(w)
    rhs = oracle.inner(d[0] - hp, hp, S, df) + oracle.inner(d[1] - hc, hc, S, df)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


@pytest.mark.parametrize("which", ["phi_phi", "phi_r"])
def test_phase_offset_identity(oracle, which):
    base = _setup()
    keep = [j for j in range(base.n_modes)
            if np.all(np.sign(base.m[j] * base.omega_phi + base.n[j] * base.omega_r) ==
                      np.sign(base.m[j] * base.omega_phi[0] + base.n[j] * base.omega_r[0]))]
    w = base.with_modes(keep)
    w = w.with_freqs(safe_grid(w))
    d = _data(oracle, w)
    S = synth.psd(w.freqs) / 1e-40
    df = 1e-7
    L, g = oracle.loglike_grad(w, d[0], d[1], S, df)
    hp, hc = oracle.sum_modes(w)
    tp, tc = np.zeros_like(hp), np.zeros_like(hc)
    for j in range(w.n_modes):
        wj = w.with_modes([j])
        sig = np.sign(wj.m[0] * wj.omega_phi[0] + wj.n[0] * wj.omega_r[0])
        k = int(wj.m[0]) if which == "phi_phi" else int(wj.n[0])
        a, b = oracle.sum_modes(wj)
        tp += -1j * k * sig * a
        tc += -1j * k * sig * b
    rhs = oracle.inner(d[0] - hp, tp, S, df) + oracle.inner(d[1] - hc, tc, S, df)
    assert abs(np.sum(g[which]) - rhs) <= 1e-9 * np.sqrt(np.sum(g[which] ** 2)) * np.sqrt(len(g[which]))


@pytest.mark.parametrize("which,step", [("phi_phi", 3e-5), ("phi_r", 3e-5), ("omega_phi", 1e-8),
                                        ("omega_r", 1e-8), ("amp", 1e-4)])
def test_central_differences(oracle, which, step):
    """directional derivatives along 3 seeded random knot directions.  Steps:
    absolute for phases (rad), relative to the series' largest value otherwise.
    A scan of steps shows the plateau: below ~1e-5 rad the FP64 rounding of the
    phase spline's coefficients (~1e-11 rad on ~1e5 rad phases) dominates the
    difference; above ~1e-7 relative on Omega the O(h^2) term does.  The
    Richardson value (4 D(h/2) - D(h))/3 and D(h/2) must agree <= 1e-6."""
    w = _setup(n_modes=20)
    w = w.with_freqs(safe_grid(w, margin=5e-6))
    d = _data(oracle, w)
    S = synth.psd(w.freqs) / 1e-40
    df = 1e-7
    L0, g = oracle.loglike_grad(w, d[0], d[1], S, df)
    rng = np.random.default_rng(11)
    for trial in range(3):
        if which == "amp":
            v = rng.normal(size=w.amp.shape) + 1j * rng.normal(size=w.amp.shape)
            scale = step * np.abs(w.amp).max()
            gv = np.sum(g["amp"].real * v.real + g["amp"].imag * v.imag)
        else:
            v = rng.normal(size=w.K)
            base = getattr(w, which)
            scale = step if which.startswith("phi") else step * np.abs(base).max()
            gv = np.dot(g[which], v)
        fd = []
        for h in (scale, scale / 2):
            Ls = []
            for sgn in (1, -1):
                wp = w.with_freqs(w.freqs)
                if which == "amp":
                    wp.amp = w.amp + sgn * h * v
                else:
                    setattr(wp, which, getattr(w, which) + sgn * h * v)
                Ls.append(_L(oracle, wp, d, S, df))
            fd.append((Ls[0] - Ls[1]) / (2 * h))
        rich = (4 * fd[1] - fd[0]) / 3
        assert abs(rich - gv) <= 1e-6 * abs(gv), (which, fd, gv)
        assert abs(fd[1] - gv) <= 1e-6 * abs(gv), (which, fd, gv)
