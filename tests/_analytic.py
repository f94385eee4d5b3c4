"""Analytic single-voice inputs whose SPA sum has a closed form (shared by
the oracle pins and the GPU parity tests; inputs only)."""
import math

import numpy as np

from paper_2307_12585_gb300.synth import Waveform


def single_voice(t, phase, omega, amp=1.0 + 0.0j, freqs=None, theta=0.7, phi=1.1, l=2, m=1, n=0):
    """One (l, m, n) mode with Phi_phi = phase(t)/m and Omega_phi = omega(t)/m
    (radial series zero), so the voice phase is phase(t) and its frequency
    omega(t)/2pi.  Amplitude constant."""
    K = t.shape[0]
    z = np.zeros(K)
    A = np.full((1, K), amp, np.complex128)
    return Waveform(t.astype(np.float64), phase(t) / m, z.copy(), omega(t) / m, z.copy(),
                    np.array([l], np.int32), np.array([m], np.int32), np.array([n], np.int32),
                    A, theta, phi, 1.0, np.asarray(freqs, np.float64))


def linear_chirp(K=37, seed=0, nb=4000):
    """F(t) = f0 + fd t on non-uniform knots over [0, T]; Phi = 2 pi (f0 t + fd t^2/2) + P0."""
    rng = np.random.default_rng(seed)
    T, f0, fd, P0 = 1e6, 1e-3, 1e-9, 0.3
    t = np.concatenate([[0.0], np.sort(rng.uniform(0, T, K - 2)), [T]])
    freqs = np.linspace(0.8e-3, 2.2e-3, nb)
    w = single_voice(t, lambda x: 2 * math.pi * (f0 * x + 0.5 * fd * x * x) + P0,
                     lambda x: 2 * math.pi * (f0 + fd * x), amp=0.8 - 0.3j, freqs=freqs)
    return w, dict(T=T, f0=f0, fd=fd, P0=P0)


def knot_rounding(w, phase_mp, series="phi_phi", deriv=0):
    """The FP64 phase knots differ from the exact phase by their rounding
    error d_k; the not-a-knot spline is linear, so the spline of the knots is
    the exact (low-degree) phase plus the spline of d_k.  Returns that
    correction as a callable (scipy spline of d_k; d_k ~ 1e-12 rad, so FP64
    is ample for it)."""
    import mpmath as mp
    from scipy.interpolate import CubicSpline
    mp.mp.dps = 40
    vals = getattr(w, series)
    d = np.array([float(mp.mpf(float(vals[k])) * int(w.m[0]) - phase_mp(mp.mpf(float(w.t[k]))))
                  for k in range(w.K)])
    cs = CubicSpline(w.t, d, bc_type="not-a-knot")
    if deriv:
        dcs = cs.derivative()
        return (lambda x: float(cs(float(x)))), (lambda x: float(dcs(float(x))))
    return lambda x: float(cs(float(x)))


def linear_chirp_expected(w, p, f):
    import mpmath as mp
    mp.mp.dps = 40
    f0, fd, P0 = mp.mpf(p["f0"]), mp.mpf(p["fd"]), mp.mpf(p["P0"])
    corr = knot_rounding(w, lambda x: 2 * mp.pi * (f0 * x + fd * x * x / 2) + P0)
    out = np.zeros(f.shape, np.complex128)
    for i, fi in enumerate(f):
        if not (p["f0"] <= fi < p["f0"] + p["fd"] * p["T"]):
            continue
        x = mp.mpf(fi) - f0
        tj = x / fd
        psi = mp.pi * x * x / fd - P0 - mp.pi / 4 - corr(tj)
        out[i] = complex(mp.cos(psi), mp.sin(psi)) / math.sqrt(p["fd"])
    return out


def quadratic_voice(K=41, seed=1, nb=5000, uniform=False):
    """F(t) = Fs - kappa (t - ts)^2 / 2 with its maximum inside [0, T];
    Phi = 2 pi [Fs (t - ts) - kappa (t - ts)^3 / 6] + Ps.  Knots random (seeded), or
    uniform (K = 40 puts the maximum mid-segment, at 21.45 segment widths)."""
    rng = np.random.default_rng(seed)
    T, ts, Fs, Ps = 1e6, 0.55e6, 2e-3, -1.2
    kappa = 1e-3 / (0.55e6) ** 2
    if uniform:
        t = np.linspace(0.0, T, K)
    else:
        t = np.concatenate([[0.0], np.sort(rng.uniform(0, T, K - 2)), [T]])
    freqs = np.linspace(1.3e-3, 2.1e-3, nb)
    w = single_voice(t, lambda x: 2 * math.pi * (Fs * (x - ts) - kappa * (x - ts) ** 3 / 6) + Ps,
                     lambda x: 2 * math.pi * (Fs - 0.5 * kappa * (x - ts) ** 2), amp=0.5 + 0.9j, freqs=freqs)
    return w, dict(T=T, ts=ts, Fs=Fs, Ps=Ps, kappa=kappa)


def quadratic_voice_expected(w, p, f):
    import mpmath as mp
    mp.mp.dps = 40
    out = np.zeros(f.shape, np.complex128)
    Fs, ts, kap, T, Ps = (mp.mpf(p[k]) for k in ("Fs", "ts", "kappa", "T", "Ps"))
    corr = knot_rounding(w, lambda x: 2 * mp.pi * (Fs * (x - ts) - kap * (x - ts) ** 3 / 6) + Ps)
    # Omega knots: their rounding moves F by sF(t) = spline(dOmega)/2pi
    sO, dsO = knot_rounding(w, lambda x: 2 * mp.pi * (Fs - kap * (x - ts) ** 2 / 2), series="omega_phi", deriv=1)
    for i, fi in enumerate(f):
        g = mp.mpf(fi)
        if g >= Fs:
            continue
        d = mp.sqrt(2 * (Fs - g) / kap)
        acc = mp.mpc(0)
        for sgn in (-1, 1):
            tj = ts + sgn * d
            if tj < 0 or tj >= T:
                continue
            # one Newton step onto the root of F_exact + sF = g
            tj = tj - mp.mpf(sO(tj)) / (2 * mp.pi) / (-kap * (tj - ts))
            Phi = 2 * mp.pi * (Fs * (tj - ts) - kap * (tj - ts) ** 3 / 6) + Ps
            Fd = -kap * (tj - ts) + mp.mpf(dsO(tj)) / (2 * mp.pi)
            psi = 2 * mp.pi * g * tj - Phi - (mp.pi / 4 if Fd > 0 else -mp.pi / 4) - corr(tj)
            acc += mp.expj(psi) / mp.sqrt(abs(Fd))
        out[i] = complex(acc)
    return out


def power_law_expected(p, f):
    """Closed-form SPA of F = F0 (1 - t/tc)^(-3/8) on [0, T]."""
    import mpmath as mp
    mp.mp.dps = 40
    F0, tc, T = mp.mpf(p["F0"]), mp.mpf(p["tc"]), mp.mpf(p["T"])
    out = np.zeros(f.shape, np.complex128)
    for i, fi in enumerate(f):
        g = mp.mpf(fi)
        tj = tc * (1 - (g / F0) ** (mp.mpf(-8) / 3))
        if tj < 0 or tj >= T:
            continue
        x = 1 - tj / tc
        Phi = mp.mpf(16) * mp.pi / 5 * F0 * tc * (1 - x ** (mp.mpf(5) / 8))
        Fd = mp.mpf(3) / 8 * F0 / tc * x ** (mp.mpf(-11) / 8)
        psi = 2 * mp.pi * g * tj - Phi - mp.pi / 4
        out[i] = complex(mp.expj(psi) / mp.sqrt(Fd))
    return out
