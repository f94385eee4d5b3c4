"""Seeded synthetic EMRI-shaped inputs for the frequency-domain SPA mode sum.

This module only manufactures inputs.  It holds none of the method's arithmetic
(no spline fit, no root finding, no stationary-phase evaluation); both the CUDA
path and the CPU oracle consume what it returns.

The paper's own inputs (an adiabatic Schwarzschild trajectory from flux grids,
Teukolsky amplitudes, Sec. 2.1) are not available, so the recipes below stand in
for them with analytic shapes that share their structure: a chirping azimuthal
frequency, a radial frequency with an interior maximum (which gives radial
harmonics a df/dt = 0 turning point, Sec. 2.2), phases obtained by integrating
the frequencies, smooth complex amplitudes per (l, m, n) mode, and frequency
grids with df = 1/T (Eq. 13) or sparse log spacing (Sec. 3.3).

Units: seconds, rad, rad/s, Hz.  Every random draw comes from
``numpy.random.default_rng(seed)`` in the order documented in each function.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
import math
import os

import numpy as np

YEAR_S = 365.25 * 86400.0  # Julian year
OMEGA0 = 2.0 * math.pi * 2e-4  # rad/s, initial azimuthal frequency


@dataclass
class Waveform:
    """One waveform's inputs, in the layout the C-ABI takes.

    t:          [K] knot times (s), strictly increasing
    phi_phi, phi_r:      [K] azimuthal / radial phase knots (rad)
    omega_phi, omega_r:  [K] azimuthal / radial angular frequency knots (rad/s)
    l, m, n:    [N_m] int32 mode numbers
    amp:        [N_m, K] complex128 amplitude knot values (mode-major)
    theta, phi: source-frame viewing angles (rad)
    prefactor:  real amplitude prefactor (mu/d_L in Eq. 1)
    freqs:      [N_f] ascending output frequencies (Hz), all > 0
    """

    t: np.ndarray
    phi_phi: np.ndarray
    phi_r: np.ndarray
    omega_phi: np.ndarray
    omega_r: np.ndarray
    l: np.ndarray
    m: np.ndarray
    n: np.ndarray
    amp: np.ndarray
    theta: float
    phi: float
    prefactor: float
    freqs: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.t.shape[0])

    @property
    def n_modes(self) -> int:
        return int(self.l.shape[0])

    @property
    def n_freqs(self) -> int:
        return int(self.freqs.shape[0])

    def with_freqs(self, freqs) -> "Waveform":
        w = Waveform(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        w.freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        w.meta = dict(self.meta)
        return w

    def with_modes(self, idx) -> "Waveform":
        idx = np.asarray(idx)
        w = Waveform(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        w.l, w.m, w.n = self.l[idx].copy(), self.m[idx].copy(), self.n[idx].copy()
        w.amp = np.ascontiguousarray(self.amp[idx])
        w.meta = dict(self.meta)
        return w


def trajectory(T: float, K: int, phi0=(0.0, 0.0), n_fine: int = 1_000_000):
    """Synthetic inspiral on K uniform knots over [0, T].

    Omega_phi(t) = OMEGA0 (1 - t/tc)^(-3/8), tc = 1.2 T;
    p(t) = 12 - 5 t/T; Omega_r = Omega_phi sqrt(1 - 6/p)  (max near t/T = 0.8).
    Phases: trapezoid rule on a fine grid that contains every knot
    (about n_fine points), sampled at the knots, offset by phi0.
    """
    tc = 1.2 * T
    per = max(1, int(math.ceil(n_fine / (K - 1))))
    nf = (K - 1) * per + 1
    tf = np.linspace(0.0, T, nf)

    def om_phi(t):
        return OMEGA0 * (1.0 - t / tc) ** (-3.0 / 8.0)

    def om_r(t):
        p = 12.0 - 5.0 * t / T
        return om_phi(t) * np.sqrt(1.0 - 6.0 / p)

    def cumtrap(y):
        out = np.zeros_like(y)
        out[1:] = np.cumsum(0.5 * (y[1:] + y[:-1]) * np.diff(tf))
        return out

    Pphi = cumtrap(om_phi(tf)) + phi0[0]
    Pr = cumtrap(om_r(tf)) + phi0[1]
    idx = np.arange(K) * per
    t = tf[idx].copy()
    return t, Pphi[idx].copy(), Pr[idx].copy(), om_phi(t), om_r(t)


def mode_pool(lmax: int, nmax: int):
    """All (l, m, n) with l = 2..lmax, m = 1..l, n = -nmax..nmax, in that nesting order."""
    ls, ms, ns = [], [], []
    for l in range(2, lmax + 1):
        for m in range(1, l + 1):
            for n in range(-nmax, nmax + 1):
                ls.append(l)
                ms.append(m)
                ns.append(n)
    return (np.array(ls, np.int32), np.array(ms, np.int32), np.array(ns, np.int32))


def amplitudes(rng, t, l, m, n, scale):
    """Smooth complex amplitude knots A(t_k) = s e^{i phi0} (1 + 0.2 u(t_k)).

    Draw order (vectorised over modes): s_u ~ U(0.5, 1) [N], phi0 ~ U(0, 2pi) [N],
    then c ~ N(0, 1) [N, 4, 3]; u(t) = sum_j (c0j cos + c1j sin)(2 pi j t/T)/3
    + i sum_j (c2j cos + c3j sin)(2 pi j t/T)/3, j = 1..3.  s = s_u * scale.
    """
    N = l.shape[0]
    T = t[-1] - t[0]
    su = rng.uniform(0.5, 1.0, N)
    ph = rng.uniform(0.0, 2.0 * math.pi, N)
    c = rng.normal(size=(N, 4, 3))
    j = np.arange(1, 4)
    arg = 2.0 * math.pi * np.outer((t - t[0]) / T, j)  # [K, 3]
    cs, sn = np.cos(arg), np.sin(arg)
    ure = (c[:, 0, None, :] * cs[None] + c[:, 1, None, :] * sn[None]).sum(-1) / 3.0
    uim = (c[:, 2, None, :] * cs[None] + c[:, 3, None, :] * sn[None]).sum(-1) / 3.0
    s = su * scale
    A = (s * np.exp(1j * ph))[:, None] * (1.0 + 0.2 * (ure + 1j * uim))
    return np.ascontiguousarray(A.astype(np.complex128))


def small_config(seed: int = 0, n_bins: int = 2 ** 15) -> Waveform:
    """Plain FP64 single waveform: T = 0.25 yr, K = 100, 55 modes
    (l = 2..3, m = 1..l, n = -5..5), theta = 0.7, phi = 1.1, n_bins uniform
    bins over [1e-4, 2e-2] Hz.  Phases start at 0.  Amplitude scale exp(-|n|/2)."""
    T = 0.25 * YEAR_S
    K = 100
    t, pp, pr, op, orr = trajectory(T, K)
    l, m, n = mode_pool(3, 5)
    rng = np.random.default_rng(seed)
    A = amplitudes(rng, t, l, m, n, np.exp(-np.abs(n) / 2.0))
    f = np.linspace(1e-4, 2e-2, n_bins)
    return Waveform(t, pp, pr, op, orr, l, m, n, A, 0.7, 1.1, 1.0, f,
                    meta={"name": "T=0.25yr K=100 modes=55 bins=%d" % n_bins, "T": T, "seed": seed})


def chirp_config(K: int = 100, n_bins: int = 2 ** 15):
    """One power-law chirp voice with a closed-form SPA: a single (l=2, m=1, n=0)
    mode, A = 1, whose azimuthal phase/frequency knots are the analytic
    Phi(t) = (16 pi/5) F0 tc [1 - (1 - t/tc)^(5/8)], F(t) = F0 (1 - t/tc)^(-3/8)
    (F0 = OMEGA0/2pi, tc = 1.2 T), T = 0.25 yr.  The radial series is zero.
    Returns (Waveform, dict of the closed-form parameters)."""
    T = 0.25 * YEAR_S
    tc = 1.2 * T
    F0 = OMEGA0 / (2.0 * math.pi)
    t = np.linspace(0.0, T, K)
    x = 1.0 - t / tc
    Phi = (16.0 * math.pi / 5.0) * F0 * tc * (1.0 - x ** 0.625)
    Om = 2.0 * math.pi * F0 * x ** (-0.375)
    z = np.zeros(K)
    A = np.ones((1, K), np.complex128)
    f = np.linspace(1e-4, 2e-2, n_bins)
    w = Waveform(t, Phi, z.copy(), Om, z.copy(), np.array([2], np.int32), np.array([1], np.int32),
                 np.array([0], np.int32), A, 0.7, 1.1, 1.0, f,
                 meta={"name": "power-law chirp K=%d" % K, "T": T})
    return w, {"F0": F0, "tc": tc, "T": T}


def paper_config(seed: int, n_modes: int = 2000, T_years: float = 2.0, K: int = 200,
                 grid: str = "dense", n_sparse: int = 10_000, f_max: float = 0.05,
                 n_bins: int | None = None) -> Waveform:
    """Paper-shaped single waveform (M = 1e6, mu = 10 scale): T = 2 yr, K = 200,
    mode pool l = 2..10, m = 1..l, n = -30..30 (3294 modes) of which the n_modes
    with the largest mean |A|^2 are kept (power-based selection, Sec. 2.1).

    Draw order: e0 ~ U(0.1, 0.7); (Phi_phi0, Phi_r0) ~ U(0, 2pi)^2; then the
    amplitude draws of ``amplitudes`` over the whole pool.  Amplitude scale
    exp(-|n|/(1 + 10 e0)) exp(-(l - 2)/2).
    grid: "dense" -> f_i = i/T, i = 1..floor(f_max T) (df = 1/T, Eq. 13);
          "sparse" -> n_sparse log-spaced bins over [1/T, f_max];
          "uniform" -> n_bins uniform bins over [1/T, f_max].
    """
    T = T_years * YEAR_S
    rng = np.random.default_rng(seed)
    e0 = rng.uniform(0.1, 0.7)
    phi0 = rng.uniform(0.0, 2.0 * math.pi, 2)
    t, pp, pr, op, orr = trajectory(T, K, phi0=(phi0[0], phi0[1]))
    l, m, n = mode_pool(10, 30)
    scale = np.exp(-np.abs(n) / (1.0 + 10.0 * e0)) * np.exp(-(l - 2) / 2.0)
    A = amplitudes(rng, t, l, m, n, scale)
    power = (np.abs(A) ** 2).mean(axis=1)
    keep = np.sort(np.argsort(-power, kind="stable")[:n_modes])
    f = make_grid(T, grid, n_sparse=n_sparse, f_max=f_max, n_bins=n_bins)
    w = Waveform(t, pp, pr, op, orr, l[keep].copy(), m[keep].copy(), n[keep].copy(),
                 np.ascontiguousarray(A[keep]), 0.7, 1.1, 1.0, f,
                 meta={"name": "T=%gyr K=%d modes=%d bins=%d %s" % (T_years, K, n_modes, f.shape[0], grid),
                       "T": T, "seed": seed, "e0": e0})
    return w


def make_grid(T, grid, n_sparse=10_000, f_max=0.05, n_bins=None):
    if grid == "dense":
        nb = int(math.floor(f_max * T))
        return np.arange(1, nb + 1, dtype=np.float64) / T
    if grid == "sparse":
        return np.geomspace(1.0 / T, f_max, n_sparse)
    if grid == "uniform":
        return np.linspace(1.0 / T, f_max, int(n_bins))
    raise ValueError(grid)


def batch_config(n_waveforms: int = 256, seed0: int = 100, max_bins: float = 6e6,
                 min_bins: float = 1e4, mode_range=(50, 3000), T_range=(0.5, 4.0), K: int = 200):
    """Batched workload: waveform i uses seed seed0 + i.  Per waveform, draw order:
    N_m ~ U{mode_range}, T ~ U(T_range) yr, N_f = round(exp(U(ln min_bins, ln max_bins))),
    grid kind ~ Bernoulli(1/2) (uniform or log-spaced over [1/T, 0.05]);
    then ``paper_config``'s draws with its own generator seeded seed0 + i.
    Waveforms are made on a thread pool; each uses only its own generators, so the
    result does not depend on the pool."""
    def one(i):
        r = np.random.default_rng(seed0 + i)
        nm = int(r.integers(mode_range[0], mode_range[1] + 1))
        Ty = float(r.uniform(*T_range))
        nf = int(round(math.exp(r.uniform(math.log(min_bins), math.log(max_bins)))))
        kind = "uniform" if r.uniform() < 0.5 else "sparse"
        return paper_config(seed0 + i, n_modes=nm, T_years=Ty, K=K, grid=kind, n_sparse=nf, n_bins=nf)
    return _pool_map(one, range(n_waveforms))


def paper_configs(seeds, **kw):
    """``paper_config(s, **kw)`` for every seed, made on a thread pool (numpy releases
    the GIL in its array loops); identical to the serial list."""
    return _pool_map(lambda s: paper_config(s, **kw), seeds)


def _pool_map(fn, items):
    items = list(items)
    if len(items) <= 1:
        return [fn(i) for i in items]
    with ThreadPoolExecutor(max_workers=min(len(items), os.cpu_count() or 1, 16)) as ex:
        return list(ex.map(fn, items))


def psd(f):
    """Analytic one-sided noise PSD S(f) = 1e-40 ((1e-3/f)^4 + 1 + (f/2e-2)^2)."""
    f = np.asarray(f, dtype=np.float64)
    return 1e-40 * ((1e-3 / f) ** 4 + 1.0 + (f / 2e-2) ** 2)


def noise(rng, freqs, df):
    """Complex Gaussian noise per bin with Re, Im iid N(0, S/(4 df)), so that
    E<n|n> with the Eq. 13 inner product equals 2 per bin (Eq. 15 with N = 2 N_f)."""
    sig = np.sqrt(psd(freqs) / (4.0 * df))
    return sig * (rng.normal(size=freqs.shape) + 1j * rng.normal(size=freqs.shape))


def likelihood_config(seed: int = 3, n_modes: int = 500, K: int = 150, T_years: float = 1.0,
                      n_bins: int | None = None) -> Waveform:
    """Whittle-likelihood workload: T = 1 yr, K = 150, 500 modes, df = 1/T grid
    (1,577,880 bins) unless n_bins selects the first n_bins of it."""
    w = paper_config(seed, n_modes=n_modes, T_years=T_years, K=K, grid="dense")
    if n_bins is not None:
        w = w.with_freqs(w.freqs[:n_bins])
    return w


def concat(wfs):
    """CSR-concatenate waveforms for a batched call: returns dict of arrays
    (knot_off, mode_off, freq_off as int64 [n+1]; concatenated series)."""
    ko = np.zeros(len(wfs) + 1, np.int64)
    mo = np.zeros(len(wfs) + 1, np.int64)
    fo = np.zeros(len(wfs) + 1, np.int64)
    for i, w in enumerate(wfs):
        ko[i + 1] = ko[i] + w.K
        mo[i + 1] = mo[i] + w.n_modes
        fo[i + 1] = fo[i] + w.n_freqs
    cat = lambda name: np.ascontiguousarray(np.concatenate([getattr(w, name) for w in wfs]))
    amp = np.concatenate([w.amp.reshape(-1) for w in wfs])
    return dict(knot_off=ko, mode_off=mo, freq_off=fo, t=cat("t"), phi_phi=cat("phi_phi"),
                phi_r=cat("phi_r"), omega_phi=cat("omega_phi"), omega_r=cat("omega_r"),
                l=cat("l"), m=cat("m"), n=cat("n"), amp=np.ascontiguousarray(amp),
                theta=np.array([w.theta for w in wfs]), phi=np.array([w.phi for w in wfs]),
                prefactor=np.array([w.prefactor for w in wfs]), freqs=cat("freqs"))
