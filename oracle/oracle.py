"""Python side of the CPU oracle (test infrastructure only).

Builds ``oracle.c`` with gcc (no implicit FMA contraction, OpenMP) into
``oracle/_build/liboracle.so`` and exposes it through ctypes.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use this
module; the CUDA library never imports it.

Also holds the checking tools that are defined by the paper's data-analysis
section: the noise-weighted inner product (Eq. 13), mismatch (Eq. 12), and a
brute-force time-domain synthesis + DFT used to pin the SPA sum on tiny inputs
(Sec. 2.3: FD vs DFT of the TD waveform).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = os.path.join(HERE, "oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.oracle_spline_coef.argtypes = [C.c_int, dp, dp, dp]
        L.oracle_spline_coef.restype = C.c_int
        L.oracle_swsh.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, dp]
        L.oracle_swsh.restype = None
        L.oracle_sum_modes.argtypes = [C.c_int, dp, dp, dp, dp, dp, C.c_int, ip, ip, ip, dp,
                                       C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                       C.c_longlong, dp, dp, dp, C.POINTER(C.c_longlong), C.c_int]
        L.oracle_ext_factor.argtypes = [C.c_longlong, dp, dp, dp]
        L.oracle_ext_factor.restype = None
        L.oracle_select_modes.argtypes = [C.c_int, C.c_int, dp, C.c_double, ip]
        L.oracle_select_modes.restype = C.c_longlong
        L.oracle_sum_modes.restype = C.c_int
        L.oracle_loglike_grad.argtypes = [C.c_int, dp, dp, dp, dp, dp, C.c_int, ip, ip, ip, dp,
                                          C.c_double, C.c_double, C.c_double, C.c_int,
                                          C.c_longlong, dp, dp, dp, dp, C.c_double, dp, dp, dp, dp, dp, dp, C.c_int]
        L.oracle_loglike_grad.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def spline_coef(t, y):
    """Not-a-knot cubic coefficients [K-1, 4] = (a, b, c, d) in tau = t - t_k."""
    t, tp = _d(t)
    y, yp = _d(y)
    out = np.zeros((t.shape[0] - 1, 4))
    o, op = _d(out)
    rc = lib().oracle_spline_coef(t.shape[0], tp, yp, op)
    if rc:
        raise ValueError("oracle_spline_coef failed: %d" % rc)
    return o


def swsh(s, l, m, theta, phi):
    out = np.zeros(2)
    o, op = _d(out)
    lib().oracle_swsh(s, l, m, theta, phi, op)
    return complex(o[0], o[1])


def default_threads():
    return max(1, min(os.cpu_count() or 1, 64))


SPA_FORMS = {"standard": 0, "extended": 1}


def ext_factor(Fd, Fdd):
    """Extended-SPA time integral G(Fdot, Fddot) of one root (Eq. 10, sign reading
    of the oracle source), complex128, elementwise."""
    Fd = np.atleast_1d(np.asarray(Fd, np.float64))
    Fdd = np.broadcast_to(np.asarray(Fdd, np.float64), Fd.shape)
    a, ap = _d(Fd.ravel())
    b, bp = _d(np.ascontiguousarray(Fdd).ravel())
    out = np.zeros(2 * a.shape[0])
    o, op = _d(out)
    lib().oracle_ext_factor(a.shape[0], ap, bp, op)
    return o.view(np.complex128).reshape(Fd.shape)


def sum_modes(w, freqs=None, conj_partners=True, nthreads=None, return_stats=False, spa="standard"):
    """SPA sum of one synthetic waveform ``w`` (see synth.Waveform) on ``freqs``
    (default: w.freqs); ``spa`` is "standard" (Fresnel integral per root) or
    "extended" (Eq. 10 per root).  Returns (h_plus, h_cross) complex128 arrays."""
    f = w.freqs if freqs is None else freqs
    f, fp = _d(f)
    t, tp = _d(w.t)
    a1, p1 = _d(w.phi_phi)
    a2, p2 = _d(w.phi_r)
    a3, p3 = _d(w.omega_phi)
    a4, p4 = _d(w.omega_r)
    l, lp = _i(w.l)
    m, mp = _i(w.m)
    n, np_ = _i(w.n)
    amp = np.ascontiguousarray(np.asarray(w.amp, np.complex128)).view(np.float64)
    amp, ap = _d(amp)
    hp = np.zeros(2 * f.shape[0])
    hc = np.zeros(2 * f.shape[0])
    hpp, hpptr = _d(hp)
    hcc, hccptr = _d(hc)
    st = (C.c_longlong * 4)()
    rc = lib().oracle_sum_modes(t.shape[0], tp, p1, p2, p3, p4, l.shape[0], lp, mp, np_, ap,
                                float(w.theta), float(w.phi), float(w.prefactor), int(conj_partners),
                                SPA_FORMS[spa], f.shape[0], fp, hpptr, hccptr, st,
                                int(nthreads or default_threads()))
    if rc:
        raise ValueError("oracle_sum_modes rejected the input: %d" % rc)
    hpc = hpp.view(np.complex128)
    hcc_ = hcc.view(np.complex128)
    if return_stats:
        return hpc, hcc_, {"contributions": int(st[0]), "zero_fdot": int(st[1]), "pieces": int(st[2])}
    return hpc, hcc_


def loglike_grad(w, dplus, dcross, psd, df, conj_partners=True, nthreads=None, grad=True):
    """Whittle log-likelihood L = -1/2 sum_alpha <d - h|d - h>_alpha (Eq. 13-14) of
    the SPA waveform of ``w`` on w.freqs, and (grad=True) its gradient with respect
    to every knot value: dict with phi_phi, phi_r, omega_phi, omega_r [K] and
    amp [N_m, K] complex (d/dRe + 1j d/dIm)."""
    f, fp = _d(w.freqs)
    t, tp = _d(w.t)
    a1, p1 = _d(w.phi_phi)
    a2, p2 = _d(w.phi_r)
    a3, p3 = _d(w.omega_phi)
    a4, p4 = _d(w.omega_r)
    l, lp = _i(w.l)
    m, mp = _i(w.m)
    n, np_ = _i(w.n)
    amp, ap = _d(np.ascontiguousarray(np.asarray(w.amp, np.complex128)).view(np.float64))
    dp_, dpp = _d(np.ascontiguousarray(np.asarray(dplus, np.complex128)).view(np.float64))
    dc_, dcp = _d(np.ascontiguousarray(np.asarray(dcross, np.complex128)).view(np.float64))
    S, Sp = _d(psd)
    K, nm = t.shape[0], l.shape[0]
    L = np.zeros(1)
    Lp = L.ctypes.data_as(C.POINTER(C.c_double))
    outs = [np.zeros(K) for _ in range(4)] + [np.zeros(2 * nm * K)]
    ptrs = [o.ctypes.data_as(C.POINTER(C.c_double)) if grad else None for o in outs]
    rc = lib().oracle_loglike_grad(K, tp, p1, p2, p3, p4, nm, lp, mp, np_, ap, float(w.theta), float(w.phi),
                                   float(w.prefactor), int(conj_partners), f.shape[0], fp, dpp, dcp, Sp,
                                   float(df), Lp, *ptrs, int(nthreads or default_threads()))
    if rc:
        raise ValueError("oracle_loglike_grad rejected the input: %d" % rc)
    if not grad:
        return float(L[0])
    g = {"phi_phi": outs[0], "phi_r": outs[1], "omega_phi": outs[2], "omega_r": outs[3],
         "amp": outs[4].view(np.complex128).reshape(nm, K)}
    return float(L[0]), g


# ---------------------------------------------------------------------------
# data-analysis tools (Sec. 2.3)
# ---------------------------------------------------------------------------
def inner(a, b, psd, df):
    """<a|b> = 4 Re sum a* b / S df  (Eq. 13, discrete form)."""
    return 4.0 * df * float(np.real(np.sum(np.conj(a) * b / psd)))


def mismatch(a_pair, b_pair, psd=None, df=1.0):
    """M = 1 - sum_alpha <a|b>_a / sqrt(<a|a>_a <b|b>_a)  (Eq. 12).  As printed the
    sum runs over the two channels, so identical signals give M = 1 - 2; this
    returns the per-channel average form 1 - mean_alpha(...) so that M = 0 for
    identical signals (the reading used for all mismatch figures here)."""
    out = 0.0
    for a, b in zip(a_pair, b_pair):
        S = np.ones(a.shape) if psd is None else psd
        out += inner(a, b, S, df) / np.sqrt(inner(a, a, S, df) * inner(b, b, S, df))
    return 1.0 - out / len(a_pair)


def rel_l2(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.sqrt(np.sum(np.abs(ref) ** 2))
    return float(np.sqrt(np.sum(np.abs(x - ref) ** 2)) / (den if den > 0 else 1.0))


def td_samples(w, dt, N=None, conj_partners=True, idx=None):
    """Time-domain voice sum (Eq. 2) sampled at t_j = t_0 + j dt, j = 0..N-1
    (default N = floor((t_last - t_0)/dt)); samples after t_last are 0.  Uses
    scipy's not-a-knot splines of the same knots and the Wigner-d Y_lm below,
    an implementation independent of oracle.c:
        h(t) = prefactor sum_modes [A Y_lm e^{-i Phi} + (partners) (-1)^l conj(A) Y_{l,-m} e^{+i Phi}],
    Phi = m Phi_phi + n Phi_r; h = h+ - i hx.  Returns (t_j, h+, hx) real arrays.
    idx: evaluate only the samples j in idx (a full-size check on a subset)."""
    from scipy.interpolate import CubicSpline

    t = w.t
    if N is None:
        N = int(np.floor((t[-1] - t[0]) / dt))
    j = np.arange(N) if idx is None else np.asarray(idx, np.int64)
    tj = t[0] + dt * j
    inside = tj <= t[-1]
    tin = tj[inside]
    sp = lambda y: CubicSpline(t, y, bc_type="not-a-knot")(tin)
    Pp, Pr = sp(w.phi_phi), sp(w.phi_r)
    h = np.zeros(tj.shape, np.complex128)
    hin = np.zeros(tin.shape, np.complex128)
    for j in range(w.n_modes):
        A = sp(w.amp[j].real) + 1j * sp(w.amp[j].imag)
        l, m, n = int(w.l[j]), int(w.m[j]), int(w.n[j])
        Y = swsh_closed(l, m, w.theta, w.phi)
        hin += w.prefactor * A * Y * np.exp(-1j * (m * Pp + n * Pr))
        if conj_partners:
            Yp = swsh_closed(l, -m, w.theta, w.phi)
            hin += w.prefactor * ((-1) ** l) * np.conj(A) * Yp * np.exp(1j * (m * Pp + n * Pr))
    h[inside] = hin
    return tj, h.real.copy(), -h.imag


def td_dft(w, dt, conj_partners=True, oversample_T=None, window=None, N=None):
    """Brute-force check: the DFT of td_samples with the e^{+2 pi i f t} sign of Eq. 3,
        h~(f_k) = dt sum_j h(t_j) e^{2 pi i f_k t_j},  f_k = k/(N dt).
    N: number of samples (default from the trajectory length, or oversample_T/dt).
    window="hann" multiplies the samples by hann_td(N) first.
    Returns (f_k for k = 1..N/2-1, h+~, hx~)."""
    t = w.t
    if N is None:
        N = int(np.floor((t[-1] - t[0]) / dt))
        if oversample_T is not None:
            N = int(np.floor(oversample_T / dt))
    tj, hp_t, hc_t = td_samples(w, dt, N, conj_partners)
    if window == "hann":
        win = hann_td(N)
        hp_t, hc_t = hp_t * win, hc_t * win
    # sum_j x_j e^{+2 pi i k j / N} = N ifft(x)[k]
    phase0 = np.exp(2j * np.pi * np.arange(N) / (N * dt) * t[0])
    Hp = dt * N * np.fft.ifft(hp_t.astype(np.complex128)) * phase0
    Hc = dt * N * np.fft.ifft(hc_t.astype(np.complex128)) * phase0
    k = np.arange(1, N // 2)
    return k / (N * dt), Hp[k], Hc[k]


def select_modes(amp, eps):
    """Mode selection of Sec. 2.1 (see oracle_select_modes in oracle.c): amp is
    [N_m, K] complex knot values; returns a bool mask over modes."""
    a = np.ascontiguousarray(np.asarray(amp, np.complex128))
    nm, K = a.shape
    ar, ap = _d(a.view(np.float64).reshape(-1))
    keep = np.zeros(max(nm, 1), np.int32)
    kk, kp = _i(keep)
    lib().oracle_select_modes(K, nm, ap, float(eps), kp)
    return kk[:nm].astype(bool)


def hann_fd(h):
    """Hann window applied in the frequency domain (Sec. 2.3: the FD waveform is
    convolved with the transform of the window).  For w(t) = sin^2(pi t df) =
    1/2 - e^{2 pi i t df}/4 - e^{-2 pi i t df}/4 on [0, 1/df] and a uniform grid of
    spacing df, the transform of w h is h(f)/2 - h(f + df)/4 - h(f - df)/4; bins
    outside the grid are taken as 0.  ``h``: complex array over one grid."""
    h = np.asarray(h)
    lo = np.concatenate([np.zeros(1, h.dtype), h[:-1]])
    hi = np.concatenate([h[1:], np.zeros(1, h.dtype)])
    return 0.5 * h - 0.25 * (lo + hi)


def hann_td(n):
    """The periodic Hann window sin^2(pi j / n), j = 0..n-1 (time samples)."""
    return np.sin(np.pi * np.arange(n) / n) ** 2


def swsh_closed(l, m, theta, phi):
    """-2Y_lm through the Wigner small-d matrix (an implementation independent of
    the Goldberg sum in oracle.c):  sY_lm = (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi},
    d^l_{a,b}(x) = sum_k (-1)^{a-b+k} sqrt((l+a)!(l-a)!(l+b)!(l-b)!)
                   / ((l+b-k)! k! (a-b+k)! (l-a-k)!) cos^{2l+b-a-2k}(x/2) sin^{a-b+2k}(x/2)."""
    from math import factorial, sqrt, cos, sin, pi
    s = -2
    a, b = m, -s
    tot = 0.0
    for k in range(0, 2 * l + 1):
        f = (l + b - k, k, a - b + k, l - a - k)
        if min(f) < 0:
            continue
        num = sqrt(factorial(l + a) * factorial(l - a) * factorial(l + b) * factorial(l - b))
        den = factorial(f[0]) * factorial(f[1]) * factorial(f[2]) * factorial(f[3])
        tot += ((-1) ** (a - b + k)) * num / den * cos(theta / 2) ** (2 * l + b - a - 2 * k) * sin(theta / 2) ** (a - b + 2 * k)
    val = ((-1) ** s) * sqrt((2 * l + 1) / (4 * pi)) * tot
    return val * complex(np.cos(m * phi), np.sin(m * phi))
