"""Pins of the oracle's spin-weight -2 spherical harmonics (Eq. 1: for
Schwarzschild the spheroidal harmonics are spin-weighted spherical harmonics)."""
import math

import numpy as np
import pytest


def textbook_l2(m, th, ph):
    c = math.cos(th)
    s = math.sin(th)
    f = {
        2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
        1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c),
        0: math.sqrt(15 / (32 * math.pi)) * s * s,
        -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
        -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2,
    }[m]
    return f * complex(math.cos(m * ph), math.sin(m * ph))


def textbook_l3(m, th, ph):
    c = math.cos(th)
    s = math.sin(th)
    f = {
        3: -math.sqrt(21 / (2 * math.pi)) * math.cos(th / 2) ** 5 * math.sin(th / 2),
        -3: math.sqrt(21 / (2 * math.pi)) * math.cos(th / 2) * math.sin(th / 2) ** 5,
        0: math.sqrt(105 / (2 * math.pi)) * c * math.sin(th / 2) ** 2 * math.cos(th / 2) ** 2,
    }[m]
    return f * complex(math.cos(m * ph), math.sin(m * ph))


@pytest.mark.parametrize("th,ph", [(0.7, 1.1), (2.3, -0.4), (1e-3, 0.0), (math.pi / 2, 3.0)])
def test_l2_closed_forms(oracle, th, ph):
    for m in range(-2, 3):
        assert abs(oracle.swsh(-2, 2, m, th, ph) - textbook_l2(m, th, ph)) < 1e-14


@pytest.mark.parametrize("m", [3, 0, -3])
def test_l3_closed_forms(oracle, m):
    for th in (0.3, 1.7, 2.9):
        assert abs(oracle.swsh(-2, 3, m, th, 0.9) - textbook_l3(m, th, 0.9)) < 1e-14


def test_matches_wigner_d_form(oracle):
    for l in range(2, 11):
        for m in range(-l, l + 1):
            a = oracle.swsh(-2, l, m, 0.7, 1.1)
            b = oracle.swsh_closed(l, m, 0.7, 1.1)
            assert abs(a - b) < 1e-12


def test_orthonormal(oracle):
    # Gauss-Legendre in cos(theta) x uniform in phi: exact for these band-limited products
    x, wx = np.polynomial.legendre.leggauss(48)
    th = np.arccos(x)
    nph = 48
    ph = 2 * np.pi * np.arange(nph) / nph
    modes = [(l, m) for l in range(2, 6) for m in range(-l, l + 1)]
    Y = np.array([[[oracle.swsh(-2, l, m, a, b) for b in ph] for a in th] for (l, m) in modes])
    G = np.einsum("iab,jab,a->ij", np.conj(Y), Y, wx) * (2 * np.pi / nph)
    assert np.max(np.abs(G - np.eye(len(modes)))) < 1e-12


def test_conjugation_identity(oracle):
    # sY*_lm = (-1)^(s+m) (-s)Y_{l,-m}
    for l in range(2, 7):
        for m in range(-l, l + 1):
            a = np.conj(oracle.swsh(-2, l, m, 1.3, 0.6))
            b = (-1) ** (-2 + m) * oracle.swsh(2, l, -m, 1.3, 0.6)
            assert abs(a - b) < 1e-13


def _wigner_form_mp(l, m, th, ph):
    """-2Y_lm from the Wigner small-d sum evaluated in 50-digit arithmetic with exact
    factorials, so its own cancellation (which grows with l) plays no part."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    s = -2
    a, b = m, -s
    c, sn = mp.cos(mp.mpf(th) / 2), mp.sin(mp.mpf(th) / 2)
    tot = mp.mpf(0)
    for k in range(0, 2 * l + 1):
        f = (l + b - k, k, a - b + k, l - a - k)
        if min(f) < 0:
            continue
        num = mp.sqrt(mp.mpf(math.factorial(l + a) * math.factorial(l - a) * math.factorial(l + b) * math.factorial(l - b)))
        den = math.factorial(f[0]) * math.factorial(f[1]) * math.factorial(f[2]) * math.factorial(f[3])
        tot += (-1) ** (a - b + k) * num / den * c ** (2 * l + b - a - 2 * k) * sn ** (a - b + 2 * k)
    v = (-1) ** s * mp.sqrt(mp.mpf(2 * l + 1) / (4 * mp.pi)) * tot
    return complex(v * mp.cos(m * mp.mpf(ph)), v * mp.sin(m * mp.mpf(ph)))


@pytest.mark.parametrize("l", [15, 20])
def test_high_l_against_extended_precision(oracle, l):
    # up to l = 20, the largest degree the library accepts; the FP64 sums lose about
    # 1e-11 to cancellation there (the oracle's measured worst case is 7e-12)
    tol = {15: 1e-12, 20: 2e-11}[l]
    for m in range(-l, l + 1):
        for th in (0.2, 1.9, 2.9):
            assert abs(oracle.swsh(-2, l, m, th, -0.8) - _wigner_form_mp(l, m, th, -0.8)) < tol


def test_high_l_orthonormal(oracle):
    x, wx = np.polynomial.legendre.leggauss(48)
    th = np.arccos(x)
    nph = 48
    ph = 2 * np.pi * np.arange(nph) / nph
    modes = [(l, m) for l in (19, 20) for m in (-l, -7, 0, 3, l)]
    Y = np.array([[[oracle.swsh(-2, l, m, a, b) for b in ph] for a in th] for (l, m) in modes])
    G = np.einsum("iab,jab,a->ij", np.conj(Y), Y, wx) * (2 * np.pi / nph)
    assert np.max(np.abs(G - np.eye(len(modes)))) < 1e-10
