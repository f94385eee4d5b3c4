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
