"""Pins of the oracle's inner product (Eq. 13) and mismatch (Eq. 12) by their
closed forms: M = 0 for identical or positively scaled signals, M = 1 - cos(phi)
for a common phase rotation, (1 - cos phi)/2 when one of the two channels is
rotated (the per-channel average reading), 1 for signals on disjoint bins, and
the PSD weighting of a two-bin signal, (1 - cos phi)/(1 + s) with S = (1, s)."""
import numpy as np
import pytest


def _pair(seed, n=257):
    rng = np.random.default_rng(seed)
    return tuple(rng.normal(size=n) + 1j * rng.normal(size=n) for _ in range(2))


def test_inner_is_4_df_re_sum_over_psd(oracle):
    O = oracle
    # <a|b> for one-bin signals: 4 df Re(conj(a) b)/S
    assert O.inner(np.array([1 + 2j]), np.array([3 - 1j]), np.array([2.0]), 0.5) == pytest.approx(4 * 0.5 * (1.0 / 2))
    assert O.inner(np.array([1j]), np.array([1.0]), np.array([1.0]), 1.0) == 0.0


def test_identical_and_scaled(oracle):
    O = oracle
    a = _pair(1)
    assert abs(O.mismatch(a, a)) < 1e-15
    assert abs(O.mismatch(a, tuple(3.7 * x for x in a))) < 1e-15
    S = np.linspace(1.0, 5.0, a[0].size)
    assert abs(O.mismatch(a, a, psd=S, df=0.3)) < 1e-15


@pytest.mark.parametrize("phi", [1e-3, 0.4, 2.0, np.pi])
def test_phase_rotation(oracle, phi):
    O = oracle
    a = _pair(2)
    rot = np.exp(1j * phi)
    assert O.mismatch(a, tuple(rot * x for x in a)) == pytest.approx(1 - np.cos(phi), rel=1e-12, abs=1e-15)
    # one channel rotated: the average over the two channels
    assert O.mismatch(a, (a[0], rot * a[1])) == pytest.approx((1 - np.cos(phi)) / 2, rel=1e-12, abs=1e-15)


def test_disjoint_support_is_one(oracle):
    O = oracle
    a = _pair(3)
    b = _pair(4)
    lo = tuple(np.where(np.arange(x.size) < 100, x, 0) for x in a)
    hi = tuple(np.where(np.arange(x.size) >= 100, x, 0) for x in b)
    assert O.mismatch(lo, hi) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("s", [0.25, 4.0, 100.0])
def test_psd_weighting(oracle, s):
    O = oracle
    phi = 0.9
    a = (np.array([1.0 + 0j, 1.0 + 0j]),) * 2
    b = (np.array([1.0 + 0j, np.exp(1j * phi)]),) * 2
    S = np.array([1.0, s])
    assert O.mismatch(a, b, psd=S, df=2.0) == pytest.approx((1 - np.cos(phi)) / (1 + s), rel=1e-12)


def test_symmetric_and_small_perturbation(oracle):
    O = oracle
    a = _pair(5)
    rng = np.random.default_rng(6)
    d = tuple(1e-4 * (rng.normal(size=x.size) + 1j * rng.normal(size=x.size)) for x in a)
    b = tuple(x + y for x, y in zip(a, d))
    m = O.mismatch(a, b)
    assert m == pytest.approx(O.mismatch(b, a), rel=1e-9)
    # second order in the perturbation: at most half the squared relative L2 of the worse channel
    e = max(np.linalg.norm(y) / np.linalg.norm(x) for x, y in zip(a, d))
    assert 0 < m <= 0.5 * e ** 2 * 1.001
