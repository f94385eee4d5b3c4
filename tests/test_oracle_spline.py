"""Pins of the oracle's not-a-knot spline (Sec. 2.1: amplitudes, phases and
frequencies are interpolated with not-a-knot cubic splines)."""
import numpy as np
import pytest
from scipy.interpolate import CubicSpline


def _eval(coef, t, x):
    k = np.clip(np.searchsorted(t, x, side="right") - 1, 0, len(t) - 2)
    tau = x - t[k]
    c = coef[k]
    return c[:, 0] + tau * (c[:, 1] + tau * (c[:, 2] + tau * c[:, 3]))


@pytest.mark.parametrize("K", [4, 5, 17, 100, 200])
def test_matches_scipy_not_a_knot(oracle, K):
    rng = np.random.default_rng(K)
    t = np.cumsum(rng.uniform(0.5, 1.5, K)) * 3e5
    y = np.sin(t / t[-1] * 7.0) * 1e3 + rng.normal(size=K)
    c = oracle.spline_coef(t, y)
    x = np.linspace(t[0], t[-1], 5001)
    ref = CubicSpline(t, y, bc_type="not-a-knot")(x)
    assert np.max(np.abs(_eval(c, t, x) - ref)) <= 1e-11 * np.max(np.abs(y))
    # interpolates the knots exactly in its a-coefficient
    assert np.array_equal(c[:, 0], y[:-1])


@pytest.mark.parametrize("K", [4, 9, 150])
def test_reproduces_cubics(oracle, K):
    rng = np.random.default_rng(100 + K)
    t = np.sort(rng.uniform(0, 6e7, K))
    T = t[-1] - t[0]
    cc = rng.normal(size=4)
    poly = lambda x: cc[0] + cc[1] * ((x - t[0]) / T) + cc[2] * ((x - t[0]) / T) ** 2 + cc[3] * ((x - t[0]) / T) ** 3
    c = oracle.spline_coef(t, poly(t))
    x = np.linspace(t[0], t[-1], 3001)
    assert np.max(np.abs(_eval(c, t, x) - poly(x))) <= 1e-12 * np.max(np.abs(cc)) * 10


def test_rejects_short(oracle):
    with pytest.raises(ValueError):
        oracle.spline_coef(np.arange(3.0), np.arange(3.0))
