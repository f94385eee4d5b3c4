"""Pins of the oracle's mode selection (Sec. 2.1): per knot, modes ordered by
decreasing |A|^2 are taken while the power before them is below 1 - eps of
the total; the selection is the union over knots.

The pins use a characterisation that needs no sort: mode j is kept at knot k
iff the power of the modes ordered before it (larger power, or equal power
and a smaller index) is below (1 - eps) of the total.  On small-integer
amplitudes and dyadic eps every sum is exact in FP64, so it is computed in
exact integer arithmetic here.  Plus limits, monotonicity in eps, the union
over knots, permutation and power-of-two scale invariance."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2307_12585_gb300 import synth


def _brute(amp, eps):
    nm, K = amp.shape
    keep = np.zeros(nm, bool)
    P = (amp.real.astype(np.int64) ** 2 + amp.imag.astype(np.int64) ** 2)
    for k in range(K):
        p = [int(x) for x in P[:, k]]
        tot = sum(p)
        thr = (1 - Fraction(eps)) * tot
        for j in range(nm):
            before = sum(p[i] for i in range(nm) if p[i] > p[j] or (p[i] == p[j] and i < j))
            if before < thr:
                keep[j] = True
    return keep


@pytest.mark.parametrize("seed", range(6))
def test_matches_exact_characterisation(oracle, seed):
    rng = np.random.default_rng(seed)
    nm, K = int(rng.integers(1, 40)), int(rng.integers(1, 6))
    amp = rng.integers(-30, 31, (nm, K)) + 1j * rng.integers(-30, 31, (nm, K))
    if seed == 0:
        amp[:, :] = 3 + 4j          # all powers equal: ties decided by index
    for eps in (0.5, 0.125, 1 / 64, 1 / 1024, 0.0, 1.0):
        assert np.array_equal(oracle.select_modes(amp, eps), _brute(amp, eps)), eps


def test_limits_and_monotone(oracle):
    w = synth.paper_config(1, n_modes=3294)
    A = w.amp
    assert oracle.select_modes(A, 1.0).sum() == 0
    assert oracle.select_modes(A, 0.0).sum() == np.count_nonzero(np.any(np.abs(A) > 0, axis=1))
    prev = None
    for eps in (1e-1, 1e-2, 1e-3, 1e-5, 1e-8):
        s = oracle.select_modes(A, eps)
        if prev is not None:
            assert np.all(s >= prev)          # smaller eps: a superset
        prev = s
    n5 = int(oracle.select_modes(A, 1e-5).sum())
    assert 100 < n5 < 3294


def test_union_over_knots(oracle):
    w = synth.paper_config(2, n_modes=3294)
    A = w.amp[:, ::20]
    full = oracle.select_modes(A, 1e-3)
    union = np.zeros_like(full)
    for k in range(A.shape[1]):
        union |= oracle.select_modes(A[:, k:k + 1], 1e-3)
    assert np.array_equal(full, union)


def test_permutation_and_scale(oracle):
    w = synth.paper_config(3, n_modes=3294)
    A = w.amp
    s = oracle.select_modes(A, 1e-4)
    perm = np.random.default_rng(0).permutation(A.shape[0])
    assert np.array_equal(oracle.select_modes(A[perm], 1e-4), s[perm])
    assert np.array_equal(oracle.select_modes(A * 2.0 ** 40, 1e-4), s)
