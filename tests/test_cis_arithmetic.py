"""The FP64 form's phase factor e^{ix} (|x| <= pi/65536 after the table entry) is
formed as (1 - q)(1 + i x'), q = x^2/2, x' = x (1 + x^2/3): q in FP32 from the top
bits of the Q0.64 remainder rr, x' from rr plus an integer correction, and 1 - q
folded into the weight's Newton step through c1 = 1 - 2q.  Its error (below 1e-15)
is far under the 1e-10 parity bound, so the GPU tests cannot see a wrong constant
here.  These CPU checks hold the constants in the kernel source to their
definitions and replay the kernel's FP32/integer steps in numpy (IEEE
round-to-nearest, as the kernel's __fmul_rn/__fadd_rn) against mpmath."""
import math
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2307_12585_gb300", "csrc",
                   "spa_math.cuh")


def _helper_source():
    s = open(SRC).read()
    i = s.index("void cis_split_q64(")
    return s[i:s.index("\n}\n", i)]


def _literals():
    h = _helper_source()
    x = float(re.search(r"rrf \* ([0-9.e+-]+)f;", h).group(1))
    corr = float(re.search(r"__fmul_rn\(qf, ([0-9.e+-]+)f\)\);", h).group(1))
    qsc = float(re.search(r"__fmul_rn\(qf, ([0-9.]+)f\), 12582912\.0f\)", h).group(1))
    k2p = float(re.search(r"kTwoPiOver2p64 = ([0-9.e+-]+);", open(SRC).read()).group(1))
    return x, corr, qsc, k2p


def test_constants_match_their_definitions():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, corr, qsc, k2p = _literals()
    assert np.float32(x) == np.float32(float(2 * mp.pi * mp.mpf(2) ** 25 / mp.mpf(2) ** 64))   # 2 pi 2^25/2^64
    assert np.float32(corr) == np.float32(float(mp.mpf(2) ** 26 / 3))                          # 2^26/3
    assert qsc == 2.0 ** 51
    assert k2p == float(2 * mp.pi / mp.mpf(2) ** 64)
    assert "12582912.0f" in _helper_source() and "0x4B400000" in _helper_source()   # 1.5 2^23, its bits


def _f32_bits(v):
    return int(np.array([v], np.float32).view(np.int32)[0])


def _small_int_to_float(v):   # exact for |v| <= 2^22, as the kernel forms it
    return np.float32(np.array([0x4B400000 + v], np.int32).view(np.float32)[0] - np.float32(12582912.0))


def _replay(rr, lits):
    x, corr_c, qsc, k2p = lits
    f = np.float32
    rrf = _small_int_to_float((rr + (1 << 24)) >> 25)
    xf = f(rrf * f(x))
    qf = f(f(f(0.5) * xf) * xf)
    corr = f(rrf * f(qf * f(corr_c)))
    ci = _f32_bits(f(corr + f(12582912.0))) - 0x4B400000
    xp = float(rr + ci) * k2p                 # the integer is exact in a double (|.| < 2^52)
    qi = _f32_bits(f(f(qf * f(qsc)) + f(12582912.0))) - 0x4B400000
    c1 = float(np.array([0x3FF0000000000000 - (qi << 3)], np.int64).view(np.float64)[0])
    return xp, c1


def test_factor_matches_exp_ix():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    lits = _literals()
    rng = np.random.default_rng(5)
    rrs = [int(v) for v in rng.integers(-2 ** 47, 2 ** 47, 4000)]
    rrs += [2 ** 47, -2 ** 47, 0, 1, -1, 2 ** 24, -2 ** 24, 2 ** 25 - 1, -(2 ** 25) - 1, 3 << 45]
    worst = 0.0
    for rr in rrs:
        xp, c1 = _replay(rr, lits)
        x = mp.mpf(rr) * 2 * mp.pi / mp.mpf(2) ** 64
        one_minus_q = 1 - (1 - mp.mpf(c1)) / 2          # the weight's real factor (1 - q)
        err = abs(one_minus_q * (1 + 1j * mp.mpf(xp)) - mp.expj(x))
        worst = max(worst, float(err))
    # the previous form, which dropped x^3/6, reached 1.9e-14 at |x| = pi/65536
    assert worst < 1e-15, worst
    assert (math.pi / 65536) ** 3 / 6 > 1e-14


def test_weight_step_folds_the_factor():
    """cw = y0 + (y0/2)(c1 - |D| y0^2) equals (1 - q) times the step with c1 = 1, to
    |e| q/2 plus rounding: y0 is an FP32 reciprocal square root within 2 ulp."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    lits = _literals()
    rng = np.random.default_rng(6)

    def step(D, y0, c1):   # the kernel's two FMAs, each rounded once
        y0h, y0sq = mp.mpf(float(np.float32(0.5) * y0)), mp.mpf(float(y0)) ** 2   # both exact
        e = mp.mpf(float(-mp.mpf(D) * y0sq + mp.mpf(c1)))
        return mp.mpf(float(y0h * e + mp.mpf(float(y0))))

    worst = 0.0
    for _ in range(2000):
        D = float(10 ** rng.uniform(-12, 6))
        y0 = np.float32(1 / math.sqrt(D)) * np.float32(1 + rng.uniform(-2.4e-7, 2.4e-7))
        rr = int(rng.integers(-2 ** 47, 2 ** 47))
        _, c1 = _replay(rr, lits)
        q = (1 - mp.mpf(c1)) / 2
        a, b = step(D, y0, c1), step(D, y0, 1.0) * (1 - q)
        worst = max(worst, float(abs(a - b) / b))
    # |e| q/2 <= 4.8e-7 x 1.15e-9 / 2 = 2.8e-16, plus one rounding in each of the two steps
    assert worst < 2.8e-16 + 2 * 2.0 ** -53, worst
