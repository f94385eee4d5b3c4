"""Every long numeric literal in the CUDA sources equals its definition, at the
precision the kernel uses it (the nearest double, the nearest float, or a float
pair hi + lo).  A wrong digit in most of them moves results by far less than the
parity bounds (a low word of 2 pi, a Taylor coefficient, a series constant of
the extended SPA), so the GPU tests alone would not catch it."""
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2307_12585_gb300", "csrc")


def _text(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def _lit(name, pattern):
    m = re.search(pattern, _text(name))
    assert m, "literal not found in %s: %s" % (name, pattern)
    return m.group(1)


def _check(kind, lit, value):
    if kind == "f64":
        assert float(lit) == float(value), (lit, float(value))
    elif kind == "f32":
        assert np.float32(float(lit)) == np.float32(float(value)), (lit, float(value))
    else:
        raise ValueError(kind)


def _cases(mp):
    pi = mp.pi
    two = mp.mpf(2)
    nu = mp.mpf(1) / 3
    a = [mp.mpf(1)]
    for k in range(1, 6):   # Hankel's expansion coefficients a_k(nu), nu = 1/3
        a.append(a[-1] * (4 * nu ** 2 - (2 * k - 1) ** 2) / (8 * k))
    f = r"([-0-9.e+]+)"
    return [
        ("spa_math.cuh", r"kTwoPiOver2p64 = " + f + ";", 2 * pi / two ** 64, "f64"),
        ("spa_math.cuh", r"rrf \* " + f + r"f;", 2 * pi * two ** 25 / two ** 64, "f32"),
        ("spa.cu", r"\* " + f + r"f,\s+// 2\^-34", two ** -34, "f32"),
        ("spa.cu", r"\* " + f + r"f\);\s+// 2\^-56", two ** -56, "f32"),
        ("spa.cu", r"\* " + f + r"f \+\s+// 2\^-21", two ** -21, "f32"),
        ("spa.cu", r"\* " + f + r"f;\s+// 2\^-43", two ** -43, "f32"),
        ("td.cu", r"\* " + f + r"f;\s+// 2 pi / 2\^32", 2 * pi / two ** 32, "f32"),
        ("spa.cu", r"__sincosf\(th \* " + f + r"f, &sn", pi, "f32"),
        ("adjoint.cu", r"kTwoPi = " + f + ";", 2 * pi, "f64"),
        ("adjoint.cu", r"kInv2Pi = " + f + ";", 1 / (2 * pi), "f64"),
        ("prep.cu", r"kTwoPi = " + f + ";", 2 * pi, "f64"),
        ("prep.cu", r"kInv2PiHi = " + f + ";", 1 / (2 * pi), "f64"),
        ("prep.cu", r"yk\[r\] = " + f + r" / h;", 3 / (2 * pi), "f64"),
        ("ext_spa.cuh", r"kExt3Over2Pi = " + f + ";", 3 / (2 * pi), "f64"),
        ("ext_spa.cuh", r"kExtA1 = " + f + ";", a[1], "f64"),
        ("ext_spa.cuh", r"kExtA2 = " + f + ";", a[2], "f64"),
        ("ext_spa.cuh", r"kExtA3 = " + f + ";", a[3], "f64"),
        ("ext_spa.cuh", r"kExtA4 = " + f + ";", a[4], "f64"),
        ("ext_spa.cuh", r"kExtA5 = " + f + ";", a[5], "f64"),
        ("ext_spa.cuh", r"kExtCoalesced = " + f + ";",
         2 * pi ** (two / 3) / (3 ** (two / 3) * mp.gamma(two / 3)), "f64"),
        ("ext_spa.cuh", r"1\.0 / " + f + r";\s+// 1/Gamma\(2/3\)", mp.gamma(two / 3), "f64"),
        ("ext_spa.cuh", r"1\.0 / " + f + r";\s+// 1/Gamma\(4/3\)", mp.gamma(two ** 2 / 3), "f64"),
        ("ext_spa.cuh", r"x16 \* " + f + r" \* s1;", mp.cbrt(2), "f64"),
        ("ext_spa.cuh", r"\(X / x16\) \* " + f + r" \* s2;", 1 / mp.cbrt(2), "f64"),
        ("ext_spa.cuh", r"c12 = " + f + ",", mp.cos(pi / 12), "f64"),
        ("ext_spa.cuh", r"s12 = " + f + ";", mp.sin(pi / 12), "f64"),
        ("ext_spa.cuh", r"k0 = " + f + r";\s+// sqrt\(2 pi/3\)", mp.sqrt(2 * pi / 3), "f64"),
    ]


def test_literals_equal_their_definitions():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for name, pattern, value, kind in _cases(mp):
        _check(kind, _lit(name, pattern), value)


def test_float_and_double_pairs():
    """2 pi as an FP32 pair (the FP64X phase) and 1/(2 pi) as an FP64 pair (the
    Q0.64 knot phases): hi is the nearest value, lo the nearest value of the rest."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    m = re.search(r"ff_make\(([-0-9.e+]+)f, ([-0-9.e+]+)f\)\);", _text("spa.cu"))
    hi, lo = np.float32(float(m.group(1))), np.float32(float(m.group(2)))
    assert hi == np.float32(float(2 * mp.pi))
    assert lo == np.float32(float(2 * mp.pi - mp.mpf(float(hi))))
    hi2 = float(_lit("prep.cu", r"kInv2PiHi = ([-0-9.e+]+);"))
    lo2 = float(_lit("prep.cu", r"kInv2PiLo = ([-0-9.e+]+);"))
    assert hi2 == float(1 / (2 * mp.pi))
    assert lo2 == float(1 / (2 * mp.pi) - mp.mpf(hi2))


def test_reciprocal_factorials():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    body = re.search(r"c_invfact\[41\] = \{([^}]*)\}", _text("prep.cu")).group(1)
    vals = [float(v) for v in body.split(",")]
    assert len(vals) == 41
    for k, v in enumerate(vals):
        assert v == float(1 / mp.factorial(k)), k


def test_oracle_constants():
    """The oracle's double-double 2 pi and pi/4 (its phase is carried to ~1e-32 of a
    turn before reduction) and pi; an error in a low word would sit far below its pins."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    with open(os.path.join(os.path.dirname(CSRC), "..", "oracle", "oracle.c")) as fh:
        src = fh.read()
    d = {k: float(v) for k, v in re.findall(r"#define (OR_[A-Z_]+) ([-0-9.e+]+)", src)}
    for name, value in (("TWO_PI", 2 * mp.pi), ("QPI", mp.pi / 4)):
        hi, lo = d["OR_%s_HI" % name], d["OR_%s_LO" % name]
        assert hi == float(value) and lo == float(value - mp.mpf(hi)), name
    assert d["OR_PI"] == float(mp.pi)
