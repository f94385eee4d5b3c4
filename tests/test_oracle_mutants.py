"""The pins catch plausible mistakes: each case plants one mistake in a copy of the
C oracle (a dropped or flipped term, a wrong index or sign, a wrong boundary
condition), builds it on the CPU, and runs the oracle's own pins on it; at least one
pin must fail.  The unmodified source passes the same battery, so a failure is the
planted mistake's doing."""
import importlib.util
import os
import shutil
import subprocess

import pytest

from tests import test_oracle_closed_form as CF
from tests import test_oracle_fft as FFT
from tests import test_oracle_invariants as INV
from tests import test_oracle_spline as SPL
from tests import test_oracle_ylm as YLM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, exact text in oracle.c, replacement); each text occurs once
MUTANTS = [
    ("pi/4 sign", "if (!ext) psi = dd_add(psi, Fd > 0.0 ? dd_neg(qpi) : qpi);",
     "if (!ext) psi = dd_add(psi, Fd > 0.0 ? qpi : dd_neg(qpi));"),
    ("weight exponent", "double w = 1.0 / sqrt(fabs(Fd));\n  acc[0] += w", "double w = 1.0 / fabs(Fd);\n  acc[0] += w"),
    ("phase sign", "dd_mul_d(Pr, (double)V->n));\n  dd_t psi = dd_add(wgt, dd_neg(PV));",
     "dd_mul_d(Pr, (double)V->n));\n  dd_t psi = dd_add(wgt, PV);"),
    ("partner amplitude sign (-1)^m", "double sgn = (l[j] & 1) ? -1.0 : 1.0;", "double sgn = (m[j] & 1) ? -1.0 : 1.0;"),
    ("partner n not negated", "v->n = part ? -n[j] : n[j];", "v->n = n[j];"),
    ("h_x sign", "hc[2 * b] = -0.5 * (pi - ni);  hc[2 * b + 1] = 0.5 * (pr - nr);",
     "hc[2 * b] = 0.5 * (pi - ni);  hc[2 * b + 1] = -0.5 * (pr - nr);"),
    ("conj H(-f) dropped", "nr = Hneg[2 * b], ni = -Hneg[2 * b + 1];", "nr = 0.0 * Hneg[2 * b], ni = 0.0;"),
    ("natural spline end", "AA(0, 0) = -h1; AA(0, 1) = h0 + h1; AA(0, 2) = -h0; }",
     "AA(0, 0) = 1.0; AA(0, 1) = 0.0; AA(0, 2) = 0.0; }"),
    ("spline c = M/3", "coef[4 * k + 2] = M[k] / 2.0;", "coef[4 * k + 2] = M[k] / 3.0;"),
    ("voice frequency sign of n", "c4[j] = ((double)mv * T->cOp[4 * k + j] + (double)nv * T->cOr[4 * k + j]) / OR_TWO_PI_HI;",
     "c4[j] = ((double)mv * T->cOp[4 * k + j] - (double)nv * T->cOr[4 * k + j]) / OR_TWO_PI_HI;"),
    ("Y_lm alternating sign", "(((l - r - s) & 1) ? -1.0 : 1.0)", "(((l - r + s + 1) & 1) ? -1.0 : 1.0)"),
    ("Y_lm prefactor (l+s)! -> (l+m)!", "(4.0 * OR_PI * fact(l + s) * fact(l - s))", "(4.0 * OR_PI * fact(l + m) * fact(l - s))"),
    ("second branch at a turnover dropped", "for (int i = 0; i < nr; i++) { xs[nx] = r[i]; Fs[nx++] = cubic(fc, r[i]); }",
     "for (int i = 0; i < nr && i < 0; i++) { xs[nx] = r[i]; Fs[nx++] = cubic(fc, r[i]); }"),
]

# the pins run on each mutant, cheapest first
BATTERY = [
    ("ylm l=2", lambda O: YLM.test_l2_closed_forms(O, 0.7, 1.1)),
    ("ylm l=3", lambda O: YLM.test_l3_closed_forms(O, 3)),
    ("spline vs scipy", lambda O: SPL.test_matches_scipy_not_a_knot(O, 17)),
    ("partners explicit", lambda O: INV.test_conj_partners_explicit(O)),
    ("linear chirp", lambda O: CF.test_linear_chirp(O)),
    ("linear chirp from two series", lambda O: CF.test_linear_chirp_from_two_series(O)),
    ("quadratic turnover", lambda O: CF.test_quadratic_turning_point(O, False)),
    ("quadratic turnover mid-segment", lambda O: CF.test_quadratic_turning_point(O, True)),
    ("DFT of TD, 4 voices", lambda O: FFT.test_spa_matches_dft_of_time_domain(O, [(2, 2, 0), (3, 3, 2), (2, 1, -3), (3, 1, 1)])),
    ("DFT of TD, turnover voice", lambda O: FFT.test_turning_point_voice_matches_dft_away_from_turnover(O)),
]


def _oracle_from(src_text, tmp):
    """A separate copy of the oracle module bound to a library built from src_text."""
    os.makedirs(tmp, exist_ok=True)
    src = os.path.join(tmp, "oracle.c")
    lib = os.path.join(tmp, "liboracle.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                           "-shared", "-o", lib, src, "-lm"])
    spec = importlib.util.spec_from_file_location("oracle_copy_%d" % abs(hash(tmp)), os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.BUILD, mod.LIB, mod.SRC = tmp, lib, src
    return mod


def _first_failing_pin(O):
    for name, pin in BATTERY:
        try:
            pin(O)
        except AssertionError:
            return name
    return None


@pytest.fixture(scope="module")
def source():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    with open(SRC) as f:
        return f.read()


def test_unmodified_oracle_passes_the_battery(source, tmp_path):
    assert _first_failing_pin(_oracle_from(source, str(tmp_path / "orig"))) is None


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(source, tmp_path, name, old, new):
    assert source.count(old) == 1, "mutation site not found (or not unique): %s" % name
    caught = _first_failing_pin(_oracle_from(source.replace(old, new), str(tmp_path / "m")))
    assert caught is not None, "no pin catches: %s" % name
