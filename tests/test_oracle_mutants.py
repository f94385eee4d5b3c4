"""The pins catch plausible mistakes: each case plants one mistake in a copy of the
oracle (a dropped or flipped term, a wrong index, sign, factor or boundary
condition) in its C part or its Python part, builds it on the CPU, and runs the
oracle's own pins on it; at least one pin must fail.  The unmodified sources
pass the same battery, so a failure is the planted mistake's doing."""
import importlib.util
import os
import shutil
import subprocess

import pytest

from tests import test_oracle_closed_form as CF
from tests import test_oracle_ext as EXT
from tests import test_oracle_fft as FFT
from tests import test_oracle_grad as GRAD
from tests import test_oracle_mismatch as MM
from tests import test_oracle_invariants as INV
from tests import test_oracle_select as SEL
from tests import test_oracle_spline as SPL
from tests import test_oracle_td as TD
from tests import test_oracle_window as WIN
from tests import test_oracle_ylm as YLM

ROOT = os.path.dirname(os.path.abspath(os.path.dirname(__file__)))
SRC_C = os.path.join(ROOT, "oracle", "oracle.c")
SRC_PY = os.path.join(ROOT, "oracle", "oracle.py")

# (name, file "c" or "py", group, exact text in that file, replacement); each text occurs once
MUTANTS = [
    # standard SPA sum (Sec. 2.2, Eq. 3-6)
    ("pi/4 sign", "c", "spa", "if (!ext) psi = dd_add(psi, Fd > 0.0 ? dd_neg(qpi) : qpi);",
     "if (!ext) psi = dd_add(psi, Fd > 0.0 ? qpi : dd_neg(qpi));"),
    ("weight exponent", "c", "spa", "double w = 1.0 / sqrt(fabs(Fd));\n  acc[0] += w", "double w = 1.0 / fabs(Fd);\n  acc[0] += w"),
    ("phase sign", "c", "spa", "dd_mul_d(Pr, (double)V->n));\n  dd_t psi = dd_add(wgt, dd_neg(PV));",
     "dd_mul_d(Pr, (double)V->n));\n  dd_t psi = dd_add(wgt, PV);"),
    ("partner amplitude sign (-1)^m", "c", "spa", "double sgn = (l[j] & 1) ? -1.0 : 1.0;", "double sgn = (m[j] & 1) ? -1.0 : 1.0;"),
    ("partner n not negated", "c", "spa", "v->n = part ? -n[j] : n[j];", "v->n = n[j];"),
    ("h_x sign", "c", "spa", "hc[2 * b] = -0.5 * (pi - ni);  hc[2 * b + 1] = 0.5 * (pr - nr);",
     "hc[2 * b] = 0.5 * (pi - ni);  hc[2 * b + 1] = -0.5 * (pr - nr);"),
    ("conj H(-f) dropped", "c", "spa", "nr = Hneg[2 * b], ni = -Hneg[2 * b + 1];", "nr = 0.0 * Hneg[2 * b], ni = 0.0;"),
    ("natural spline end", "c", "spa", "AA(0, 0) = -h1; AA(0, 1) = h0 + h1; AA(0, 2) = -h0; }",
     "AA(0, 0) = 1.0; AA(0, 1) = 0.0; AA(0, 2) = 0.0; }"),
    ("spline c = M/3", "c", "spa", "coef[4 * k + 2] = M[k] / 2.0;", "coef[4 * k + 2] = M[k] / 3.0;"),
    ("voice frequency sign of n", "c", "spa",
     "c4[j] = ((double)mv * T->cOp[4 * k + j] + (double)nv * T->cOr[4 * k + j]) / OR_TWO_PI_HI;",
     "c4[j] = ((double)mv * T->cOp[4 * k + j] - (double)nv * T->cOr[4 * k + j]) / OR_TWO_PI_HI;"),
    ("Y_lm alternating sign", "c", "spa", "(((l - r - s) & 1) ? -1.0 : 1.0)", "(((l - r + s + 1) & 1) ? -1.0 : 1.0)"),
    ("Y_lm prefactor (l+s)! -> (l+m)!", "c", "spa", "(4.0 * OR_PI * fact(l + s) * fact(l - s))",
     "(4.0 * OR_PI * fact(l + m) * fact(l - s))"),
    ("second branch at a turnover dropped", "c", "spa",
     "for (int i = 0; i < nr; i++) { xs[nx] = r[i]; Fs[nx++] = cubic(fc, r[i]); }",
     "for (int i = 0; i < nr && i < 0; i++) { xs[nx] = r[i]; Fs[nx++] = cubic(fc, r[i]); }"),
    # extended SPA factor (Eq. 7-10)
    ("Eq. 10 factor not negated", "c", "ext", "return -(2.0 / sqrt(3.0)) * (I * Fd / fabs(Fdd)) * ext_E(X);",
     "return (2.0 / sqrt(3.0)) * (I * Fd / fabs(Fdd)) * ext_E(X);"),
    ("K_nu integrand exponent", "c", "ext", "cpow(2.0 + I * ev, -1.0 / 6.0)", "cpow(2.0 + I * ev, 1.0 / 6.0)"),
    ("X loses the sign of Fdot", "c", "ext", "const double X = 2.0 * OR_PI * Fd * Fd * Fd / (3.0 * Fdd * Fdd);",
     "const double X = 2.0 * OR_PI * Fd * Fd * fabs(Fd) / (3.0 * Fdd * Fdd);"),
    ("double-root Gamma(2/3) -> Gamma(1/3)", "c", "ext", "tgamma(2.0 / 3.0)) / cbrt(fabs(Fdd));",
     "tgamma(1.0 / 3.0)) / cbrt(fabs(Fdd));"),
    ("Fresnel limit sign", "c", "ext", "return cexp(-I * (Fd > 0.0 ? 1.0 : -1.0) * (OR_PI / 4.0)) / sqrt(fabs(Fd));",
     "return cexp(I * (Fd > 0.0 ? 1.0 : -1.0) * (OR_PI / 4.0)) / sqrt(fabs(Fd));"),
    # mode selection (Sec. 2.1)
    ("selection sorted by ascending power", "c", "select", "if (x->p > y->p) return -1;\n  if (x->p < y->p) return 1;",
     "if (x->p > y->p) return 1;\n  if (x->p < y->p) return -1;"),
    ("selection threshold eps instead of 1 - eps", "c", "select", "const double thr = (1.0 - eps) * total;",
     "const double thr = eps * total;"),
    # Hann window (Sec. 2.3)
    ("three-term window sign", "py", "window", "return 0.5 * h - 0.25 * (lo + hi)", "return 0.5 * h + 0.25 * (lo + hi)"),
    ("symmetric instead of periodic window", "py", "window", "return np.sin(np.pi * np.arange(n) / n) ** 2",
     "return np.sin(np.pi * np.arange(n) / (n - 1)) ** 2"),
    # time-domain voice sum (Eq. 2)
    ("TD partner phase sign", "py", "td",
     "hin += w.prefactor * ((-1) ** l) * np.conj(A) * Yp * np.exp(1j * (m * Pp + n * Pr))",
     "hin += w.prefactor * ((-1) ** l) * np.conj(A) * Yp * np.exp(-1j * (m * Pp + n * Pr))"),
    ("TD h_x sign", "py", "td", "return tj, h.real.copy(), -h.imag", "return tj, h.real.copy(), h.imag"),
    # Whittle likelihood and its knot gradient (Eq. 13-14)
    ("likelihood -2 df -> -df", "c", "grad", "L += -2.0 * df * (rpr * rpr + rpi * rpi + rcr * rcr + rci * rci) / psd[i];",
     "L += -1.0 * df * (rpr * rpr + rpi * rpi + rcr * rcr + rci * rci) / psd[i];"),
    ("residual weight 4 df -> 2 df", "c", "grad", "double s = 4.0 * df / psd[i];", "double s = 2.0 * df / psd[i];"),
    ("d^2F/dt^2 term of the weight dropped", "c", "grad", "- 0.5 * Xr * Fdd / Fd - Xi", "- 0.0 * Xr * Fdd / Fd - Xi"),
    ("dFdot/dc_j without its factor j", "c", "grad", "double dfdot = (j == 0) ? 0.0 : j * xp[j - 1];",
     "double dfdot = (j == 0) ? 0.0 : xp[j - 1];"),
    ("partner amplitude gradient sign", "c", "grad", "ga[sc + 4 * k + q] += -sgn * a[12 + q]; }",
     "ga[sc + 4 * k + q] += sgn * a[12 + q]; }"),
    ("negative-branch residual weight", "c", "grad", "else { Wr = 0.5 * (Gb[0] - Gb[3]); Wi = 0.5 * (Gb[1] + Gb[2]); }",
     "else { Wr = 0.5 * (Gb[0] + Gb[3]); Wi = 0.5 * (Gb[1] + Gb[2]); }"),
    ("Phi_r chain rule uses m", "c", "grad", "gcf[1 * sc + 4 * k + q] += (double)V->n * a[4 + q];",
     "gcf[1 * sc + 4 * k + q] += (double)V->m * a[4 + q];"),
    # inner product and mismatch (Eq. 12-13)
    ("inner product multiplies by the PSD", "py", "mismatch", "np.sum(np.conj(a) * b / psd)", "np.sum(np.conj(a) * b * psd)"),
    ("inner product without the conjugate", "py", "mismatch", "np.sum(np.conj(a) * b / psd)", "np.sum(a * b / psd)"),
    ("mismatch summed over the channels", "py", "mismatch", "return 1.0 - out / len(a_pair)", "return 1.0 - out"),
]

# the pins run on each mutant: (group, name, call)
BATTERY = [
    ("spa", "ylm l=2", lambda O: YLM.test_l2_closed_forms(O, 0.7, 1.1)),
    ("spa", "ylm l=3", lambda O: YLM.test_l3_closed_forms(O, 3)),
    ("spa", "spline vs scipy", lambda O: SPL.test_matches_scipy_not_a_knot(O, 17)),
    ("spa", "partners explicit", lambda O: INV.test_conj_partners_explicit(O)),
    ("spa", "linear chirp", lambda O: CF.test_linear_chirp(O)),
    ("spa", "linear chirp from two series", lambda O: CF.test_linear_chirp_from_two_series(O)),
    ("spa", "quadratic turnover", lambda O: CF.test_quadratic_turning_point(O, False)),
    ("spa", "quadratic turnover mid-segment", lambda O: CF.test_quadratic_turning_point(O, True)),
    ("spa", "DFT of TD, 4 voices", lambda O: FFT.test_spa_matches_dft_of_time_domain(O, [(2, 2, 0), (3, 3, 2), (2, 1, -3), (3, 1, 1)])),
    ("spa", "DFT of TD, turnover voice", lambda O: FFT.test_turning_point_voice_matches_dft_away_from_turnover(O)),
    ("ext", "factor vs scipy kv", lambda O: [EXT.test_factor_matches_library_bessel(O, x) for x in (1.0, -3e-18, 2.5e-15)]),
    ("ext", "factor limits", lambda O: EXT.test_factor_limits(O)),
    ("ext", "cubic-phase voice is Airy", lambda O: EXT.test_cubic_phase_voice_is_airy(O)),
    ("select", "exact characterisation", lambda O: [SEL.test_matches_exact_characterisation(O, s) for s in range(6)]),
    ("select", "limits and monotone", lambda O: SEL.test_limits_and_monotone(O)),
    ("select", "union over knots", lambda O: SEL.test_union_over_knots(O)),
    ("window", "three-term form on the DFT", lambda O: WIN.test_three_term_form_is_exact_on_dft(O)),
    ("window", "FD definition", lambda O: WIN.test_hann_fd_definition(O)),
    ("td", "linear chirp samples", lambda O: TD.test_linear_chirp_samples(O)),
    ("grad", "likelihood definition", lambda O: GRAD.test_loglike_definition(O)),
    ("grad", "Euler identity", lambda O: GRAD.test_euler_identity_amplitudes(O)),
    ("grad", "phase offset identities", lambda O: [GRAD.test_phase_offset_identity(O, x) for x in ("phi_phi", "phi_r")]),
    ("mismatch", "inner product", lambda O: MM.test_inner_is_4_df_re_sum_over_psd(O)),
    ("mismatch", "phase rotation", lambda O: [MM.test_phase_rotation(O, x) for x in (0.4, 2.0)]),
    ("mismatch", "PSD weighting", lambda O: MM.test_psd_weighting(O, 4.0)),
    ("mismatch", "identical signals", lambda O: MM.test_identical_and_scaled(O)),
    ("grad", "central differences", lambda O: [GRAD.test_central_differences(O, x, h) for x, h in
                                               (("phi_phi", 3e-5), ("phi_r", 3e-5), ("omega_phi", 1e-8),
                                                ("omega_r", 1e-8), ("amp", 1e-4))]),
]


def _oracle_from(c_text, py_text, tmp):
    """A separate copy of the oracle module, from py_text, bound to a library built from c_text."""
    os.makedirs(tmp, exist_ok=True)
    src, lib, mod_path = os.path.join(tmp, "oracle.c"), os.path.join(tmp, "liboracle.so"), os.path.join(tmp, "oracle.py")
    with open(src, "w") as f:
        f.write(c_text)
    with open(mod_path, "w") as f:
        f.write(py_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                           "-shared", "-o", lib, src, "-lm"])
    spec = importlib.util.spec_from_file_location("oracle_copy_%d" % abs(hash(tmp)), mod_path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.BUILD, mod.LIB, mod.SRC = tmp, lib, src
    return mod


def _first_failing_pin(O, group=None):
    """The first pin that fails, the mutant's own group first (only to finish sooner)."""
    order = sorted(BATTERY, key=lambda b: b[0] != group)
    for _, name, pin in order:
        try:
            pin(O)
        except AssertionError:
            return name
    return None


@pytest.fixture(scope="module")
def sources():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    pytest.importorskip("scipy")
    with open(SRC_C) as f, open(SRC_PY) as g:
        return {"c": f.read(), "py": g.read()}


def test_unmodified_oracle_passes_the_battery(sources, tmp_path):
    assert _first_failing_pin(_oracle_from(sources["c"], sources["py"], str(tmp_path / "orig"))) is None


@pytest.mark.parametrize("name,where,group,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(sources, tmp_path, name, where, group, old, new):
    assert sources[where].count(old) == 1, "mutation site not found (or not unique): %s" % name
    text = dict(sources)
    text[where] = sources[where].replace(old, new)
    caught = _first_failing_pin(_oracle_from(text["c"], text["py"], str(tmp_path / "m")), group)
    assert caught is not None, "no pin catches: %s" % name
