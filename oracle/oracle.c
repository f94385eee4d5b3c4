/*
 * CPU oracle for the frequency-domain stationary-phase (SPA) mode sum of
 * "Fast and Fourier: EMRI waveforms in the frequency domain" (arXiv 2307.12585).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * reference that the CUDA path is checked against.  Only tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Arithmetic: IEEE binary64 throughout.  The only extension is double-double
 * (error-free transformations of Dekker 1971 / Knuth TAOCP vol. 2) for the
 * phase 2 pi f t - Phi(t), whose terms reach 1e7 rad while the result is
 * needed to ~1e-12 rad; build with -ffp-contract=off so that no implicit FMA
 * changes roundings.
 *
 * What is computed (one waveform):
 *  1. Every knot series (Phi_phi, Phi_r, Omega_phi, Omega_r, Re A, Im A of
 *     each voice) is an independent not-a-knot cubic spline in t (Sec. 2.1:
 *     amplitudes, phases and frequencies are interpolated with not-a-knot
 *     cubic splines on the sparse trajectory).  Solved densely: the K x K
 *     system for the knot second derivatives by Gaussian elimination with
 *     partial pivoting (one LU, one solve per series).
 *  2. Voices (Eq. 2): mode (l,m,n) gives H_V(t) = prefactor A(t) Y_lm(theta,phi)
 *     and Phi_V = m Phi_phi + n Phi_r (Eq. 1 with k = 0, Schwarzschild);
 *     with conj_partners each m >= 0 mode also gives the voice (l,-m,-n) with
 *     amplitude (-1)^l conj(A) (Schwarzschild reflection symmetry).
 *  3. Voice frequency F_V(t) = (m Omega_phi + n Omega_r)/(2 pi) (Sec. 2.2);
 *     per spline segment it is the cubic of Eq. 6.
 *  4. For a signed frequency g, every real root t_j of F_V(t) = g in the
 *     trajectory contributes H_V(t_j) exp(i[2 pi g t_j - Phi_V(t_j)
 *     - sgn(Fdot_j) pi/4]) / sqrt|Fdot_j|: the Fourier integral of Eq. 3
 *     with the phase expanded to second order (Eq. 4) and the Fresnel
 *     integral done exactly; it is the standard-SPA limit of Eq. 10 (Fddot
 *     -> 0), summed over the N roots of Eq. 9.  Roots are bracketed on the
 *     monotone pieces of each segment (split where Fdot = 0, at most one
 *     turnover per segment in practice, Sec. 2.2) and found by bisection
 *     to the last bit.  A root with Fdot == 0 exactly contributes 0.
 *  4'. Extended form (spa_form = 1): each root instead contributes
 *     H_V(t_j) exp(i[2 pi g t_j - Phi_V(t_j)]) G(Fdot_j, Fddot_j), where G is
 *     the Fourier integral of the phase expanded to third order (Eq. 7-10)
 *     in terms of K_{1/3}; see ext_factor() for the reading of its sign.
 *  5. Output at f > 0 (h = h+ - i hx, Eq. 1; Fourier sign of Eq. 3):
 *     h+(f) = [H(f) + conj H(-f)]/2,  hx(f) = i [H(f) - conj H(-f)]/2.
 *
 * Ownership of a frequency by a monotone piece [tau_a, tau_b) with end
 * frequencies Fa, Fb: increasing pieces own [Fa, Fb), decreasing pieces own
 * (Fb, Fa].  Knot frequencies are always (m*Om_phi_k + n*Om_r_k)/(2 pi)
 * evaluated in that order, so every frequency crossing of the whole track is
 * counted exactly once.  Interior turnover frequencies come from the cubic.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_TWO_PI_HI 6.283185307179586232
#define OR_TWO_PI_LO 2.4492935982947064e-16
#define OR_QPI_HI 0.7853981633974483096
#define OR_QPI_LO 3.061616997868383e-17
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* double-double helpers (Dekker 1971; Knuth TAOCP 4.2.2)               */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd_t;

static dd_t two_sum(double a, double b) {
  dd_t r; double s = a + b; double bb = s - a;
  r.hi = s; r.lo = (a - (s - bb)) + (b - bb); return r;
}
static dd_t two_prod(double a, double b) {
  dd_t r; r.hi = a * b; r.lo = fma(a, b, -r.hi); return r;
}
static dd_t dd_norm(double hi, double lo) { return two_sum(hi, lo); }
static dd_t dd_add(dd_t a, dd_t b) {
  dd_t s = two_sum(a.hi, b.hi);
  double lo = s.lo + a.lo + b.lo;
  return dd_norm(s.hi, lo);
}
static dd_t dd_add_d(dd_t a, double b) {
  dd_t s = two_sum(a.hi, b);
  return dd_norm(s.hi, s.lo + a.lo);
}
static dd_t dd_neg(dd_t a) { dd_t r; r.hi = -a.hi; r.lo = -a.lo; return r; }
static dd_t dd_mul_d(dd_t a, double b) {
  dd_t p = two_prod(a.hi, b);
  return dd_norm(p.hi, p.lo + a.lo * b);
}
static dd_t dd_mul(dd_t a, dd_t b) {
  dd_t p = two_prod(a.hi, b.hi);
  return dd_norm(p.hi, p.lo + (a.hi * b.lo + a.lo * b.hi));
}
static dd_t dd_from(double a) { dd_t r; r.hi = a; r.lo = 0.0; return r; }

/* ------------------------------------------------------------------ */
/* 1. not-a-knot cubic spline, dense Gaussian elimination               */
/* ------------------------------------------------------------------ */
/* System for the knot second derivatives M_0..M_{K-1}:
 *   rows 1..K-2 (C2 continuity):
 *     h_{k-1} M_{k-1} + 2 (h_{k-1}+h_k) M_k + h_k M_{k+1}
 *        = 6 [ (y_{k+1}-y_k)/h_k - (y_k-y_{k-1})/h_{k-1} ]
 *   row 0 (not-a-knot at t_1, third derivative continuous):
 *     (M_1 - M_0)/h_0 - (M_2 - M_1)/h_1 = 0, times h_0 h_1
 *   row K-1 (not-a-knot at t_{K-2}):
 *     (M_{K-2} - M_{K-3})/h_{K-3} - (M_{K-1} - M_{K-2})/h_{K-2} = 0, times h_{K-3} h_{K-2}
 * Segment k, tau = t - t_k in [0, h_k]:
 *   S = y_k + b tau + c tau^2 + d tau^3,
 *   b = (y_{k+1}-y_k)/h_k - h_k (2 M_k + M_{k+1})/6, c = M_k/2,
 *   d = (M_{k+1} - M_k)/(6 h_k).                                         */
typedef struct { int K; double* LU; int* piv; const double* t; } spl_sys_t;

static int spl_factor(spl_sys_t* S, int K, const double* t) {
  S->K = K; S->t = t;
  S->LU = (double*)calloc((size_t)K * K, sizeof(double));
  S->piv = (int*)malloc(sizeof(int) * K);
  if (!S->LU || !S->piv) return -1;
  double* A = S->LU;
#define AA(i, j) A[(size_t)(i) * K + (j)]
  for (int k = 1; k <= K - 2; k++) {
    double h0 = t[k] - t[k - 1], h1 = t[k + 1] - t[k];
    AA(k, k - 1) = h0; AA(k, k) = 2.0 * (h0 + h1); AA(k, k + 1) = h1;
  }
  /* not-a-knot rows multiplied through by h_0 h_1 (resp. h_{K-3} h_{K-2}) so
   * that their entries have the scale of the interior rows */
  { double h0 = t[1] - t[0], h1 = t[2] - t[1];
    AA(0, 0) = -h1; AA(0, 1) = h0 + h1; AA(0, 2) = -h0; }
  { double ha = t[K - 2] - t[K - 3], hb = t[K - 1] - t[K - 2];
    AA(K - 1, K - 3) = -hb; AA(K - 1, K - 2) = ha + hb; AA(K - 1, K - 1) = -ha; }
  /* LU with partial pivoting (row exchanges recorded in piv). */
  for (int c = 0; c < K; c++) {
    int p = c; double best = fabs(AA(c, c));
    for (int r = c + 1; r < K; r++) if (fabs(AA(r, c)) > best) { best = fabs(AA(r, c)); p = r; }
    S->piv[c] = p;
    if (best == 0.0) return -2;
    if (p != c) for (int j = 0; j < K; j++) { double tmp = AA(c, j); AA(c, j) = AA(p, j); AA(p, j) = tmp; }
    for (int r = c + 1; r < K; r++) {
      double f = AA(r, c) / AA(c, c);
      AA(r, c) = f;
      for (int j = c + 1; j < K; j++) AA(r, j) -= f * AA(c, j);
    }
  }
#undef AA
  return 0;
}

static void spl_free(spl_sys_t* S) { free(S->LU); free(S->piv); }

/* Solve for M given y, then write coef[k*4 + {0,1,2,3}] = (a, b, c, d). */
static void spl_coef(const spl_sys_t* S, const double* y, double* coef, double* work) {
  int K = S->K; const double* t = S->t; const double* A = S->LU;
  double* M = work;
  for (int k = 0; k < K; k++) M[k] = 0.0;
  for (int k = 1; k <= K - 2; k++) {
    double h0 = t[k] - t[k - 1], h1 = t[k + 1] - t[k];
    M[k] = 6.0 * ((y[k + 1] - y[k]) / h1 - (y[k] - y[k - 1]) / h0);
  }
  /* the factorization swapped whole rows (multipliers included), so apply
   * every recorded interchange to the right-hand side first, in order */
  for (int c = 0; c < K; c++) { int p = S->piv[c]; if (p != c) { double tmp = M[c]; M[c] = M[p]; M[p] = tmp; } }
  for (int c = 0; c < K; c++)
    for (int r = c + 1; r < K; r++) M[r] -= A[(size_t)r * K + c] * M[c];
  for (int r = K - 1; r >= 0; r--) {
    double s = M[r];
    for (int j = r + 1; j < K; j++) s -= A[(size_t)r * K + j] * M[j];
    M[r] = s / A[(size_t)r * K + r];
  }
  for (int k = 0; k < K - 1; k++) {
    double h = t[k + 1] - t[k];
    coef[4 * k + 0] = y[k];
    coef[4 * k + 1] = (y[k + 1] - y[k]) / h - h * (2.0 * M[k] + M[k + 1]) / 6.0;
    coef[4 * k + 2] = M[k] / 2.0;
    coef[4 * k + 3] = (M[k + 1] - M[k]) / (6.0 * h);
  }
}

/* Public: spline coefficients of one series; returns 0 on success. */
int oracle_spline_coef(int K, const double* t, const double* y, double* coef) {
  if (K < 4) return -1;
  spl_sys_t S; if (spl_factor(&S, K, t)) { spl_free(&S); return -2; }
  double* w = (double*)malloc(sizeof(double) * K);
  spl_coef(&S, y, coef, w);
  free(w); spl_free(&S); return 0;
}

/* ------------------------------------------------------------------ */
/* spin-weighted spherical harmonic, Goldberg et al. 1967 sum formula   */
/* sY_lm = (-1)^m sqrt[(l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)]
 *         sin^{2l}(theta/2) sum_r C(l-s,r) C(l+s,r+s-m) (-1)^{l-r-s}
 *         e^{i m phi} cot^{2r+s-m}(theta/2)                               */
/* ------------------------------------------------------------------ */
static double fact(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }
static double binom(int n, int k) { if (k < 0 || k > n) return 0.0; return fact(n) / (fact(k) * fact(n - k)); }

void oracle_swsh(int s, int l, int m, double theta, double phi, double* out) {
  double pre = ((m & 1) ? -1.0 : 1.0) *
               sqrt(fact(l + m) * fact(l - m) * (2.0 * l + 1.0) / (4.0 * OR_PI * fact(l + s) * fact(l - s)));
  double sh = sin(0.5 * theta), ch = cos(0.5 * theta);
  double sum = 0.0;
  for (int r = 0; r <= l - s; r++) {
    double c = binom(l - s, r) * binom(l + s, r + s - m);
    if (c == 0.0) continue;
    int k = 2 * r + s - m;                 /* power of cot(theta/2), >= 0 for nonzero terms */
    double term = c * (((l - r - s) & 1) ? -1.0 : 1.0) * pow(sh, 2 * l - k) * pow(ch, k);
    sum += term;
  }
  out[0] = pre * sum * cos(m * phi);
  out[1] = pre * sum * sin(m * phi);
}

/* ------------------------------------------------------------------ */
/* 2-5. the SPA sum                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  int l, m, n;            /* voice mode numbers (m may be negative for partners) */
  double Y[2];            /* -2Y_lm(theta, phi) */
  const double* are;      /* amplitude spline coef, Re, [K-1][4] */
  const double* aim;      /* amplitude spline coef, Im */
} voice_t;

typedef struct {
  int voice, seg;
  double ta, tb;          /* monotone piece [ta, tb] inside the segment */
  int dir;                /* +1 increasing, -1 decreasing */
  long long lo[2], hi[2]; /* owned bin ranges for g = +f (index 0) and g = -f (index 1) */
} piece_t;

static long long lower_bound(const double* f, long long nf, double x) {
  long long a = 0, b = nf; while (a < b) { long long c = a + (b - a) / 2; if (f[c] < x) a = c + 1; else b = c; } return a;
}
static long long upper_bound(const double* f, long long nf, double x) {
  long long a = 0, b = nf; while (a < b) { long long c = a + (b - a) / 2; if (f[c] <= x) a = c + 1; else b = c; } return a;
}

typedef struct {
  int K; const double* t;
  const double *cPp, *cPr, *cOp, *cOr;   /* fundamental spline coefs [K-1][4] */
  const double *Op, *Or;                 /* knot values of Omega_phi, Omega_r */
  double prefactor;
} traj_t;

/* voice frequency at knot k: the ownership rule's exact expression */
static double knot_freq(const traj_t* T, int mv, int nv, int k) {
  return ((double)mv * T->Op[k] + (double)nv * T->Or[k]) / OR_TWO_PI_HI;
}

/* cubic coefficients of F_V in segment k: (F_k, B, C, D) */
static void voice_fcubic(const traj_t* T, int mv, int nv, int k, double* c4) {
  c4[0] = knot_freq(T, mv, nv, k);
  for (int j = 1; j < 4; j++)
    c4[j] = ((double)mv * T->cOp[4 * k + j] + (double)nv * T->cOr[4 * k + j]) / OR_TWO_PI_HI;
}
static double cubic(const double* c, double x) { return c[0] + x * (c[1] + x * (c[2] + x * c[3])); }
static double dcubic(const double* c, double x) { return c[1] + x * (2.0 * c[2] + x * 3.0 * c[3]); }

/* roots of c1 + 2 c2 x + 3 c3 x^2 in the open interval (0, h), ascending; returns count */
static int turnovers(const double* c, double h, double* r) {
  double a = 3.0 * c[3], b = 2.0 * c[2], cc = c[1];
  double x[2]; int nx = 0;
  if (a == 0.0) {
    if (b != 0.0) x[nx++] = -cc / b;
  } else {
    double disc = b * b - 4.0 * a * cc;
    if (disc >= 0.0) {
      double sq = sqrt(disc);
      double q = -0.5 * (b + (b >= 0.0 ? sq : -sq));
      if (q != 0.0) { x[nx++] = q / a; x[nx++] = cc / q; }
      else x[nx++] = 0.0;          /* b = 0 and disc = 0: double root at 0 */
    }
  }
  int n = 0;
  for (int i = 0; i < nx; i++) if (x[i] > 0.0 && x[i] < h) r[n++] = x[i];
  if (n == 2 && r[1] < r[0]) { double tmp = r[0]; r[0] = r[1]; r[1] = tmp; }
  if (n == 2 && r[1] == r[0]) n = 1;
  return n;
}

/* bisection for F(x) = g on [a, b], F monotone with direction dir */
static double bisect(const double* c, double g, double a, double b, int dir) {
  double lo = a, hi = b;
  for (int it = 0; it < 400; it++) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    double v = cubic(c, mid) - g;
    if (dir * v < 0.0) lo = mid; else hi = mid;
  }
  double vl = fabs(cubic(c, lo) - g), vh = fabs(cubic(c, hi) - g);
  return (vh < vl) ? hi : lo;
}

/* Phi spline value in double-double at tau in segment k */
static dd_t dd_spline(const double* c4, double x) {
  dd_t r = dd_from(c4[3]);
  r = dd_add_d(dd_mul_d(r, x), c4[2]);
  r = dd_add_d(dd_mul_d(r, x), c4[1]);
  r = dd_add_d(dd_mul_d(r, x), c4[0]);
  return r;
}

/* ------------------------------------------------------------------ */
/* Extended SPA factor (Sec. 2.2, Eq. 7-10)                             */
/* ------------------------------------------------------------------ */
/*
 * E(X) = e^z K_{1/3}(z) at z = -i X, X real and non-zero, straight from an
 * integral definition of K_nu (DLMF 10.32.8):
 *   K_nu(z) = sqrt(pi) (z/2)^nu / Gamma(nu + 1/2) int_1^inf e^{-z t} (t^2 - 1)^{nu - 1/2} dt.
 * For X > 0 the path t = 1 + i s (s >= 0) turns the oscillating integrand
 * into a decaying one; with s = e^v this gives
 *   E(X) = sqrt(pi)/Gamma(5/6) (X/2)^{1/3} e^{i pi/4}
 *          int_R exp(5v/6 - X e^v) (2 + i e^v)^{-1/6} dv,
 * an analytic integrand that decays exponentially on both sides, so the
 * trapezoid rule on a fixed step converges geometrically.  For X < 0,
 * E(X) = conj E(-X) (K_nu(conj z) = conj K_nu(z) for real nu).
 */
static double complex ext_E(double X) {
  const double ax = fabs(X);
  const double hv = 0.1;
  const double v0 = log(1e-20 / ax), v1 = log(60.0 / ax);
  const long long nstep = (long long)ceil((v1 - v0) / hv);
  double complex sum = 0.0;
  for (long long i = 0; i <= nstep; i++) {
    const double v = v0 + hv * (double)i;
    const double ev = exp(v);
    sum += exp(5.0 * v / 6.0 - ax * ev) * cpow(2.0 + I * ev, -1.0 / 6.0);
  }
  sum *= hv;
  const double complex e = sqrt(OR_PI) / tgamma(5.0 / 6.0) * cbrt(0.5 * ax) * cexp(I * (OR_PI / 4.0)) * sum;
  return X > 0.0 ? e : conj(e);
}

/*
 * G(Fdot, Fddot): the time integral of Eq. 8 for one root, in the closed form
 * of Eq. 10, int exp(-i pi [Fdot t^2 + Fddot t^3/3]) dt ->
 *   -(2/sqrt 3) (i Fdot/|Fddot|) e^z K_{1/3}(z),   z = -2 pi i Fdot^3 / (3 Fddot^2),
 * with the principal branch of K_{1/3}.  The overall sign is the reading
 * taken here: Eq. 10 as printed tends to -exp(-i sgn(Fdot) pi/4)/sqrt|Fdot|
 * when Fddot -> 0, the negative of the Fresnel value that Eq. 10 must reduce
 * to, so the factor is negated.  With that sign the two roots of a pure
 * cubic phase add up to its exact (Airy-function) Fourier transform.
 *   Fddot == 0: the Fresnel value exp(-i sgn(Fdot) pi/4)/sqrt|Fdot|.
 *   Fdot == 0 (a double root at a turnover): the limit of the two-root sum,
 *     2 pi (pi |Fddot|)^{-1/3} Ai(0) = 2 pi^{2/3} / (3^{2/3} Gamma(2/3)) |Fddot|^{-1/3}.
 *   both zero: 0.
 */
static double complex ext_factor(double Fd, double Fdd) {
  if (Fdd == 0.0) {
    if (Fd == 0.0) return 0.0;
    return cexp(-I * (Fd > 0.0 ? 1.0 : -1.0) * (OR_PI / 4.0)) / sqrt(fabs(Fd));
  }
  if (Fd == 0.0) return 2.0 * pow(OR_PI, 2.0 / 3.0) / (pow(3.0, 2.0 / 3.0) * tgamma(2.0 / 3.0)) / cbrt(fabs(Fdd));
  const double X = 2.0 * OR_PI * Fd * Fd * Fd / (3.0 * Fdd * Fdd);
  return -(2.0 / sqrt(3.0)) * (I * Fd / fabs(Fdd)) * ext_E(X);
}

/* exported for tests: G(Fdot, Fddot) as (re, im) */
void oracle_ext_factor(long long n, const double* Fd, const double* Fdd, double* out) {
  for (long long i = 0; i < n; i++) {
    const double complex g = ext_factor(Fd[i], Fdd[i]);
    out[2 * i] = creal(g);
    out[2 * i + 1] = cimag(g);
  }
}

/* contribution of one root: adds H_V e^{i psi}/sqrt|Fdot| (standard form) or
 * H_V e^{i psi0} G(Fdot, Fddot) (extended form) to acc[0..1] */
static int contrib(const traj_t* T, const voice_t* V, int k, const double* fc, double g, double x, int ext,
                   double* acc) {
  double Fd = dcubic(fc, x);
  double complex G = 1.0;
  if (ext) {
    const double Fdd = 2.0 * fc[2] + 6.0 * fc[3] * x;
    G = ext_factor(Fd, Fdd);
    if (G == 0.0) return 1;
  } else if (Fd == 0.0) {
    return 1;
  }
  /* phase psi = 2 pi g (t_k + x) - Phi_V(t_k + x) - sgn(Fdot) pi / 4 in double-double */
  dd_t tt = two_sum(T->t[k], x);
  dd_t gt = dd_mul_d(tt, g);
  dd_t twopi; twopi.hi = OR_TWO_PI_HI; twopi.lo = OR_TWO_PI_LO;
  dd_t wgt = dd_mul(gt, twopi);
  dd_t Pp = dd_spline(T->cPp + 4 * k, x), Pr = dd_spline(T->cPr + 4 * k, x);
  dd_t PV = dd_add(dd_mul_d(Pp, (double)V->m), dd_mul_d(Pr, (double)V->n));
  dd_t psi = dd_add(wgt, dd_neg(PV));
  dd_t qpi; qpi.hi = OR_QPI_HI; qpi.lo = OR_QPI_LO;
  if (!ext) psi = dd_add(psi, Fd > 0.0 ? dd_neg(qpi) : qpi);
  /* reduce modulo 2 pi */
  double kk = nearbyint(psi.hi / OR_TWO_PI_HI);
  psi = dd_add(psi, dd_neg(dd_mul_d(twopi, kk)));
  double cs = cos(psi.hi) - psi.lo * sin(psi.hi);
  double sn = sin(psi.hi) + psi.lo * cos(psi.hi);
  /* H_V(t) = prefactor A(t) Y */
  double are = cubic(V->are + 4 * k, x), aim = cubic(V->aim + 4 * k, x);
  double hr = T->prefactor * (are * V->Y[0] - aim * V->Y[1]);
  double hi = T->prefactor * (are * V->Y[1] + aim * V->Y[0]);
  if (ext) {
    const double complex z = (hr + I * hi) * (cs + I * sn) * G;
    acc[0] += creal(z);
    acc[1] += cimag(z);
    return 0;
  }
  double w = 1.0 / sqrt(fabs(Fd));
  acc[0] += w * (hr * cs - hi * sn);
  acc[1] += w * (hr * sn + hi * cs);
  return 0;
}

/* Build the monotone pieces of every voice, with owned bin ranges. */
static piece_t* build_pieces(const traj_t* T, const voice_t* V, int nv, const double* freqs, long long nf, long long* npieces) {
  int K = T->K;
  size_t cap = (size_t)nv * (K - 1) * 3 + 1, np = 0;
  piece_t* P = (piece_t*)malloc(sizeof(piece_t) * cap);
  if (!P) return NULL;
  for (int v = 0; v < nv; v++) {
    for (int k = 0; k < K - 1; k++) {
      double fc[4]; voice_fcubic(T, V[v].m, V[v].n, k, fc);
      double h = T->t[k + 1] - T->t[k];
      double r[2]; int nr = turnovers(fc, h, r);
      double xs[4], Fs[4]; int nx = 0;
      xs[nx] = 0.0; Fs[nx++] = fc[0];
      for (int i = 0; i < nr; i++) { xs[nx] = r[i]; Fs[nx++] = cubic(fc, r[i]); }
      xs[nx] = h; Fs[nx++] = knot_freq(T, V[v].m, V[v].n, k + 1);
      for (int i = 0; i + 1 < nx; i++) {
        double Fa = Fs[i], Fb = Fs[i + 1];
        if (Fa == Fb) continue;
        piece_t p; p.voice = v; p.seg = k; p.ta = xs[i]; p.tb = xs[i + 1];
        if (Fa < Fb) {
          p.dir = 1;
          p.lo[0] = lower_bound(freqs, nf, Fa);  p.hi[0] = lower_bound(freqs, nf, Fb);   /* Fa <= f < Fb */
          p.lo[1] = upper_bound(freqs, nf, -Fb); p.hi[1] = upper_bound(freqs, nf, -Fa);  /* Fa <= -f < Fb */
        } else {
          p.dir = -1;
          p.lo[0] = upper_bound(freqs, nf, Fb);  p.hi[0] = upper_bound(freqs, nf, Fa);   /* Fb < f <= Fa */
          p.lo[1] = lower_bound(freqs, nf, -Fa); p.hi[1] = lower_bound(freqs, nf, -Fb);  /* Fb < -f <= Fa */
        }
        if (p.hi[0] > p.lo[0] || p.hi[1] > p.lo[1]) P[np++] = p;
      }
    }
  }
  *npieces = (long long)np;
  return P;
}

/* ------------------------------------------------------------------ */
/* shared set-up: splines, voices, monotone pieces                     */
/* ------------------------------------------------------------------ */
typedef struct {
  int K, nm, nv, conj, ext;
  spl_sys_t S;
  double* cf;          /* fundamental spline coef: Phi_phi, Phi_r, Om_phi, Om_r, each [K-1][4] */
  double* ac;          /* voice amplitude coef: per voice Re [K-1][4] then Im [K-1][4] */
  voice_t* V;
  int* vmode;          /* input mode of each voice */
  int* vpart;          /* 0: the listed mode, 1: its conjugate partner */
  traj_t T;
  piece_t* P;
  long long np;
} ctx_t;

static void ctx_free(ctx_t* c) {
  free(c->cf); free(c->ac); free(c->V); free(c->vmode); free(c->vpart); free(c->P); spl_free(&c->S);
}

static int ctx_init(ctx_t* c, int K, const double* t, const double* phi_phi, const double* phi_r,
                    const double* omega_phi, const double* omega_r, int nm, const int* l, const int* m,
                    const int* n, const double* amp, double theta, double phi, double prefactor,
                    int conj_partners, long long nf, const double* freqs) {
  memset(c, 0, sizeof(*c));
  if (K < 4 || nm < 0 || nf < 0) return -1;
  for (int k = 0; k + 1 < K; k++) if (!(t[k + 1] > t[k])) return -2;
  for (long long i = 0; i < nf; i++) if (!(freqs[i] > 0.0) || (i && !(freqs[i] > freqs[i - 1]))) return -3;
  for (int j = 0; j < nm; j++) if (l[j] < 2 || abs(m[j]) > l[j] || (conj_partners && m[j] < 0)) return -4;
  c->K = K; c->nm = nm; c->conj = conj_partners;
  if (spl_factor(&c->S, K, t)) { spl_free(&c->S); return -5; }
  double* work = (double*)malloc(sizeof(double) * K);
  double* y = (double*)malloc(sizeof(double) * K);
  size_t sc = (size_t)(K - 1) * 4;
  c->cf = (double*)malloc(sizeof(double) * sc * 4);
  int nv = conj_partners ? 2 * nm : nm;
  c->nv = nv;
  c->ac = (double*)malloc(sizeof(double) * sc * 2 * (size_t)(nv > 0 ? nv : 1));
  c->V = (voice_t*)malloc(sizeof(voice_t) * (size_t)(nv > 0 ? nv : 1));
  c->vmode = (int*)malloc(sizeof(int) * (size_t)(nv > 0 ? nv : 1));
  c->vpart = (int*)malloc(sizeof(int) * (size_t)(nv > 0 ? nv : 1));
  traj_t* T = &c->T;
  T->K = K; T->t = t; T->Op = omega_phi; T->Or = omega_r; T->prefactor = prefactor;
  spl_coef(&c->S, phi_phi, c->cf + 0 * sc, work); spl_coef(&c->S, phi_r, c->cf + 1 * sc, work);
  spl_coef(&c->S, omega_phi, c->cf + 2 * sc, work); spl_coef(&c->S, omega_r, c->cf + 3 * sc, work);
  T->cPp = c->cf; T->cPr = c->cf + sc; T->cOp = c->cf + 2 * sc; T->cOr = c->cf + 3 * sc;
  int iv = 0;
  for (int j = 0; j < nm; j++) {
    for (int part = 0; part < (conj_partners ? 2 : 1); part++) {
      voice_t* v = &c->V[iv];
      v->l = l[j]; v->m = part ? -m[j] : m[j]; v->n = part ? -n[j] : n[j];
      double sgn = (l[j] & 1) ? -1.0 : 1.0;
      double* cre = c->ac + (size_t)iv * 2 * sc; double* cim = cre + sc;
      for (int k = 0; k < K; k++) y[k] = part ? sgn * amp[((size_t)j * K + k) * 2 + 0] : amp[((size_t)j * K + k) * 2 + 0];
      spl_coef(&c->S, y, cre, work);
      for (int k = 0; k < K; k++) y[k] = part ? -sgn * amp[((size_t)j * K + k) * 2 + 1] : amp[((size_t)j * K + k) * 2 + 1];
      spl_coef(&c->S, y, cim, work);
      v->are = cre; v->aim = cim;
      oracle_swsh(-2, v->l, v->m, theta, phi, v->Y);
      c->vmode[iv] = j; c->vpart[iv] = part;
      iv++;
    }
  }
  c->P = build_pieces(T, c->V, nv, freqs, nf, &c->np);
  free(work); free(y);
  return 0;
}

/* h+ and hx on the bins, plus counters */
static void ctx_forward(const ctx_t* c, long long nf, const double* freqs, double* hp, double* hc,
                        long long* stats, int nthreads) {
  double* Hpos = (double*)calloc((size_t)(nf > 0 ? nf : 1) * 2, sizeof(double));
  double* Hneg = (double*)calloc((size_t)(nf > 0 ? nf : 1) * 2, sizeof(double));
  long long nev = 0, nzero = 0, np = c->np;
  const piece_t* P = c->P;
  if (nthreads < 1) nthreads = 1;
  /* Parallel over contiguous chunks of bins; every bin sums its voices in
   * ascending voice order, so the result does not depend on nthreads. */
  long long nchunk = nthreads * 8LL;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(+ : nev, nzero)
  for (long long ch = 0; ch < nchunk; ch++) {
    long long b0 = nf * ch / nchunk, b1 = nf * (ch + 1) / nchunk;
    if (b0 >= b1) continue;
    for (long long ip = 0; ip < np; ip++) {
      const piece_t* p = &P[ip];
      const voice_t* v = &c->V[p->voice];
      double fc[4];
      int have_fc = 0;
      for (int sgn = 0; sgn < 2; sgn++) {
        long long lo = p->lo[sgn] > b0 ? p->lo[sgn] : b0;
        long long hi = p->hi[sgn] < b1 ? p->hi[sgn] : b1;
        if (lo >= hi) continue;
        if (!have_fc) { voice_fcubic(&c->T, v->m, v->n, p->seg, fc); have_fc = 1; }
        double* H = sgn ? Hneg : Hpos;
        for (long long b = lo; b < hi; b++) {
          double g = sgn ? -freqs[b] : freqs[b];
          double x = bisect(fc, g, p->ta, p->tb, p->dir);
          nzero += contrib(&c->T, v, p->seg, fc, g, x, c->ext, H + 2 * b);
          nev++;
        }
      }
    }
  }
  for (long long b = 0; b < nf; b++) {
    double pr = Hpos[2 * b], pi = Hpos[2 * b + 1], nr = Hneg[2 * b], ni = -Hneg[2 * b + 1]; /* conj H(-f) */
    hp[2 * b] = 0.5 * (pr + nr);   hp[2 * b + 1] = 0.5 * (pi + ni);
    /* hx = i/2 (H(f) - conj H(-f)) */
    hc[2 * b] = -0.5 * (pi - ni);  hc[2 * b + 1] = 0.5 * (pr - nr);
  }
  if (stats) { stats[0] = nev; stats[1] = nzero; stats[2] = np; }
  free(Hpos); free(Hneg);
}

/*
 * oracle_sum_modes: one waveform.
 *   K knots t[K]; phi_phi, phi_r, omega_phi, omega_r [K];
 *   nm modes l, m, n [nm]; amp [nm][K][2] (re, im interleaved);
 *   theta, phi, prefactor; conj_partners (0/1);
 *   spa_form: 0 standard SPA (item 4), 1 extended SPA (item 4');
 *   nf ascending freqs (> 0); outputs hp, hc [nf][2];
 *   stats[0] = contributions evaluated, stats[1] = roots with no contribution
 *   (Fdot == 0 in the standard form; Fdot == Fddot == 0 in the extended form),
 *   stats[2] = number of monotone pieces.
 * Returns 0 on success, < 0 on bad input.
 */
int oracle_sum_modes(int K, const double* t, const double* phi_phi, const double* phi_r,
                     const double* omega_phi, const double* omega_r,
                     int nm, const int* l, const int* m, const int* n, const double* amp,
                     double theta, double phi, double prefactor, int conj_partners, int spa_form,
                     long long nf, const double* freqs, double* hp, double* hc,
                     long long* stats, int nthreads) {
  ctx_t c;
  if (spa_form != 0 && spa_form != 1) return -1;
  int rc = ctx_init(&c, K, t, phi_phi, phi_r, omega_phi, omega_r, nm, l, m, n, amp, theta, phi, prefactor,
                    conj_partners, nf, freqs);
  if (rc) { ctx_free(&c); return rc; }
  c.ext = spa_form;
  ctx_forward(&c, nf, freqs, hp, hc, stats, nthreads);
  ctx_free(&c);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Whittle log-likelihood and its gradient                              */
/* ------------------------------------------------------------------ */
/*
 * L = -1/2 sum_alpha <d - h | d - h>_alpha with <a|b> = 4 Re sum_i a* b / S_i df
 * (Eq. 13-14).  The gradient is the plain chain rule: with
 * G_alpha = dL/dRe h_alpha + i dL/dIm h_alpha = 4 df (d - h)_alpha / S, a root
 * contribution C = prefactor A_V(tau) Y_V e^{i psi}/sqrt|Fdot| of voice V at
 * signed frequency g changes L by Re[W dC], W = (conj G+ + i conj Gx)/2 for
 * g = f and W = (G+ + i Gx)/2 for g = -f (from h+ = [H(f) + conj H(-f)]/2,
 * hx = i [H(f) - conj H(-f)]/2).  C depends on the segment's coefficients
 * directly and through the root tau of F(tau) = g, with
 * dtau = -(dF/dcoef) / Fdot (implicit differentiation), and through
 * dC/C = dA_V/A_V - dFdot/(2 Fdot) + i dpsi,
 * dpsi = (2 pi g - Phi_V'(tau)) dtau - dPhi_V.
 * Voice-coefficient gradients are mapped to the series (F_V = (m Om_phi +
 * n Om_r)/2pi, Phi_V = m Phi_phi + n Phi_r, partner amplitude (-1)^l conj A)
 * and then to knot values through the spline's Jacobian, built column by
 * column from the same dense solve.
 */
static double dd_to_d(dd_t a) { return a.hi + a.lo; }

int oracle_loglike_grad(int K, const double* t, const double* phi_phi, const double* phi_r,
                        const double* omega_phi, const double* omega_r,
                        int nm, const int* l, const int* m, const int* n, const double* amp,
                        double theta, double phi, double prefactor, int conj_partners,
                        long long nf, const double* freqs, const double* dplus, const double* dcross,
                        const double* psd, double df, double* loglike,
                        double* g_phi_phi, double* g_phi_r, double* g_omega_phi, double* g_omega_r,
                        double* g_amp, int nthreads) {
  ctx_t c;
  int rc = ctx_init(&c, K, t, phi_phi, phi_r, omega_phi, omega_r, nm, l, m, n, amp, theta, phi, prefactor,
                    conj_partners, nf, freqs);
  if (rc) { ctx_free(&c); return rc; }
  for (long long i = 0; i < nf; i++) if (!(psd[i] > 0.0)) { ctx_free(&c); return -6; }
  double* hp = (double*)malloc(sizeof(double) * 2 * (size_t)(nf > 0 ? nf : 1));
  double* hc = (double*)malloc(sizeof(double) * 2 * (size_t)(nf > 0 ? nf : 1));
  ctx_forward(&c, nf, freqs, hp, hc, NULL, nthreads);
  /* likelihood and G = 4 df r / S per channel */
  double* G = (double*)malloc(sizeof(double) * 4 * (size_t)(nf > 0 ? nf : 1));
  double L = 0.0;
  for (long long i = 0; i < nf; i++) {
    double rpr = dplus[2 * i] - hp[2 * i], rpi = dplus[2 * i + 1] - hp[2 * i + 1];
    double rcr = dcross[2 * i] - hc[2 * i], rci = dcross[2 * i + 1] - hc[2 * i + 1];
    L += -2.0 * df * (rpr * rpr + rpi * rpi + rcr * rcr + rci * rci) / psd[i];
    double s = 4.0 * df / psd[i];
    G[4 * i + 0] = s * rpr; G[4 * i + 1] = s * rpi; G[4 * i + 2] = s * rcr; G[4 * i + 3] = s * rci;
  }
  *loglike = L;
  int want = g_phi_phi || g_phi_r || g_omega_phi || g_omega_r || g_amp;
  if (!want) { free(hp); free(hc); free(G); ctx_free(&c); return 0; }

  const int nseg = K - 1, nv = c.nv;
  /* per (voice, segment): d/d of F cubic (4), Phi_V cubic (4), A_V cubic Re (4), Im (4) */
  double* gv = (double*)calloc((size_t)(nv > 0 ? nv : 1) * nseg * 16, sizeof(double));
  if (nthreads < 1) nthreads = 1;
  const piece_t* P = c.P;
  const traj_t* T = &c.T;
  /* pieces of one voice are contiguous: parallel over voices, no shared accumulators */
  long long* vstart = (long long*)malloc(sizeof(long long) * (size_t)(nv + 1));
  {
    long long ip = 0;
    for (int v = 0; v <= nv; v++) { while (ip < c.np && P[ip].voice < v) ip++; vstart[v] = ip; }
  }
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
  for (int v = 0; v < nv; v++) {
    const voice_t* V = &c.V[v];
    for (long long ip = vstart[v]; ip < vstart[v + 1]; ip++) {
      const piece_t* p = &P[ip];
      int k = p->seg;
      double fc[4]; voice_fcubic(T, V->m, V->n, k, fc);
      const double* cPp = T->cPp + 4 * k; const double* cPr = T->cPr + 4 * k;
      const double* are = V->are + 4 * k; const double* aim = V->aim + 4 * k;
      double* acc = gv + ((size_t)v * nseg + k) * 16;
      for (int sgn = 0; sgn < 2; sgn++) {
        for (long long b = p->lo[sgn]; b < p->hi[sgn]; b++) {
          double g = sgn ? -freqs[b] : freqs[b];
          double x = bisect(fc, g, p->ta, p->tb, p->dir);
          double Fd = dcubic(fc, x);
          if (Fd == 0.0) continue;
          double Fdd = 2.0 * fc[2] + 6.0 * fc[3] * x;
          /* phase, as in contrib() */
          dd_t tt = two_sum(T->t[k], x);
          dd_t gt = dd_mul_d(tt, g);
          dd_t twopi; twopi.hi = OR_TWO_PI_HI; twopi.lo = OR_TWO_PI_LO;
          dd_t wgt = dd_mul(gt, twopi);
          dd_t PV = dd_add(dd_mul_d(dd_spline(cPp, x), (double)V->m), dd_mul_d(dd_spline(cPr, x), (double)V->n));
          dd_t psi = dd_add(wgt, dd_neg(PV));
          dd_t qpi; qpi.hi = OR_QPI_HI; qpi.lo = OR_QPI_LO;
          psi = dd_add(psi, Fd > 0.0 ? dd_neg(qpi) : qpi);
          double kk = nearbyint(psi.hi / OR_TWO_PI_HI);
          psi = dd_add(psi, dd_neg(dd_mul_d(twopi, kk)));
          double cs = cos(psi.hi) - psi.lo * sin(psi.hi);
          double sn = sin(psi.hi) + psi.lo * cos(psi.hi);
          (void)dd_to_d;
          /* E = prefactor Y |Fdot|^(-1/2) e^{i psi};  C = A_V E */
          double w = 1.0 / sqrt(fabs(Fd));
          double Er = T->prefactor * w * (V->Y[0] * cs - V->Y[1] * sn);
          double Ei = T->prefactor * w * (V->Y[0] * sn + V->Y[1] * cs);
          double Ar = cubic(are, x), Ai = cubic(aim, x);
          double dAr = dcubic(are, x), dAi = dcubic(aim, x);
          const double* Gb = G + 4 * b;
          double Wr, Wi;
          if (!sgn) { Wr = 0.5 * (Gb[0] + Gb[3]); Wi = 0.5 * (-Gb[1] + Gb[2]); }   /* (conj G+ + i conj Gx)/2 */
          else { Wr = 0.5 * (Gb[0] - Gb[3]); Wi = 0.5 * (Gb[1] + Gb[2]); }         /* (G+ + i Gx)/2 */
          double WEr = Wr * Er - Wi * Ei, WEi = Wr * Ei + Wi * Er;
          double Xr = WEr * Ar - WEi * Ai, Xi = WEr * Ai + WEi * Ar;
          double dPV = (double)V->m * dcubic(cPp, x) + (double)V->n * dcubic(cPr, x);
          /* coefficient of dtau */
          double Tdt = (WEr * dAr - WEi * dAi) - 0.5 * Xr * Fdd / Fd - Xi * (OR_TWO_PI_HI * g - dPV);
          double xp[4] = {1.0, x, x * x, x * x * x};
          for (int j = 0; j < 4; j++) {
            double dtau = -xp[j] / Fd;                     /* dtau/dfc_j */
            double dfdot = (j == 0) ? 0.0 : j * xp[j - 1]; /* dFdot/dfc_j at fixed tau */
            acc[j] += Tdt * dtau - 0.5 * Xr * dfdot / Fd;   /* F cubic */
            acc[4 + j] += Xi * xp[j];                       /* Phi_V cubic */
            acc[8 + j] += WEr * xp[j];                      /* Re A_V */
            acc[12 + j] += -WEi * xp[j];                    /* Im A_V */
          }
        }
      }
    }
  }
  /* voice coefficients -> series coefficients */
  size_t sc = (size_t)nseg * 4;
  double* gcf = (double*)calloc(sc * 4, sizeof(double));       /* Phi_phi, Phi_r, Om_phi, Om_r */
  double* gca = (double*)calloc(sc * 2 * (size_t)(nm > 0 ? nm : 1), sizeof(double));  /* per mode Re, Im */
  for (int v = 0; v < nv; v++) {
    const voice_t* V = &c.V[v];
    int j = c.vmode[v], part = c.vpart[v];
    double sgn = (V->l & 1) ? -1.0 : 1.0;
    for (int k = 0; k < nseg; k++) {
      const double* a = gv + ((size_t)v * nseg + k) * 16;
      for (int q = 0; q < 4; q++) {
        gcf[0 * sc + 4 * k + q] += (double)V->m * a[4 + q];
        gcf[1 * sc + 4 * k + q] += (double)V->n * a[4 + q];
        gcf[2 * sc + 4 * k + q] += (double)V->m / OR_TWO_PI_HI * a[q];
        gcf[3 * sc + 4 * k + q] += (double)V->n / OR_TWO_PI_HI * a[q];
        double* ga = gca + (size_t)j * 2 * sc;
        if (!part) { ga[4 * k + q] += a[8 + q]; ga[sc + 4 * k + q] += a[12 + q]; }
        else { ga[4 * k + q] += sgn * a[8 + q]; ga[sc + 4 * k + q] += -sgn * a[12 + q]; }
      }
    }
  }
  /* series coefficients -> knot values through the spline Jacobian J[i] = coef(e_i) */
  double* J = (double*)malloc(sizeof(double) * sc * (size_t)K);
  {
    double* e = (double*)calloc((size_t)K, sizeof(double));
    double* work = (double*)malloc(sizeof(double) * K);
    for (int i = 0; i < K; i++) { e[i] = 1.0; spl_coef(&c.S, e, J + (size_t)i * sc, work); e[i] = 0.0; }
    free(e); free(work);
  }
  double* outs[4] = {g_phi_phi, g_phi_r, g_omega_phi, g_omega_r};
  for (int q = 0; q < 4; q++) {
    if (!outs[q]) continue;
    for (int i = 0; i < K; i++) {
      double s = 0.0;
      for (size_t r = 0; r < sc; r++) s += J[(size_t)i * sc + r] * gcf[q * sc + r];
      outs[q][i] = s;
    }
  }
  if (g_amp) {
    for (int j = 0; j < nm; j++)
      for (int part = 0; part < 2; part++)
        for (int i = 0; i < K; i++) {
          double s = 0.0;
          const double* ga = gca + (size_t)j * 2 * sc + part * sc;
          for (size_t r = 0; r < sc; r++) s += J[(size_t)i * sc + r] * ga[r];
          g_amp[((size_t)j * K + i) * 2 + part] = s;
        }
  }
  free(J); free(gcf); free(gca); free(vstart); free(gv); free(hp); free(hc); free(G); ctx_free(&c);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Mode selection (Sec. 2.1)                                             */
/* ------------------------------------------------------------------ */
/*
 * At each knot t_k every mode's power is P_j = |A_j(t_k)|^2 = re^2 + im^2.
 * The modes are ordered by decreasing power (equal powers: increasing mode
 * index) and their cumulative sums S_1, S_2, ... taken in that order, one
 * FP64 addition at a time; the total is the last of them.  Walking down the
 * ordered list, a mode still contributes while the power before it is below
 * the fraction 1 - eps of the total: mode (i) is kept at t_k when
 * S_{i-1} < (1 - eps) S_N.  The selected modes are the union over all knots.
 * amp: [nm][K][2] (re, im); keep: [nm], set to 0/1.  Returns the count kept.
 */
typedef struct { double p; int j; } or_pw_t;

static int or_pw_cmp(const void* a, const void* b) {
  const or_pw_t* x = (const or_pw_t*)a;
  const or_pw_t* y = (const or_pw_t*)b;
  if (x->p > y->p) return -1;
  if (x->p < y->p) return 1;
  return (x->j > y->j) - (x->j < y->j);
}

long long oracle_select_modes(int K, int nm, const double* amp, double eps, int* keep) {
  or_pw_t* P = (or_pw_t*)malloc(sizeof(or_pw_t) * (size_t)(nm > 0 ? nm : 1));
  for (int j = 0; j < nm; j++) keep[j] = 0;
  for (int k = 0; k < K; k++) {
    for (int j = 0; j < nm; j++) {
      const double re = amp[((size_t)j * K + k) * 2], im = amp[((size_t)j * K + k) * 2 + 1];
      P[j].p = re * re + im * im;
      P[j].j = j;
    }
    qsort(P, (size_t)nm, sizeof(or_pw_t), or_pw_cmp);
    double total = 0.0;
    for (int i = 0; i < nm; i++) total += P[i].p;
    const double thr = (1.0 - eps) * total;
    double before = 0.0;
    for (int i = 0; i < nm; i++) {
      if (!(before < thr)) break;
      keep[P[i].j] = 1;
      before += P[i].p;
    }
  }
  long long n = 0;
  for (int j = 0; j < nm; j++) n += keep[j];
  free(P);
  return n;
}
