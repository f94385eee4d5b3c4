// Per-(branch, bin) arithmetic of the SPA sum shared by the output kernel and
// the adjoint kernel, so that both evaluate exactly the same quantities.
// (arXiv 2307.12585, Sec. 2.2, Eq. 6: root of the segment cubic; Eq. 3-4, 10:
// phase 2 pi f t - Phi_V(t) - sgn(Fdot) pi/4 and weight 1/sqrt|Fdot|.)
#pragma once
#include "common.cuh"

namespace emrifd {

constexpr double kTwoPiOver2p64 = 3.4061215800865545e-19;   // 2 pi / 2^64 (exact scaling of 2 pi)

// root of b u + c u^2 + d u^3 = delta on [ulo, uhi] (monotone, direction dir):
// FP32 safeguarded Newton from a regula-falsi start, at most NIT steps, stopping
// once a step is below 4e-7; returns u and dF/du (FP32)
template <int NIT>
__device__ __forceinline__ float root_f32(float bf, float cf, float df, float dl, float lo, float hi, int dir,
                                          float& Dout) {
  float flo = ((df * lo + cf) * lo + bf) * lo - dl;
  float fhi = ((df * hi + cf) * hi + bf) * hi - dl;
  float u = lo + (hi - lo) * __fdividef(flo, flo - fhi);
  if (!(u >= lo && u <= hi)) u = 0.5f * (lo + hi);
  float D = 0.f;
#pragma unroll 1
  for (int it = 0; it < NIT; it++) {
    float fu = ((df * u + cf) * u + bf) * u - dl;
    D = (3.f * df * u + 2.f * cf) * u + bf;
    if (fu == 0.f) break;
    if ((fu > 0.f) == (dir > 0)) hi = u; else lo = u;
    float un = u - __fdividef(fu, D);
    if (!(un >= lo && un <= hi)) un = 0.5f * (lo + hi);
    const bool done = fabsf(un - u) <= 4e-7f;   // the next step would be below FP32 resolution
    u = un;
    if (done) break;
  }
  D = (3.f * df * u + 2.f * cf) * u + bf;
  Dout = D;
  return u;
}

// a5: segment of the run holding the root for key(g): s0 + knots already passed
__device__ __forceinline__ int run_segment(const Run& R, const long long* keyF, long long key_base, long long key) {
  int a = R.s0 + 1, bb = R.s1 + 1;
  while (a < bb) {
    int c = (a + bb) >> 1;
    long long kk = keyF[key_base + c];
    bool passed = R.dir > 0 ? (kk <= key) : (kk >= key);
    if (passed) a = c + 1; else bb = c;
  }
  return a - 1;
}

// a6 fallback: bracketed Newton-bisection in FP64 on [ulo, uhi] for the rare
// roots the fast path does not settle: next to a turnover the FP32 cubic can
// lose the root altogether (its coefficients' rounding exceeds |F* - f|) and
// Newton from there converges slowly or leaves the piece.  Bounded iterations.
static __device__ __noinline__ double solve_root_safe(const SegCore& C, double delta, double ulo, double uhi, int dir,
                                               double u) {
  double lo = ulo, hi = uhi;
  if (!(u > lo && u < hi)) u = 0.5 * (lo + hi);
  for (int it = 0; it < 200; it++) {
    const double r = fma(u, fma(u, fma(u, C.d, C.c), C.b), -delta);
    if (r == 0.0) break;
    if ((r > 0.0) == (dir > 0)) hi = u;
    else lo = u;
    const double D = fma(u, fma(u, C.d3, C.c2), C.b);
    double un = u - r / D;
    if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
    if (un == u || !(hi > lo)) break;
    u = un;
  }
  // the end of the bracket with the smaller residual if the iteration stalled there
  const double rl = fabs(fma(lo, fma(lo, fma(lo, C.d, C.c), C.b), -delta));
  const double rh = fabs(fma(hi, fma(hi, fma(hi, C.d, C.c), C.b), -delta));
  const double ru = fabs(fma(u, fma(u, fma(u, C.d, C.c), C.b), -delta));
  if (rl < ru && rl <= rh) return lo;
  if (rh < ru) return hi;
  return u;
}

// a6, FP64 polish of an FP32 root uf (with its FP32 dF/du Df): Newton steps with the
// FP64 residual and the FP32 reciprocal derivative, iterated where the predicted
// error of one step exceeds 1e-13 (i.e. near turnovers), clamped into [ulo, uhi].
// With SETTLE (the extended form, which is finite and well-conditioned next to
// turnovers), a polish that has not settled or had to be clamped is redone by
// solve_root_safe; the standard form's weight diverges there anyway, and the
// call's register cost is not worth paying in its hot loop.
template <bool SETTLE = false>
__device__ __forceinline__ double polish_root_f64(const SegCore& C, double delta, double ulo, double uhi, int dir,
                                                  float& uf, float& Df) {
  double u = f2d_bits(uf);
  double res = fma(u, fma(u, fma(u, C.d, C.c), C.b), -delta);
  float rcf = __fdividef(1.f, Df);
  u = fma(-res, f2d_bits(rcf), u);
  float stp = fabsf(d2f_bits(res) * rcf);
  float kap = fabsf(__fdividef(C.cf + 3.f * C.df * uf, Df));
  float err = stp * (kap * stp + 4.8e-7f);
#pragma unroll 1
  for (int it = 0; it < 4 && err > 1e-13f; it++) {
    float ufc = d2f_bits(u);
    float Dc = (3.f * C.df * ufc + 2.f * C.cf) * ufc + C.bf;
    res = fma(u, fma(u, fma(u, C.d, C.c), C.b), -delta);
    float rc2 = __fdividef(1.f, Dc);
    u = fma(-res, f2d_bits(rc2), u);
    stp = fabsf(d2f_bits(res) * rc2);
    kap = fabsf(__fdividef(C.cf + 3.f * C.df * ufc, Dc));
    err = stp * (kap * stp + 4.8e-7f);
  }
  // clamp into the piece (integer order of the bits is numeric order for u >= 0;
  // a negative u has the sign bit set and compares below ulo)
  bool settle = err > 1e-13f;
  const long long ub_ = __double_as_longlong(u);
  if (ub_ < __double_as_longlong(ulo)) { u = ulo; settle = true; }
  else if (ub_ > __double_as_longlong(uhi)) { u = uhi; settle = true; }
  if (SETTLE && settle) {
    u = solve_root_safe(C, delta, ulo, uhi, dir, u);
    uf = d2f_bits(u);
    Df = (3.f * C.df * uf + 2.f * C.cf) * uf + C.bf;
  }
  return u;
}


// a6, FP32 root in one pass for well-conditioned pieces: the inverse series of the
// cubic b u + c u^2 + d u^3 = dl about u = 0 to third order in x = dl/b,
// u0 = x - p x^2 + (2 p^2 - q) x^3 (p = c/b, q = d/b, from the record's rb = 1/b),
// then one Newton step.  The series' error is O(p^3 x^4) and the step squares it, so
// the result is taken when |p x| and |q x^2| are at most 1/32, the step keeps u in
// [lo, hi], and the predicted error of a further step is below 1e-8; otherwise (near
// turnovers, strong curvature) ok = false and the caller runs the safeguarded
// iteration.  Returns u, dF/du at u0 (within |F''| |step| of dF/du(u)) and the
// reciprocal of that derivative.
__device__ __forceinline__ float root_f32_series(float bf, float cf, float df, float rbf, float dl, float lo,
                                                 float hi, float& Dout, float& rDout, float& stepout, bool& ok) {
  const float x = dl * rbf;
  const float p = cf * rbf, q = df * rbf;
  const float px = p * x, qxx = q * x * x;
  const float u0 = x * fmaf(-x, fmaf(-x, fmaf(2.f * p, p, -q), p), 1.f);
  const float D = fmaf(fmaf(3.f * df, u0, 2.f * cf), u0, bf);
  const float fu = fmaf(fmaf(fmaf(df, u0, cf), u0, bf), u0, -dl);
  const float rD = __fdividef(1.f, D);
  const float step = fu * rD;
  const float u = u0 - step;
  ok = rbf != 0.f && fabsf(px) <= 0.03125f && fabsf(qxx) <= 0.03125f && u >= lo && u <= hi &&
       fabsf(p) * step * step <= 1e-8f;
  Dout = D;
  rDout = rD;
  stepout = step;
  return u;
}

// a6: FP32 start value (the series and one Newton step where they settle it, the
// safeguarded iteration elsewhere), then the FP64 polish above.  ulof, uhif: the
// piece's bounds as floats (rounded; they only bracket the FP32 start)
template <int NIT, bool SETTLE = false>
__device__ __forceinline__ double solve_root(const SegCore& C, double delta, double ulo, double uhi, float ulof,
                                             float uhif, int dir, float& uf_out, float& Df_out) {
  float Df, rD, st;
  bool ok;
  const float dl = d2f_bits(delta);
  float uf = root_f32_series(C.bf, C.cf, C.df, C.rbf, dl, ulof, uhif, Df, rD, st, ok);
  if (!ok) uf = root_f32<NIT>(C.bf, C.cf, C.df, dl, ulof, uhif, dir, Df);
  const double u = polish_root_f64<SETTLE>(C, delta, ulo, uhi, dir, uf, Df);
  uf_out = uf;
  Df_out = Df;
  return u;
}

// a7: Q0.64 phase (turns) of 2 pi g t - Phi_V(t) + m phi - sgn(Fdot) pi/4.  g t_s is
// reduced modulo one turn from its exact integer mantissa product.  With INT_INSEG the
// in-segment product u (delta h - Q1 - ...) is too, in place of an FP64 multiply (one
// FP64 instruction fewer for FP64-bound kernels; the mixed form, which is bound by its
// integer work as much, keeps the multiply).
template <bool INT_INSEG = true>
__device__ __forceinline__ unsigned long long phase_q64(const SegCore& C, double g, double delta, double u,
                                                        bool pos_slope) {
  const double inner = fma(u, fma(u, C.P3, C.P2), C.Q1);
  unsigned long long Th = q64_mul(g, C.ts) - C.theta0;
  if constexpr (INT_INSEG) Th += q64_mul(u, fma(delta, C.h, -inner));
  else Th += q64_of(u * (delta * C.h - inner));
  Th += pos_slope ? (0ull - (1ull << 61)) : (1ull << 61);
  return Th;
}

// exact double of an integer with |r| < 2^52, from its bits (integer instructions only)
__device__ __forceinline__ double small_ll_to_double(long long r) {
  if (r == 0) return 0.0;
  const unsigned long long a = r < 0 ? 0ull - (unsigned long long)r : (unsigned long long)r;
  const int e = 63 - __clzll(a);                                   // 2^e <= a < 2^(e+1), e <= 51
  const unsigned long long bits = ((unsigned long long)(e + 1023) << 52) | ((a << (52 - e)) & 0xFFFFFFFFFFFFFull) |
                                  ((unsigned long long)r & 0x8000000000000000ull);
  return __longlong_as_double((long long)bits);
}

// -x/2 for a normal double x, from its bits: the sign flipped and the exponent
// lowered by one (integer instructions only)
__device__ __forceinline__ double neg_half_normal(double x) {
  return __hiloint2double((__double2hiint(x) ^ (int)0x80000000) - 0x00100000, __double2loint(x));
}

// w e^{2 pi i Th/2^64}: the table entry T_k = e^{2 pi i k/65536} nearest Th, times
// w (1 - x^2/2 + i x) with x = 2 pi (Th/2^64 - k/65536), |x| <= pi/65536.  The
// omitted terms of e^{ix} are below |x|^3/6 = 1.9e-14; the real factor w enters
// the two-term factor without a separate multiply (7 FP64 instructions in all).
// The extended form and the adjoint use it: both need w apart from the factor.
__device__ __forceinline__ void cis_w_q64(unsigned long long Th, const double2* tab, double w, double& er,
                                          double& ei) {
  const unsigned long long kq = (Th + (1ull << (63 - kTab64Bits))) >> (64 - kTab64Bits);
  const long long rr = (long long)(Th - (kq << (64 - kTab64Bits)));   // |rr| <= 2^47
  const double x = small_ll_to_double(rr) * kTwoPiOver2p64;   // 0, or normal (|x| >= 3.4e-19)
  const double wx = w * x;
  const double cw = rr != 0 ? fma(wx, neg_half_normal(x), w) : w;
  const double2 T = __ldg(tab + (kq & (kTab64N - 1)));
  er = fma(T.x, cw, -T.y * wx);
  ei = fma(T.y, cw, T.x * wx);
}

// The parts of e^{2 pi i Th/2^64} used by the standard FP64 form: the table entry
// T_k = e^{2 pi i k/65536} nearest Th, and with x = 2 pi (Th/2^64 - k/65536),
// |x| <= pi/65536, the factor e^{ix} = (1 - x^2/2)(1 + i x') + O(x^4) where
// x' = x (1 + x^2/3) (so that (1 - x^2/2) x' = x - x^3/6 + O(x^5)).  q = x^2/2 is a
// correction below 1.2e-9 and is formed in FP32 (its error is below 5e-16 of the
// result); it is returned as c1 = 1 - 2q, the double that folds it into the
// weight's Newton step.  x' is formed from the integer remainder, corrected in the
// integer domain, times 2 pi/2^64: one FP64 instruction in all.
__device__ __forceinline__ void cis_split_q64(unsigned long long Th, const double2* tab, double2& T, double& xp,
                                              double& c1) {
  const unsigned long long kq = (Th + (1ull << (63 - kTab64Bits))) >> (64 - kTab64Bits);
  const long long rr = (long long)(Th - (kq << (64 - kTab64Bits)));   // |rr| <= 2^47
  // x in FP32 from the top bits of rr (rr/2^25 rounded, |.| <= 2^22)
  const float rrf = small_int_to_float((int)((rr + (1ll << 24)) >> 25));
  const float xf = rrf * 1.1429048e-11f;                  // 2 pi 2^25/2^64
  const float qf = 0.5f * xf * xf;                        // <= 1.15e-9
  // rr x^2/3 = rr (2q/3) = (rr/2^25)(q 2^26/3), |.| <= 1.1e5, rounded to an integer
  const float corr = __fmul_rn(rrf, __fmul_rn(qf, 22369621.3f));
  const long long ci = (long long)(__float_as_int(__fadd_rn(corr, 12582912.0f)) - 0x4B400000);
  xp = small_ll_to_double(rr + ci) * kTwoPiOver2p64;
  // 2q in units of 2^-50 (q 2^51 <= 2.6e6 < 2^22); 1 - n 2^-53 has the bits of 1.0 minus n
  const long long qi =
      (long long)(__float_as_int(__fadd_rn(__fmul_rn(qf, 2251799813685248.0f), 12582912.0f)) - 0x4B400000);
  c1 = __longlong_as_double(0x3FF0000000000000ll - (qi << 3));
  T = __ldg(tab + (kq & (kTab64N - 1)));
}

// y^2 exactly, as a double, for a positive normal float y: the product of the
// 24-bit significands has at most 48 bits (integer instructions only)
__device__ __forceinline__ double sq_exact(float y) {
  const unsigned b = __float_as_uint(y);
  const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
  const unsigned long long p = m * m;                  // in [2^46, 2^48)
  const int top = (p >> 47) ? 47 : 46;                 // y^2 = p 2^(2e - 46), e the unbiased exponent
  const long long ex = 2 * ((int)(b >> 23) - 127) - 46 + top + 1023;
  return __longlong_as_double((ex << 52) | (long long)((p << (52 - top)) & 0xFFFFFFFFFFFFFull));
}

// a8: 1/sqrt|D| from an FP32 seed y0 and one FP64 Newton step,
// y = y0 + (y0/2)(1 - |D| y0^2); y0^2 and y0/2 are formed exactly outside the
// FP64 pipe, so the step takes two FP64 instructions.  A |D| below the float
// range gives an infinite seed (such a root sits on a turnover, where the
// standard form diverges anyway).
// With c1 = 1 - 2q in place of 1 the step returns (1 - q)/sqrt|D| to within
// |e| q/2 (below 3e-16 for a seed within 2 ulp), the weight already times a real
// factor 1 - q.
__device__ __forceinline__ double rsqrt_abs(double Dd, double c1 = 1.0) {
  const double Dabs = abs_bits(Dd);
  const float y0f = rsqrtf(d2f_bits(Dabs));
  const double y0 = f2d_bits(y0f), y0h = f2d_bits(0.5f * y0f);
  const double e = fma(-Dabs, sq_exact(y0f), c1);
  return fma(y0h, e, y0);
}

}  // namespace emrifd
