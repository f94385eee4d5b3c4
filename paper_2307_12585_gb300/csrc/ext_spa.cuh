// Extended stationary-phase factor (arXiv 2307.12585, Sec. 2.2, Eq. 7-10).
//
// Expanding a voice's phase to third order about a root t_j of F(t) = f turns
// the Fresnel integral of the standard SPA into
//   G(Fdot, Fddot) = -(2/sqrt 3) (i Fdot/|Fddot|) e^z K_{1/3}(z),
//   z = -i X,  X = 2 pi Fdot^3 / (3 Fddot^2),
// with the principal branch of K_{1/3}.  The leading minus sign is the
// reading taken of Eq. 10: as printed, Eq. 10 tends to the negative of the
// Fresnel value exp(-i sgn(Fdot) pi/4)/sqrt|Fdot| as Fddot -> 0; negated, the
// two roots of a pure cubic phase add up exactly to its Airy-function
// Fourier transform, and a single root tends to the Fresnel value.
//
// The kernels keep the standard weight and phase shift and multiply by
//   R(X) = G / [exp(-i sgn(Fdot) pi/4) / sqrt|Fdot|],
// which depends on X alone, tends to 1 as |X| -> inf and satisfies
// R(-X) = conj R(X).  It is evaluated from y = 1/X in one of three ways:
//   |X| >= 1000  Hankel's expansion of K_nu (DLMF 10.40.2) to (iy)^5:
//                R = sum_k a_k (i y)^k, a_k = prod_{j<=k} (4 nu^2 - (2j-1)^2)/(8 j);
//   12 <= |X|    the same expansion, summed until the terms fall below 1e-17
//                (the smallest term at |X| = 12 is 2e-12 relative);
//   |X| < 12     the ascending series of J_{+-1/3} (DLMF 10.2.2, 10.27.3 with
//                K_nu(-i x) written through J_{+-nu}(x)):
//                R = sqrt(2 pi/3) e^{-iX} [e^{-i pi/12} sqrt(X) J_{-1/3}(X)
//                                          - e^{-5 i pi/12} sqrt(X) J_{1/3}(X)].
// Worst relative error of R in FP64: about 3e-12, where the two forms meet.
#pragma once
#include "common.cuh"

namespace emrifd {

// a_k(1/3), k = 1..5: -5/72, 385/10368, -85085/2239488, 37182145/644972544,
// -5391411025/46438023168
constexpr double kExtA1 = -0.069444444444444444444;
constexpr double kExtA2 = 0.037133487654320987654;
constexpr double kExtA3 = -0.037993059127800640146;
constexpr double kExtA4 = 0.057649190412669721333;
constexpr double kExtA5 = -0.11609906402551541102;
constexpr double kExt3Over2Pi = 0.47746482927568600731;   // 3/(2 pi)
// limit of the two-root sum at a double root (Fdot = 0):
// 2 pi (pi |Fddot|)^{-1/3} Ai(0) = [2 pi^{2/3} / (3^{2/3} Gamma(2/3))] |Fddot|^{-1/3}
constexpr double kExtCoalesced = 1.5230912247769706422;

// |y| <= 1e-3 (|X| >= 1000): five terms of the expansion, error < 2e-16
__device__ __forceinline__ void ext_ratio_fast(double y, double& rr, double& ri) {
  const double y2 = y * y;
  rr = fma(y2, fma(y2, kExtA4, -kExtA2), 1.0);
  ri = y * fma(y2, fma(y2, kExtA5, -kExtA3), kExtA1);
}

// FP32 form of the five-term expansion for |y| <= 1e-2, returned as R - 1
__device__ __forceinline__ void ext_delta_f32(float y, float& dr, float& di) {
  const float y2 = y * y;
  dr = y2 * (y2 * (float)kExtA4 - (float)kExtA2);
  di = y * (y2 * (y2 * (float)kExtA5 - (float)kExtA3) + (float)kExtA1);
}

// any y (0 < |X| < inf; y = 0 gives 1)
static __device__ __noinline__ void ext_ratio_general(double y, double& rr, double& ri) {
  const double X = 1.0 / fabs(y);
  if (X >= 12.0) {
    double tr = 1.0, ti = 0.0, sr = 1.0, si = 0.0;
    for (int k = 1; k <= 40; k++) {
      const double c = (4.0 / 9.0 - (double)((2 * k - 1) * (2 * k - 1))) / (double)(8 * k) * y;
      const double nr = -ti * c, ni = tr * c;   // term *= a_k/a_{k-1} * (i y)
      tr = nr;
      ti = ni;
      sr += tr;
      si += ti;
      if (fabs(tr) + fabs(ti) < 1e-17) break;
    }
    rr = sr;
    ri = si;
    return;
  }
  const double q = -0.25 * X * X;
  double t = 1.0 / 1.3541179394264004169;     // 1/Gamma(2/3)
  double u = 1.0 / 0.89297951156924921122;    // 1/Gamma(4/3)
  double s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < 48; k++) {
    s1 += t;
    s2 += u;
    const double kk = (double)(k + 1);
    t *= q / (kk * (kk - 1.0 / 3.0));
    u *= q / (kk * (kk + 1.0 / 3.0));
    if (fabs(t) + fabs(u) < 1e-18 * (fabs(s1) + fabs(s2))) break;
  }
  const double x16 = sqrt(cbrt(X));                               // X^{1/6}
  const double jm = x16 * 1.2599210498948731648 * s1;             // sqrt(X) J_{-1/3}(X)
  const double jp = (X / x16) * 0.79370052598409973738 * s2;      // sqrt(X) J_{1/3}(X)
  const double c12 = 0.96592582628906828675, s12 = 0.25881904510252076235;   // cos, sin pi/12
  const double br = c12 * jm - s12 * jp;    // e^{-i pi/12} jm - e^{-5 i pi/12} jp
  const double bi = -s12 * jm + c12 * jp;
  double sx, cx;
  sincos(X, &sx, &cx);
  const double k0 = 1.4472025091165353187;   // sqrt(2 pi/3)
  rr = k0 * (cx * br + sx * bi);
  ri = k0 * (cx * bi - sx * br);
  if (y < 0.0) ri = -ri;
}

// R from y in FP64, choosing the form by |y|
__device__ __forceinline__ void ext_ratio(double y, double& rr, double& ri) {
  if (fabs(y) <= 1e-3) ext_ratio_fast(y, rr, ri);
  else ext_ratio_general(y, rr, ri);
}

// y = 1/X from dF/du (D), d2F/du2 (D2) and h (u = tau/h): 3 D2^2 / (2 pi h D^3)
__device__ __forceinline__ double ext_y(double D, double D2, double h) {
  return kExt3Over2Pi * D2 * D2 / (h * D * D * D);
}

// a root with dF/du == 0 exactly (a double root): the real factor that replaces
// sqrt(h)/sqrt|dF/du| (the amplitudes carry sqrt(h)), with no pi/4 phase shift;
// 0 when d2F/du2 is 0 as well
static __device__ __noinline__ double ext_coalesced(double D2, double h) {
  if (D2 == 0.0) return 0.0;
  // [2 pi^{2/3}/(3^{2/3} Gamma(2/3))] |Fddot|^{-1/3} / sqrt(h), Fddot = D2/h^2
  return kExtCoalesced * cbrt(h * h / fabs(D2)) / sqrt(h);
}

}  // namespace emrifd
