// Hot kernel of the SPA mode sum (arXiv 2307.12585, Sec. 2.2).
//
// For every output bin f and every monotone branch ("run") of every voice
// track that covers f (directly for F > 0, through conj H(-f) for F < 0):
//   a5  the spline segment holding the root: binary search over the run's
//       knot-frequency keys (integer compares);
//   a6  t(f): root of the segment cubic F(u) = f (Eq. 6) on the run's piece:
//       safeguarded FP32 Newton for the start point, FP64 Newton polish;
//   a7  the phase 2 pi f t - Phi_V(t) - sgn(Fdot) pi/4 (+ m phi from Y_lm) in
//       Q0.64 fixed-point turns: f t_s from the exact integer product of the
//       mantissas, Phi_V(t_s)/2pi precomputed in double-double, and the small
//       in-segment remainder in FP64;
//   a8  the weight 1/sqrt|Fdot|;
//   a9  the amplitude cubic;
//   a10 the voice value A w e^{i psi} times the polarisation weights;
//   a11 accumulation in registers in a fixed order, one store per bin.
// Extended plans (EXT) multiply each root's standard factor by the ratio R(X)
// of the extended SPA (Eq. 10; see ext_spa.cuh).
//
// Work decomposition: a persistent grid takes tiles of 32*BPL consecutive bins
// from a queue.  A tile's (run, sign) entries are collected in shared memory
// in ascending run order; warp w handles entries w, w+8, ... for all bins of
// the tile (BPL per lane) and the 8 warp partials are summed in warp order,
// so every bin's sum has a fixed order (no atomics on the outputs).
#include "spa_math.cuh"
#include "ff.cuh"
#include "ext_spa.cuh"
#include <cooperative_groups.h>

namespace emrifd {
namespace {

// FP32 Newton steps of the FP64X root's start value (the pair polish that follows
// iterates until its predicted error is below 1e-13)
#ifndef EMRI_FD_X_ROOT_NIT
#define EMRI_FD_X_ROOT_NIT 4
#endif

constexpr int kRpt = 4;   // runs tested per thread and pass when a tile collects its entries
static_assert(2 * kRpt * kThreads <= kListCap, "a pass must fit the entry list");

struct SpaParams {
  const WfInfo* wf;
  int n_wf;
  const ModeInfo* modes;
  const SegCore* core;
  const SegAmp64* amp64;
  const SegAmp32* amp32;
  const SegFF* segff;
  const long long* keyF;
  const Run* runs;
  const RunBins* rb;
  const double* freqs;
  void* hp;
  void* hc;
  const double2* tab;      // e^{2 pi i k/65536}
  const float4* tabf;
  const double* prefactor;
  const double* yk;                 // [segments] 3/(2 pi h), extended plans
  unsigned long long* counters;
  const int* status;
  long long tiles_total;
  long long run_cap, nm_total, seg_total, nf_total;   // array sizes (checked builds)
};

template <int BPL, int PREC>
struct Smem {
  int list[kListCap];
  int wsum[kWarps + 1];
  long long tile;
  int anyv[4];     // cluster members' "has entries" flags (tile split)
  float2 pf;       // the waveform's prefactor as an FP32 pair (FP64X)
  // The two are never live together: suni while a pass evaluates its entries, red after
  // a tile's last pass (barriers separate the uses), so they share their bytes.
  union {
    struct {
      int suni[kListCap];              // FP32-path kernels: each entry's segment when one holds all its tile bins
      int smode[BPL >= 2 ? kListCap : 1];   // and (tiles of 64 bins or more) its run's mode
    } ent;
    double red[kWarps][32 * BPL][4];   // FP64 partials, or FP32-pair partials in the same bytes
  };
};
// the entry table fits in the reduction buffer (with the mode only where it has room)
static_assert(sizeof(int) * (kListCap + kListCap) <= sizeof(double) * kWarps * 32 * 2 * 4, "entry table");

// FP64X per-(branch, bin) body: returns the four increments (h+ re, h+ im,
// hx re, hx im) as FP32 pairs in v[0..7]; false if the root has Fdot == 0
template <bool EXT>
__device__ __forceinline__ bool body_fp64x(const SegCore& C, const SegFF& X, double f, ff fx, bool neg, ff ulo, ff uhi,
                                           int dir, ff fa, ff fb, const float4* tabf, float* v) {
  const ff Ax = ff_make(X.A[0], X.A[1]), bx = ff_make(X.b[0], X.b[1]), cx_ = ff_make(X.c[0], X.c[1]),
           dx = ff_make(X.d[0], X.d[1]);
  const ff gx = neg ? ff_neg(fx) : fx;
  const ff dl = ff_sub(gx, Ax);
  // a6: FP32 start, then Newton with the residual in FP32 pairs
  float Df, rDs, sts;
  bool sok;
  float uf = root_f32_series(C.bf, C.cf, C.df, C.rbf, dl.hi, ulo.hi, uhi.hi, Df, rDs, sts, sok);
  if (!sok) uf = root_f32<EMRI_FD_X_ROOT_NIT>(C.bf, C.cf, C.df, dl.hi, ulo.hi, uhi.hi, dir, Df);
  ff t = ff_add(ff_mul_f(dx, uf), cx_);
  t = ff_add(ff_mul_f(t, uf), bx);
  ff res = ff_sub(ff_mul_f(t, uf), dl);
  const float rcf = __fdividef(1.f, Df);
  float stepf = -res.hi * rcf;
  ff u = two_sum(uf, stepf);
  float stp = fabsf(stepf);
  float kap = fabsf(__fdividef(C.cf + 3.f * C.df * uf, Df));
  float err = stp * (kap * stp + 4.8e-7f);
#pragma unroll 1
  for (int it = 0; it < 4 && err > 1e-13f; it++) {
    const float ufc = u.hi;
    const float Dc = (3.f * C.df * ufc + 2.f * C.cf) * ufc + C.bf;
    t = ff_add(ff_mul(dx, u), cx_);
    t = ff_add(ff_mul(t, u), bx);
    res = ff_sub(ff_mul(t, u), dl);
    const float rc2 = __fdividef(1.f, Dc);
    stepf = -res.hi * rc2;
    u = ff_add_f(u, stepf);
    stp = fabsf(stepf);
    kap = fabsf(__fdividef(C.cf + 3.f * C.df * ufc, Dc));
    err = stp * (kap * stp + 4.8e-7f);
  }
  bool settle = err > 1e-13f;
  if (ff_lt(u, ulo)) { u = ulo; settle = true; }
  else if (ff_lt(uhi, u)) { u = uhi; settle = true; }
  if (EXT && settle) {   // extended form only: rare, next to a turnover or at the piece's end
    const double ud = solve_root_safe(C, (neg ? -f : f) - C.A, ff_to_double(ulo), ff_to_double(uhi), dir,
                                      ff_to_double(u));
    u = ff_from_double(ud);
  }
  // a8: dF/du and 1/sqrt|dF/du| (rsqrtf seed, one Newton step in pairs)
  const ff D = ff_add(ff_mul(ff_add(ff_mul(ff_make(X.d3[0], X.d3[1]), u), ff_make(X.c2[0], X.c2[1])), u), bx);
  bool coal = D.hi == 0.f;   // a double root: no contribution, or (extended) the coalesced limit
  if (!EXT && coal) return false;
  const bool pos = D.hi > 0.f;
  const ff Da = pos ? D : ff_neg(D);
  // extended form: y = 1/X in FP32 where |y| <= 1e-3 (|R - 1| <= 7e-5), else in FP64
  float yf = 0.f;
  double yd = 0.0, D2d = 0.0;
  bool slow = false;
  if constexpr (EXT) {
    const float D2f = fmaf(2.f * X.d3[0], u.hi, X.c2[0]);
    const float r0 = rsqrtf(Da.hi), r2 = r0 * r0;
    yf = __fdividef((float)kExt3Over2Pi, X.h[0]) * D2f * D2f * (r2 * r2 * r2);
    if (!pos) yf = -yf;
    if (coal || !(fabsf(yf) <= 1e-3f)) {
      slow = true;
      D2d = fma(2.0 * C.d3, ff_to_double(u), C.c2);
      if (!coal) {
        yd = ext_y(ff_to_double(D), D2d, C.h);
        if (!(fabs(yd) < INFINITY)) coal = true;
      }
    }
  }
  ff wgt;
  if (coal) {
    const double m0 = ext_coalesced(D2d, C.h);
    if (m0 == 0.0) return false;
    wgt = ff_from_double(m0);
  } else {
    // one Newton step y0 (1 + e/2), e = 1 - |D| y0^2 (|e| ~ 1e-7): y0^2 exactly as a pair,
    // the leading product of e by an FMA, its small cross terms in FP32
    const float y0 = rsqrtf(Da.hi);
    const ff t2 = two_prod(y0, y0);
    const float e = __fsub_rn(__fmaf_rn(-Da.hi, t2.hi, 1.f), __fmaf_rn(Da.hi, t2.lo, __fmul_rn(Da.lo, t2.hi)));
    wgt = fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e));
  }
  // a7: phase, Q0.64 turns
  const ff dh = ff_mul(dl, ff_make(X.h[0], X.h[1]));
  const ff inner = ff_add(ff_mul(ff_add(ff_mul(ff_make(X.P3[0], X.P3[1]), u), ff_make(X.P2[0], X.P2[1])), u),
                          ff_make(X.Q1[0], X.Q1[1]));
  const ff inseg = ff_mul(ff_sub(dh, inner), u);
  const unsigned long long ft = q64_mul(f, C.ts);           // f t_s; the branch sign is applied here
  unsigned long long Th = (neg ? 0ull - ft : ft) - C.theta0 + q64_of_float(inseg.hi) + q64_of_float(inseg.lo);
  if (!coal) Th += pos ? (0ull - (1ull << 61)) : (1ull << 61);
  // e^{2 pi i Th/2^64}: table entry times (1 - x^2/2) + i x (and - i x^3/6 with the
  // coarse table), |x| <= pi/2^kTabBits
  const unsigned long long kq = (Th + (1ull << (63 - kTabBits))) >> (64 - kTabBits);
  const long long rr = (long long)(Th - (kq << (64 - kTabBits))) >> 8;   // units of 2^-56 turn
  const ff xt = two_sum(small_int_to_float((int)(rr >> 22)) * 5.820766091346741e-11f,        // 2^-34
                        small_int_to_float((int)(rr & 0x3FFFFF)) * 1.3877787807814457e-17f);  // 2^-56
  const ff xr = ff_mul(xt, ff_make(6.2831854820251465f, -1.7484555314695172e-07f));
  const float qx = 0.5f * xr.hi * xr.hi;
  const float4 T = __ldg(tabf + (kq & (kTabN - 1)));
  const ff Tc = ff_make(T.x, T.y), Ts = ff_make(T.z, T.w);
  ff er, ei;
  if constexpr (kTabBits >= 16) {
    // |x| <= 4.8e-5: x^3/6 < 2e-14 is dropped; x^2/2 < 1.2e-9 times the entry lies below
    // the pair's low word and is added into it
    er = ff_sub(Tc, ff_mul(Ts, xr));
    ei = ff_add(Ts, ff_mul(Tc, xr));
    er.lo = __fmaf_rn(-T.x, qx, er.lo);
    ei.lo = __fmaf_rn(-T.z, qx, ei.lo);
  } else {
    const ff sx = ff_add_f(xr, -xr.hi * xr.hi * xr.hi * (1.f / 6.f));
    er = ff_add_f(ff_sub(Tc, ff_mul(Ts, sx)), -T.x * qx);
    ei = ff_add_f(ff_add(Ts, ff_mul(Tc, sx)), -T.z * qx);
  }
  // a9-a10
  ff ar = ff_make(X.are[3][0], X.are[3][1]), ai = ff_make(X.aim[3][0], X.aim[3][1]);
#pragma unroll
  for (int k = 2; k >= 0; k--) {
    ar = ff_add(ff_mul(ar, u), ff_make(X.are[k][0], X.are[k][1]));
    ai = ff_add(ff_mul(ai, u), ff_make(X.aim[k][0], X.aim[k][1]));
  }
  ar = ff_mul(ar, wgt);
  ai = ff_mul(ai, wgt);
  if constexpr (EXT) {
    if (!coal) {
      if (!slow) {   // R = 1 + delta, |delta| <= 7e-5: the correction in FP32
        float dr, di;
        ext_delta_f32(yf, dr, di);
        const float cr = ar.hi * dr - ai.hi * di, ci = ar.hi * di + ai.hi * dr;
        ar = ff_add_f(ar, cr);
        ai = ff_add_f(ai, ci);
      } else {
        double rr, ri;
        ext_ratio(yd, rr, ri);
        const ff Rr = ff_from_double(rr), Ri = ff_from_double(ri);
        const ff nr = ff_sub(ff_mul(ar, Rr), ff_mul(ai, Ri));
        ai = ff_add(ff_mul(ar, Ri), ff_mul(ai, Rr));
        ar = nr;
      }
    }
  }
  const ff zr = ff_sub(ff_mul(ar, er), ff_mul(ai, ei));
  const ff zi = ff_add(ff_mul(ar, ei), ff_mul(ai, er));
  // a11: h+ += alpha Z (conj Z for F < 0), hx += i beta Z (-i beta conj Z)
  const ff o0 = ff_mul(fa, zr), o1 = ff_mul(neg ? ff_neg(fa) : fa, zi);
  const ff o2 = ff_mul(ff_neg(fb), zi), o3 = ff_mul(neg ? ff_neg(fb) : fb, zr);
  v[0] = o0.hi; v[1] = o0.lo; v[2] = o1.hi; v[3] = o1.lo; v[4] = o2.hi; v[5] = o2.lo; v[6] = o3.hi; v[7] = o3.lo;
  return true;
}

// mixed per-(branch, bin) body: FP64 in-segment phase (and, in the extended form,
// the root polish), FP32 root, weight, sincos, amplitude and products; increments in v[0..3]
template <bool EXT>
__device__ __forceinline__ bool body_mixed(const SegCore& C, const SegAmp32& Am, double f, bool neg, double ulo,
                                           double uhi, float ulof, float uhif, int dir, float fa, float fb,
                                           float* v) {
  const double g = neg ? flip_sign(f) : f;
  const double delta = g - C.A;
  float uf, Df;
  double u;
  if constexpr (EXT) {
    u = solve_root<4, EXT>(C, delta, ulo, uhi, ulof, uhif, dir, uf, Df);
  } else {
    // an FP32 root: the phase is stationary at the root (Eq. 4), so a root error du
    // moves it by only (1/2)(dF/du) h du^2 turns (below 1e-12 for an FP32 root's
    // ~1e-7).  The series start and one Newton step settle it in well-conditioned
    // pieces, the safeguarded iteration elsewhere.
    const float dl = d2f_bits(delta);
    float rD, step;
    bool ok;
    uf = root_f32_series(C.bf, C.cf, C.df, C.rbf, dl, ulof, uhif, Df, rD, step, ok);
    if (!ok) {
      uf = root_f32<4>(C.bf, C.cf, C.df, dl, ulof, uhif, dir, Df);
      rD = __fdividef(1.f, Df);
    }
    // the weight needs dF/du to ~5e-7: its FP32 rounding, eps (|b| + 2|c| + 3|d|)/|D|,
    // plus |F''| times the FP32 root's error, about 4 eps (|c| + 3|d|)(|dl| + |b|)/D^2
    // (eps = 2^-23 for the truncated coefficients).  Next to a turnover, where that
    // exceeds the bound, the root gets the FP64 polish and dF/du is taken in FP64.
    const float r = fabsf(rD);
    const float S1 = fmaf(3.f, fabsf(C.df), fmaf(2.f, fabsf(C.cf), fabsf(C.bf)));
    const float S2 = fmaf(3.f, fabsf(C.df), fabsf(C.cf));
    if (!(fmaf(4.f * S2, (fabsf(dl) + fabsf(C.bf)) * r, S1) * r <= 4.2f)) {
      u = polish_root_f64<false>(C, delta, ulo, uhi, dir, uf, Df);
      uf = d2f_bits(u);
      Df = d2f_bits(fma(u, fma(u, C.d3, C.c2), C.b));
    } else {
      u = f2d_bits(uf);
    }
  }
  // the standard form needs dF/du only in FP32 (for the weight); its sign is the run's
  // direction, and a root with Df == 0 sits on a turnover (no contribution)
  double Dd = 0.0;
  bool coal, pos;
  if constexpr (EXT) {
    Dd = fma(u, fma(u, C.d3, C.c2), C.b);
    coal = is_zero_bits(Dd);
    pos = __double_as_longlong(Dd) >= 0;
  } else {
    if (Df == 0.f) return false;
    coal = false;
    pos = dir > 0;
  }
  float wgt = rsqrtf(fabsf(Df));
  float rr = 1.f, ri = 0.f;
  if constexpr (EXT) {
    // extended form: R in FP32 where |y| <= 1e-2, else in FP64
    float yf = 0.f;
    if (!coal) {
      const float D2f = fmaf(2.f * C.df * 3.f, uf, 2.f * C.cf);
      const float r2 = wgt * wgt;
      yf = __fdividef((float)kExt3Over2Pi, d2f_bits(C.h)) * D2f * D2f * (r2 * r2 * r2);
      if (!pos) yf = -yf;
    }
    if (!coal && fabsf(yf) <= 1e-2f) {
      float dr, di;
      ext_delta_f32(yf, dr, di);
      rr = 1.f + dr;
      ri = di;
    } else {
      const double D2d = fma(2.0 * C.d3, u, C.c2);
      double y = 0.0;
      if (!coal) {
        y = ext_y(Dd, D2d, C.h);
        if (!(fabs(y) < INFINITY)) coal = true;
      }
      if (coal) {
        const double m0 = ext_coalesced(D2d, C.h);
        if (m0 == 0.0) return false;
        wgt = (float)m0;
      } else {
        double r0, r1;
        ext_ratio(y, r0, r1);
        rr = (float)r0;
        ri = (float)r1;
        wgt = (float)(1.0 / sqrt(fabs(Dd)));   // |y| > 1e-2: near a turnover, where FP32 dF/du is too coarse
      }
    }
  }
  // a7: g t - Phi_V(t)/2pi = delta t - u inner(u) - theta0' turns, with t = t_s + u h,
  // delta = g - A and theta0' = frac(Phi_V(t_s)/2pi - m phi/2pi - A t_s) (the mixed
  // plan's record); |delta t| stays below a few thousand turns, so its FP64 rounding
  // is ~1e-13 turn (the exact integer product g t_s is not needed at FP32 accuracy)
  const double inner = fma(u, fma(u, C.P3, C.P2), C.Q1);
  unsigned long long Th = q64_of(fma(delta, C.ts, u * fma(delta, C.h, -inner))) - C.theta0;
  Th += coal ? 0ull : (pos ? (0ull - (1ull << 61)) : (1ull << 61));
  // half-turns in [-1, 1) from the top 46 bits of Th, without conversion instructions,
  // then the hardware sine and cosine of pi th in [-pi, pi) (the XU pipe; absolute error
  // below 4e-7, as the FP32 form's other steps)
  const long long ts_ = (long long)Th;
  const float th = small_int_to_float((int)(ts_ >> 42)) * 4.76837158203125e-07f +              // 2^-21
                   small_int_to_float((int)((ts_ >> 20) & 0x3FFFFF)) * 1.1368683772161603e-13f;  // 2^-43
  float sn, cs;
#if EMRI_FD_MIXED_SINCOSPIF
  sincospif(th, &sn, &cs);
#else
  __sincosf(th * 3.14159265358979f, &sn, &cs);
#endif
  float are = ((Am.re[3] * uf + Am.re[2]) * uf + Am.re[1]) * uf + Am.re[0];
  float aim = ((Am.im[3] * uf + Am.im[2]) * uf + Am.im[1]) * uf + Am.im[0];
  are *= wgt;
  aim *= wgt;
  if constexpr (EXT) {
    const float nr = are * rr - aim * ri;
    aim = are * ri + aim * rr;
    are = nr;
  }
  const float zr = are * cs - aim * sn;
  const float zi = are * sn + aim * cs;
  v[0] = fa * zr; v[1] = (neg ? -fa : fa) * zi; v[2] = -fb * zi; v[3] = (neg ? -fb : fb) * zr;
  return true;
}

// resident CTAs per SM the FP32-path kernels are compiled for (sets their register budget)
#ifndef EMRI_FD_SPA_MINB
#define EMRI_FD_SPA_MINB 4
#endif
// and the standard FP64X kernel (five CTAs: 51 registers; 3% faster than four on the 2-yr,
// 2000-mode workload at 32-bin tiles, where four leave its 63 registers unspilled)
#ifndef EMRI_FD_SPAX_MINB
#define EMRI_FD_SPAX_MINB 5
#endif
// and the standard-SPA FP64 kernel (three CTAs of 256 threads: 80 registers, a few
// spilled; 1.4% faster than two CTAs at 128 registers on the 2-yr, 2000-mode
// workload).  The extended form's FP64 kernel keeps two.
#ifndef EMRI_FD_SPA64_MINB
#define EMRI_FD_SPA64_MINB 3
#endif
// 1: the mixed form takes e^{i psi} from sincospif; 0: from the hardware sine and cosine
#ifndef EMRI_FD_MIXED_SINCOSPIF
#define EMRI_FD_MIXED_SINCOSPIF 0
#endif
// 1: the FP64 kernel's loop over a lane's bins is rolled (one copy of the body), as in
// the FP32-path kernels; 0: unrolled
#ifndef EMRI_FD_SPA64_ROLLED
#define EMRI_FD_SPA64_ROLLED 1
#endif
// and the extended-SPA FP64 kernel
#ifndef EMRI_FD_SPA64_EXT_MINB
#define EMRI_FD_SPA64_EXT_MINB 3
#endif

// store one bin of the FP32-pair forms: FP64X applies mu/d_L (an FP32 pair) and writes
// doubles; the mixed form writes floats
template <int PREC>
__device__ __forceinline__ void store_bin(const SpaParams& P, float2 pf2, long long bin, const ff (&v)[4]) {
  if constexpr (PREC == 2) {
    const ff pf = ff_make(pf2.x, pf2.y);
    double o[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const ff r = ff_mul(v[c], pf);
      o[c] = f2d_bits(r.hi) + f2d_bits(r.lo);
    }
    reinterpret_cast<double2*>(P.hp)[bin] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(P.hc)[bin] = make_double2(o[2], o[3]);
  } else {
    reinterpret_cast<float2*>(P.hp)[bin] = make_float2(v[0].hi + v[0].lo, v[1].hi + v[1].lo);
    reinterpret_cast<float2*>(P.hc)[bin] = make_float2(v[2].hi + v[2].lo, v[3].hi + v[3].lo);
  }
}

constexpr int kBackPerFront = 8;   // back-of-queue (empty) tiles a CTA may take after each front tile

// CL > 1: a thread-block cluster of CL CTAs shares each tile.  Rank 0 takes the tile
// and writes it into every member's shared memory; member r scans every CL-th chunk of
// kRpt runs (chunk index = r mod CL), evaluates the entries it found and sums its warps'
// partials; the members' "has entries" flags are exchanged; after a cluster barrier,
// member r sums bins i = r (mod CL) over the members' partials in rank order
// (distributed shared memory) and stores them.  The order of every sum is fixed, so
// results do not depend on scheduling.  Every cluster barrier is reached by all threads
// of all members the same number of times: the tile and the exchanged flags are the
// same for all members.
template <int BPL, int PREC, bool EXT, int CL>
__global__ void __launch_bounds__(kThreads, PREC == 0 ? (EXT ? EMRI_FD_SPA64_EXT_MINB : EMRI_FD_SPA64_MINB)
                                                      : (PREC == 2 && !EXT ? EMRI_FD_SPAX_MINB : EMRI_FD_SPA_MINB))
    k_spa(SpaParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<BPL, PREC>& S = *reinterpret_cast<Smem<BPL, PREC>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int TB = 32 * BPL;
  static_assert(CL == 1 || CL == 2 || CL == 4, "cluster of 1, 2 or 4 CTAs");
  const int crank = CL > 1 ? (int)cooperative_groups::this_cluster().block_rank() : 0;
  if (*P.status != 0) return;

  // Two-ended tile queue in one 64-bit counter: the low word counts tiles taken from the
  // front (ascending bins: the heavy low-frequency tiles first), the high word tiles taken
  // from the back.  After each front tile a CTA takes up to kBackPerFront tiles from the
  // back while they are empty (beyond every run), so the zero output of the empty tail is
  // written while the heavy tiles are computed, not in a burst at the end (which matters
  // when the output is host memory written over the host link).
  int back = 0;                               // thread 0: back claims left
  bool prev_back = false, prev_any = true;    // thread 0: how the previous tile was taken / had entries
  bool started = false;                       // thread 0: a tile has been taken
  for (;;) {
    if (tid == 0 && crank == 0) {
      back = !started ? 0 : (prev_back ? (prev_any ? 0 : back - 1) : kBackPerFront);
      started = true;
      const bool fb = back > 0;
      const unsigned long long old = atomicAdd(&P.counters[0], fb ? (1ull << 32) : 1ull);
      const long long a = (long long)(old & 0xFFFFFFFFull), b = (long long)(old >> 32);
      const long long tv = a + b < P.tiles_total ? (fb ? P.tiles_total - 1 - b : a) : -1;
      if constexpr (CL > 1) {
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        for (int r = 0; r < CL; r++) *cl.map_shared_rank(&S.tile, r) = tv;
      } else {
        S.tile = tv;
      }
      prev_back = fb;
    }
    if constexpr (CL > 1) cooperative_groups::this_cluster().sync();
    else __syncthreads();
    const long long tile = S.tile;   // every member reads its own copy
    if (tile < 0) break;
    int lo = 0, hi = P.n_wf - 1;
    while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (P.wf[mid].tile_base <= tile) lo = mid; else hi = mid - 1; }
    const WfInfo W = P.wf[lo];
    const long long bin0 = W.fo + (tile - W.tile_base) * TB;
    const long long binEnd = min(bin0 + TB, W.fo + W.nf);

    double fq[BPL];
    long long kp[BPL], kn[BPL];
#pragma unroll
    for (int q = 0; q < BPL; q++) {
      long long b = bin0 + lane + 32 * q;
      fq[q] = b < binEnd ? P.freqs[b] : 1.0;
      kp[q] = ordkey(fq[q]);
      kn[q] = ordkey(flip_sign(fq[q]));
    }
    double acc[BPL][4];
    float accf[BPL][4], cmp[BPL][4];
    ff fqf[BPL], accx[BPL][4];
#pragma unroll
    for (int q = 0; q < BPL; q++) {
      fqf[q] = PREC == 2 ? ff_from_double(fq[q]) : ff_make(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 4; c++) accx[q][c] = ff_make(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < BPL; q++)
#pragma unroll
      for (int c = 0; c < 4; c++) { acc[q][c] = 0.0; accf[q][c] = 0.f; cmp[q][c] = 0.f; }

    long long rcur = 0;
    bool any = false;   // the tile has at least one entry (block-uniform)
    // a tile outside the waveform's occupied bin range has no entries: skip the run scan
    const long long nruns = (bin0 < W.occ_hi && binEnd > W.occ_lo) ? W.nruns : 0;
    while (rcur < nruns || rcur == 0) {
      // ---- collect (run, sign) entries overlapping [bin0, binEnd), ascending; each
      // thread tests kRpt consecutive runs per pass (one block-wide scan per
      // kRpt * kThreads runs), so the list order is the run order as before
      int cnt = 0;
      while (rcur < nruns && cnt + 2 * kRpt * kThreads <= kListCap) {
        const long long rb = rcur + ((long long)tid * CL + crank) * kRpt;
        unsigned flags = 0u;   // bit 2k: run rb + k covers the tile for +f, bit 2k + 1: for -f
#pragma unroll
        for (int k = 0; k < kRpt; k++) {
          if (rb + k < nruns) {
            const RunBins B = P.rb[W.run_base + rb + k];
            if (B.b0p < binEnd && B.b1p > bin0) flags |= 1u << (2 * k);
            if (B.b0n < binEnd && B.b1n > bin0) flags |= 2u << (2 * k);
          }
        }
        const int c = __popc(flags);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        if (lane == 31) S.wsum[warp] = incl;
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int w2 = 0; w2 < kWarps; w2++) {
          int v = S.wsum[w2];
          if (w2 < warp) before += v;
          total += v;
        }
        int pos = cnt + before + incl - c;
#pragma unroll
        for (int k = 0; k < kRpt; k++) {
          if (flags & (1u << (2 * k))) S.list[pos++] = (int)((rb + k) << 1);
          if (flags & (2u << (2 * k))) S.list[pos++] = (int)(((rb + k) << 1) | 1);
        }
        cnt += total;
        any |= total > 0;
        rcur += (long long)kRpt * kThreads * CL;
        __syncthreads();
      }
      if (rcur == 0) rcur = 1;   // no runs at all: leave the loop after this pass

      // ---- FP32-path kernels: each entry's segment when one segment holds all of its
      // tile bins (-1 otherwise), one thread per entry.  A search per thread, all of
      // them at once, instead of each warp searching at the head of every entry it
      // evaluates, where the search's dependent loads sat on the entry's critical path.
      // The segment is monotone in the bin: the first bin's segment holds the last bin
      // when that bin has passed the segment's first knot (or it is the run's first
      // segment) and not its next knot (or it is the run's last).
      if constexpr (PREC != 0) {
        for (int e = tid; e < cnt; e += kThreads) {
          const int ent = S.list[e];
          const long long r = W.run_base + (ent >> 1);
          const bool neg = ent & 1;
          int su = -1, md = 0;
          if (r >= 0 && r < P.run_cap) {
            const Run R = P.runs[r];
            const RunBins B = P.rb[r];
            const int b0 = neg ? B.b0n : B.b0p, b1 = neg ? B.b1n : B.b1p;
            if (R.mode >= 0 && R.mode < P.nm_total && R.s0 >= 0 && R.s0 <= R.s1 && b0 >= 0 && b1 <= P.nf_total) {
              md = R.mode;
              const long long kb = P.modes[R.mode].key_base;
              const long long lo_b = max((long long)b0, bin0), hi_b = min((long long)b1, binEnd) - 1;
              const double flo = P.freqs[lo_b], fhi = P.freqs[hi_b];
              const int s_lo = run_segment(R, P.keyF, kb, ordkey(neg ? flip_sign(flo) : flo));
              const long long khi = ordkey(neg ? flip_sign(fhi) : fhi);
              auto passed = [&](int k) {
                const long long kk = P.keyF[kb + k];
                return R.dir > 0 ? (kk <= khi) : (kk >= khi);
              };
              if ((s_lo == R.s0 || passed(s_lo)) && (s_lo == R.s1 || !passed(s_lo + 1))) su = s_lo;
            }
          }
          S.ent.suni[e] = su;
          if constexpr (BPL >= 2) S.ent.smode[e] = md;
        }
        __syncthreads();
      }
      // ---- evaluate: warp w takes entries w, w + kWarps, ...
      for (int e = warp; e < cnt; e += kWarps) {
        const int ent = S.list[e];
        const long long r = W.run_base + (ent >> 1);
        const bool neg = ent & 1;
        if (check_fails(r >= 0 && r < P.run_cap, P.status)) continue;
        const Run R = P.runs[r];
        const RunBins B = P.rb[r];
        const int b0 = neg ? B.b0n : B.b0p, b1 = neg ? B.b1n : B.b1p;
        if (check_fails(R.mode >= 0 && R.mode < P.nm_total && R.s0 >= 0 && R.s0 <= R.s1 && b0 >= 0 &&
                            b1 <= P.nf_total,
                        P.status))
          continue;
        const ModeInfo M = P.modes[(PREC != 0 && BPL >= 2) ? S.ent.smode[e] : R.mode];
        // a5 for the whole entry where one segment holds all its tile bins (FP32-path
        // kernels, found in the setup step above; in the FP64 kernel the per-bin integer
        // search overlaps the FP64 pipe for free)
        const int s_uni = PREC != 0 ? S.ent.suni[e] : -1;
        if constexpr (PREC == 0) {
          // h+ += alpha Z~, hx += i beta Z~ (conjugates on the negative branch).  The
          // amplitude record carries the factor scale (alpha or beta, the larger in
          // magnitude), so the two multipliers are 1 and rho in some order: with the
          // weight, cw and rho cw.  Sign flips are integer operations on the sign bit.
          const bool amaj = alpha_major(M.alpha, M.beta);
          const double rho = M.rho;
#if EMRI_FD_SPA64_ROLLED
#pragma unroll 1
#else
#pragma unroll
#endif
          for (int q = 0; q < BPL; q++) {
            const long long bin = bin0 + lane + 32 * q;
            if (bin < b0 || bin >= b1) continue;
            double fqq = fq[0];   // the lane's q-th bin (a predicated select when the loop is rolled)
#pragma unroll
            for (int qq = 1; qq < BPL; qq++)
              if (qq == q) fqq = fq[qq];
            const double g = neg ? flip_sign(fqq) : fqq;
            const long long key = ordkey(g);
            // a5: segment holding the root
            const int s = run_segment(R, P.keyF, M.key_base, key);
            if (check_fails(s >= R.s0 && s <= R.s1 && M.seg_base + s < P.seg_total, P.status)) continue;
            const double ulo = (s == R.s0) ? R.u0 : 0.0, uhi = (s == R.s1) ? R.u1 : 1.0;
            const SegCore& C = P.core[M.seg_base + s];
            // a6: root
            const double delta = g - C.A;
            float uf, Df;
            const double u = solve_root<6, EXT>(C, delta, ulo, uhi, s == R.s0 ? R.u0f[0] : 0.f,
                                                s == R.s1 ? R.u1f[0] : 1.f, R.dir, uf, Df);
            // a8: dF/du
            const double Dd = fma(u, fma(u, C.d3, C.c2), C.b);
            const long long Dbits = __double_as_longlong(Dd);
            bool coal = is_zero_bits(Dd);   // Fdot == 0
            if (!EXT && coal) continue;                         // standard form: no contribution
            const bool pos_slope = Dbits >= 0;
            const SegAmp64 Am = P.amp64[M.seg_base + s];
            double zr, zi, mp, mx;   // h+ += mp Z, hx += i mx Z (Z without the weight's factor)
            // extended form: R(X) = G_ext / G_std depends on y = 1/X = yk (d2F/du2)^2 / (dF/du)^3
            // alone; where |y| <= 1e-3 (almost every bin) R - 1 is below 7e-5, so it is
            // formed in FP32 and applied to the standard tail's Z (its error, ~1e-11 of Z,
            // is far inside the FP64 bound).  Next to turnovers R comes from FP64 below.
            float yf = 0.f;
            bool fast = !EXT;
            if constexpr (EXT) {
              if (!coal) {
                const float r0 = rsqrtf(d2f_bits(abs_bits(Dd))), r2 = r0 * r0;
                const float D2f = fmaf(6.f * C.df, uf, 2.f * C.cf);
                yf = d2f_bits(P.yk[M.seg_base + s]) * D2f * D2f * (r2 * r2 * r2);
                if (!pos_slope) yf = -yf;
                fast = fabsf(yf) <= 1e-3f;
              }
            }
            if (fast) {
              // a7: phase in Q0.64 turns; e^{i psi} = T_k (1 - q)(1 + i x')
              const unsigned long long Th = phase_q64(C, g, delta, u, pos_slope);
              double2 T;
              double xp, c1;
              cis_split_q64(Th, P.tab, T, xp, c1);   // the 1 MB table is read through L1 and L2
              // a8: the weight (1 - q)/sqrt|dF/du| (sqrt(h) is in the amplitude)
              const double cw = rsqrt_abs(Dd, c1);
              // a9-a10: Z = (A T)(1 + i x'), the multipliers cw and rho cw
              const double are = fma(u, fma(u, fma(u, Am.re[3], Am.re[2]), Am.re[1]), Am.re[0]);
              const double aim = fma(u, fma(u, fma(u, Am.im[3], Am.im[2]), Am.im[1]), Am.im[0]);
              const double atr = fma(are, T.x, -aim * T.y), ati = fma(are, T.y, aim * T.x);
              zr = fma(-xp, ati, atr);
              zi = fma(xp, atr, ati);
              if constexpr (EXT) {   // Z R = Z + Z (R - 1), the correction in FP32
                float dr, di;
                ext_delta_f32(yf, dr, di);
                const float zrf = d2f_bits(zr), zif = d2f_bits(zi);
                zr += f2d_bits(fmaf(zrf, dr, -zif * di));
                zi += f2d_bits(fmaf(zrf, di, zif * dr));
              }
              const double t = rho * cw;
              mp = amaj ? cw : t;
              mx = amaj ? t : cw;
            } else {
              // extended form: R(X) from y = 1/X = 3 (d2F/du2)^2 / (2 pi h (dF/du)^3)
              double wgt = coal ? 0.0 : rsqrt_abs(Dd);
              double rr = 1.0, ri = 0.0;
              const double D2 = fma(2.0 * C.d3, u, C.c2);
              if (!coal) {
                const double w2 = wgt * wgt;
                double y = P.yk[M.seg_base + s] * (D2 * D2) * (w2 * w2 * w2);
                if (!pos_slope) y = -y;
                if (fabs(y) < INFINITY) ext_ratio(y, rr, ri);
                else coal = true;
              }
              if (coal) {
                wgt = ext_coalesced(D2, C.h);
                if (wgt == 0.0) continue;
              }
              // a7: phase in Q0.64 turns (a double root has no pi/4 shift)
              unsigned long long Th = phase_q64(C, g, delta, u, pos_slope);
              if (coal) Th += pos_slope ? (1ull << 61) : (0ull - (1ull << 61));
              double er, ei;
              cis_w_q64(Th, P.tab, wgt, er, ei);   // w e^{i psi}
              // a9-a10
              double are = fma(u, fma(u, fma(u, Am.re[3], Am.re[2]), Am.re[1]), Am.re[0]);
              double aim = fma(u, fma(u, fma(u, Am.im[3], Am.im[2]), Am.im[1]), Am.im[0]);
              const double nr = fma(are, rr, -aim * ri);
              aim = fma(are, ri, aim * rr);
              are = nr;
              zr = fma(are, er, -aim * ei);
              zi = fma(are, ei, aim * er);
              mp = amaj ? 1.0 : rho;
              mx = amaj ? rho : 1.0;
            }
            // a11: positive branch h+ += alpha Z, hx += i beta Z;
            //      negative branch h+ += alpha conj Z, hx += -i beta conj Z
#pragma unroll
            for (int qq = 0; qq < BPL; qq++) {
              if (qq != q) continue;
              acc[qq][0] = fma(mp, zr, acc[qq][0]);
              acc[qq][1] = fma(neg ? flip_sign(mp) : mp, zi, acc[qq][1]);
              acc[qq][2] = fma(flip_sign(mx), zi, acc[qq][2]);
              acc[qq][3] = fma(neg ? flip_sign(mx) : mx, zr, acc[qq][3]);
            }
          }
        } else {
          // FP64X and mixed: one copy of the per-bin body (rolled loop over the
          // lane's bins); per-lane values and accumulators are selected with
          // predicated moves so they stay in registers
          const ff fa = ff_make(M.af[0], M.af[1]), fb = ff_make(M.bf[0], M.bf[1]);
          const ff u0x = ff_make(R.u0f[0], R.u0f[1]), u1x = ff_make(R.u1f[0], R.u1f[1]);
#pragma unroll 1
          for (int q = 0; q < BPL; q++) {
            const long long bin = bin0 + lane + 32 * q;
            if (bin < b0 || bin >= b1) continue;
            double fqq = fq[0];
            long long kq_ = neg ? kn[0] : kp[0];
            ff fx = fqf[0];
#pragma unroll
            for (int qq = 1; qq < BPL; qq++)
              if (qq == q) { fqq = fq[qq]; kq_ = neg ? kn[qq] : kp[qq]; fx = fqf[qq]; }
            const int s = s_uni >= 0 ? s_uni : run_segment(R, P.keyF, M.key_base, kq_);
            if (check_fails(s >= R.s0 && s <= R.s1 && M.seg_base + s < P.seg_total, P.status)) continue;
            // the record is read through a reference, so that fields used only on the rare
            // slow paths (the FP64 root polish) are loaded there rather than held in registers
            const SegCore& C = P.core[M.seg_base + s];
            float v[8];
            bool ok;
            if constexpr (PREC == 2) {
              ok = body_fp64x<EXT>(C, P.segff[M.seg_base + s], fqq, fx, neg, s == R.s0 ? u0x : ff_make(0.f, 0.f),
                              s == R.s1 ? u1x : ff_make(1.f, 0.f), R.dir, fa, fb, P.tabf, v);
            } else {
              const double ulo = (s == R.s0) ? R.u0 : 0.0, uhi = (s == R.s1) ? R.u1 : 1.0;
              ok = body_mixed<EXT>(C, P.amp32[M.seg_base + s], fqq, neg, ulo, uhi, s == R.s0 ? R.u0f[0] : 0.f,
                                   s == R.s1 ? R.u1f[0] : 1.f, R.dir, M.af[0], M.bf[0], v);
            }
            if (!ok) continue;
#pragma unroll
            for (int qq = 0; qq < BPL; qq++) {
              if (qq != q) continue;
              if constexpr (PREC == 2) {
#pragma unroll
                for (int c = 0; c < 4; c++) accx[qq][c] = ff_acc(accx[qq][c], ff_make(v[2 * c], v[2 * c + 1]));
              } else {
#pragma unroll
                for (int c = 0; c < 4; c++) {   // Kahan-compensated accumulation
                  float y = v[c] - cmp[qq][c];
                  float t2 = accf[qq][c] + y;
                  cmp[qq][c] = (t2 - accf[qq][c]) - y;
                  accf[qq][c] = t2;
                }
              }
            }
          }
        }
      }
      __syncthreads();
      if (rcur >= nruns) break;
    }

    if constexpr (CL > 1) {
      // the cluster has entries if any member has: every member gets every flag (this
      // barrier also orders rank 0's next tile broadcast after every member's read)
      cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
      if (tid == 0)
        for (int r = 0; r < CL; r++) *cl.map_shared_rank(&S.anyv[crank], r) = any ? 1 : 0;
      cl.sync();
      any = false;
#pragma unroll
      for (int r = 0; r < CL; r++) any |= S.anyv[r] != 0;
    }
    if (tid == 0) prev_any = any;
    // ---- a tile without entries is written as zeros, without the reduction
    if (!any) {
      for (int i = tid; i < TB; i += kThreads) {
        const long long bin = bin0 + i;
        if (bin >= binEnd || i % CL != crank) continue;
        if constexpr (PREC == 1) {
          reinterpret_cast<float2*>(P.hp)[bin] = make_float2(0.f, 0.f);
          reinterpret_cast<float2*>(P.hc)[bin] = make_float2(0.f, 0.f);
        } else {
          reinterpret_cast<double2*>(P.hp)[bin] = make_double2(0.0, 0.0);
          reinterpret_cast<double2*>(P.hc)[bin] = make_double2(0.0, 0.0);
        }
      }
      continue;   // the loop's closing barrier above (and, for CL > 1, the flag exchange) separates the tiles
    }
    // ---- fixed-order reduction over warps, one store per bin (FP64 sums for the
    // FP64 form; FP32 pairs for the other two, so that they spend no FP64
    // instruction per bin beyond the final conversion)
    if constexpr (PREC == 0) {
#pragma unroll
      for (int q = 0; q < BPL; q++)
#pragma unroll
        for (int c = 0; c < 4; c++) S.red[warp][lane + 32 * q][c] = acc[q][c];
    } else {
      float2(&redf)[kWarps][32 * BPL][4] = *reinterpret_cast<float2(*)[kWarps][32 * BPL][4]>(&S.red[0][0][0]);
#pragma unroll
      for (int q = 0; q < BPL; q++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const ff v = PREC == 2 ? fast_two_sum(accx[q][c].hi, accx[q][c].lo) : fast_two_sum(accf[q][c], -cmp[q][c]);
          redf[warp][lane + 32 * q][c] = make_float2(v.hi, v.lo);
        }
    }
    if (PREC == 2 && tid == 0) {
      const ff pf = ff_from_double(P.prefactor[lo]);
      S.pf = make_float2(pf.hi, pf.lo);
    }
    __syncthreads();
    if constexpr (CL == 1) {
      for (int i = tid; i < TB; i += kThreads) {
        const long long bin = bin0 + i;
        if (bin >= binEnd) continue;
        if constexpr (PREC == 0) {
          double v[4] = {S.red[0][i][0], S.red[0][i][1], S.red[0][i][2], S.red[0][i][3]};
          for (int w2 = 1; w2 < kWarps; w2++)
#pragma unroll
            for (int c = 0; c < 4; c++) v[c] += S.red[w2][i][c];
          reinterpret_cast<double2*>(P.hp)[bin] = make_double2(v[0], v[1]);
          reinterpret_cast<double2*>(P.hc)[bin] = make_double2(v[2], v[3]);
        } else {
          const float2(&redf)[kWarps][32 * BPL][4] =
              *reinterpret_cast<const float2(*)[kWarps][32 * BPL][4]>(&S.red[0][0][0]);
          ff v[4];
#pragma unroll
          for (int c = 0; c < 4; c++) v[c] = ff_make(0.f, 0.f);
          for (int w2 = 0; w2 < kWarps; w2++)
#pragma unroll
            for (int c = 0; c < 4; c++) v[c] = ff_add(v[c], ff_make(redf[w2][i][c].x, redf[w2][i][c].y));
          store_bin<PREC>(P, S.pf, bin, v);
        }
      }
      __syncthreads();
    } else {
      // this member's partial of each bin, in warp order, into warp 0's slot
      for (int i = tid; i < TB; i += kThreads) {
        if constexpr (PREC == 0) {
          double v[4] = {S.red[0][i][0], S.red[0][i][1], S.red[0][i][2], S.red[0][i][3]};
          for (int w2 = 1; w2 < kWarps; w2++)
#pragma unroll
            for (int c = 0; c < 4; c++) v[c] += S.red[w2][i][c];
#pragma unroll
          for (int c = 0; c < 4; c++) S.red[0][i][c] = v[c];
        } else {
          float2(&redf)[kWarps][32 * BPL][4] = *reinterpret_cast<float2(*)[kWarps][32 * BPL][4]>(&S.red[0][0][0]);
          ff v[4];
#pragma unroll
          for (int c = 0; c < 4; c++) v[c] = ff_make(0.f, 0.f);
          for (int w2 = 0; w2 < kWarps; w2++)
#pragma unroll
            for (int c = 0; c < 4; c++) v[c] = ff_add(v[c], ff_make(redf[w2][i][c].x, redf[w2][i][c].y));
#pragma unroll
          for (int c = 0; c < 4; c++) redf[0][i][c] = make_float2(v[c].hi, v[c].lo);
        }
      }
      cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
      cl.sync();
      // member r stores bins i = r (mod CL): the members' partials summed in rank order
      for (int i = tid; i < TB; i += kThreads) {
        const long long bin = bin0 + i;
        if (bin >= binEnd || i % CL != crank) continue;
        if constexpr (PREC == 0) {
          double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
          for (int r = 0; r < CL; r++) {
            const double* src = cl.map_shared_rank(&S.red[0][i][0], r);
#pragma unroll
            for (int c = 0; c < 4; c++) v[c] = r == 0 ? src[c] : v[c] + src[c];
          }
          reinterpret_cast<double2*>(P.hp)[bin] = make_double2(v[0], v[1]);
          reinterpret_cast<double2*>(P.hc)[bin] = make_double2(v[2], v[3]);
        } else {
          ff v[4];
#pragma unroll
          for (int c = 0; c < 4; c++) v[c] = ff_make(0.f, 0.f);
#pragma unroll
          for (int r = 0; r < CL; r++) {
            const float2* src = cl.map_shared_rank(reinterpret_cast<const float2*>(&S.red[0][0][0]) + 4 * i, r);
#pragma unroll
            for (int c = 0; c < 4; c++) v[c] = ff_add(v[c], ff_make(src[c].x, src[c].y));
          }
          store_bin<PREC>(P, S.pf, bin, v);
        }
      }
      cl.sync();   // the partials are read before any member overwrites them or exits
    }
  }
}

template <int BPL, int PREC, bool EXT, int CL>
void launch_one(const SpaParams& p, int num_sms, cudaStream_t st) {
  size_t sm = sizeof(Smem<BPL, PREC>);
  cudaFuncSetAttribute(k_spa<BPL, PREC, EXT, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spa<BPL, PREC, EXT, CL>, kThreads, sm);
  if (per_sm < 1) per_sm = 1;
  if constexpr (CL == 1) {
    long long grid = (long long)num_sms * per_sm;
    if (grid > p.tiles_total) grid = p.tiles_total > 0 ? p.tiles_total : 1;
    k_spa<BPL, PREC, EXT, 1><<<(unsigned)grid, kThreads, sm, st>>>(p);
  } else {
    // clusters of CL CTAs: as many as can be resident, at most one per tile
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    long long grid = ((long long)num_sms * per_sm / CL) * CL;
    if (grid < CL) grid = CL;
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_spa<BPL, PREC, EXT, CL>, &cfg) == cudaSuccess && nclusters > 0)
      grid = (long long)nclusters * CL;
    else
      cudaGetLastError();
    const long long need = (p.tiles_total > 0 ? p.tiles_total : 1) * CL;
    if (grid > need) grid = need;
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cudaLaunchKernelEx(&cfg, k_spa<BPL, PREC, EXT, CL>, p);
  }
}

template <int PREC, bool EXT>
void launch_tile(const SpaParams& p, int bpl, int split, int num_sms, cudaStream_t st) {
  // tile splitting is built for the small tiles (sparse grids have few tiles)
  if (bpl == 1) {
    if (split == 4) launch_one<1, PREC, EXT, 4>(p, num_sms, st);
    else if (split == 2) launch_one<1, PREC, EXT, 2>(p, num_sms, st);
    else launch_one<1, PREC, EXT, 1>(p, num_sms, st);
  } else if (bpl == 2) {
    if (split == 4) launch_one<2, PREC, EXT, 4>(p, num_sms, st);
    else if (split == 2) launch_one<2, PREC, EXT, 2>(p, num_sms, st);
    else launch_one<2, PREC, EXT, 1>(p, num_sms, st);
  } else {
    launch_one<4, PREC, EXT, 1>(p, num_sms, st);
  }
}

template <bool EXT>
void launch_prec(const SpaParams& p, int bpl, int split, int precision, int num_sms, cudaStream_t st) {
  if (precision == 0) launch_tile<0, EXT>(p, bpl, split, num_sms, st);
  else if (precision == 2) launch_tile<2, EXT>(p, bpl, split, num_sms, st);
  else launch_tile<1, EXT>(p, bpl, split, num_sms, st);
}

}  // namespace

void launch_spa(const CallShape& cs, const DevInputs& in, const DevScratch& s, int num_sms, cudaStream_t st) {
  SpaParams p;
  p.wf = s.wf; p.n_wf = cs.n_wf; p.modes = s.modes; p.core = s.core; p.amp64 = s.amp64; p.amp32 = s.amp32;
  p.keyF = s.keyF; p.runs = s.runs; p.rb = s.rbins; p.freqs = in.freqs; p.hp = in.h_plus; p.hc = in.h_cross;
  p.tab = s.tab; p.counters = s.counters; p.status = s.status; p.tiles_total = cs.tiles_total;
  p.run_cap = s.run_cap; p.nm_total = cs.nm_total; p.seg_total = cs.seg_total; p.nf_total = cs.nf_total;
  p.segff = s.segff; p.tabf = s.tabf; p.prefactor = in.prefactor; p.yk = s.yk;
  cudaMemsetAsync(s.counters, 0, sizeof(unsigned long long), st);
  const int bpl = cs.tile_bins / 32;
  if (cs.ext) launch_prec<true>(p, bpl, cs.tile_split, cs.precision, num_sms, st);
  else launch_prec<false>(p, bpl, cs.tile_split, cs.precision, num_sms, st);
}

}  // namespace emrifd
