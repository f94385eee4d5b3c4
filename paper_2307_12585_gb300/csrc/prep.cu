// Preparation kernels of the SPA mode sum: input checks, polarisation weights,
// not-a-knot spline solves, per-(mode, segment) records, turnovers, and the
// monotone branches ("runs") of every voice's frequency track.
//
// Paper: arXiv 2307.12585, Sec. 2.1 (not-a-knot splines of phases, frequencies
// and amplitudes on the sparse trajectory), Sec. 2.2 (Eq. 6: per-segment
// frequency cubic from the fundamental-frequency spline coefficients weighted
// by the mode numbers; turnovers where dF/dt = 0, at most one per segment in
// practice; the segment of each frequency is determined before the summation).
#include "common.cuh"
#include "ff.cuh"

namespace emrifd {

namespace {

constexpr double kTwoPi = 6.283185307179586;
constexpr double kInv2PiHi = 0.15915494309189535;
constexpr double kInv2PiLo = -9.839338337591243e-18;

// ------------------------------------------------------------------ checks
__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

__device__ __forceinline__ bool finite_bits(double x) {
  return (__double_as_longlong(x) & 0x7FF0000000000000LL) != 0x7FF0000000000000LL;
}

__global__ void k_validate_knots(const WfInfo* wf, DevInputs in, int* status) {
  const WfInfo W = wf[blockIdx.y];
  int bad = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < W.K; k += (long long)gridDim.x * blockDim.x) {
    long long i = W.ko + k;
    double t = in.t[i];
    if (!(finite_bits(t) && finite_bits(in.phi_phi[i]) && finite_bits(in.phi_r[i]) && finite_bits(in.omega_phi[i]) &&
          finite_bits(in.omega_r[i])))
      bad |= ST_NONFINITE;
    if (k + 1 < W.K && !(ordkey(in.t[i + 1]) > ordkey(t))) bad |= ST_KNOTS;
  }
  if (bad) atomicOr(status, bad);
}

// frequencies: positive, finite and strictly increasing, checked on the bit
// patterns (for positive doubles integer order is numeric order)
__global__ void k_validate_freqs(const WfInfo* wf, DevInputs in, int* status) {
  const WfInfo W = wf[blockIdx.y];
  int bad = 0;
  const long long* fb = reinterpret_cast<const long long*>(in.freqs) + W.fo;
#pragma unroll 4
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < W.nf; k += (long long)gridDim.x * blockDim.x) {
    const long long u = fb[k];
    if (!(u > 0 && u < 0x7FF0000000000000LL)) bad |= ST_FREQ;
    if (k + 1 < W.nf && !(fb[k + 1] > u)) bad |= ST_FREQ;
  }
  if (bad) atomicOr(status, bad);
}

__global__ void k_validate_amp(long long n2, const double* amp, int* status) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x)
    if (!finite_bits(amp[i])) bad = ST_NONFINITE;
  if (bad) atomicOr(status, bad);
}

// ---------------------------------------------------- spin-weighted harmonic
// -2Y_lm(theta, phi) = S_lm(theta) e^{i m phi} with
// S_lm = (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta), s = -2, and the Wigner
// small-d sum (1/k! from a table of the nearest doubles, k <= 40)  d^l_{a,b}(x) = sum_k (-1)^{a-b+k} sqrt((l+a)!(l-a)!(l+b)!(l-b)!)
//   / ((l+b-k)! k! (a-b+k)! (l-a-k)!) cos^{2l+b-a-2k}(x/2) sin^{a-b+2k}(x/2).
__constant__ double c_invfact[41] = {1.0, 1.0, 0.5, 0.16666666666666666, 0.041666666666666664, 0.008333333333333333, 0.001388888888888889, 0.0001984126984126984, 2.48015873015873e-05, 2.7557319223985893e-06, 2.755731922398589e-07, 2.505210838544172e-08, 2.08767569878681e-09, 1.6059043836821613e-10, 1.1470745597729725e-11, 7.647163731819816e-13, 4.779477332387385e-14, 2.8114572543455206e-15, 1.5619206968586225e-16, 8.22063524662433e-18, 4.110317623312165e-19, 1.9572941063391263e-20, 8.896791392450574e-22, 3.868170170630684e-23, 1.6117375710961184e-24, 6.446950284384474e-26, 2.4795962632247976e-27, 9.183689863795546e-29, 3.279889237069838e-30, 1.1309962886447716e-31, 3.7699876288159054e-33, 1.216125041553518e-34, 3.8003907548547434e-36, 1.151633562077195e-37, 3.387157535521162e-39, 9.67759295863189e-41, 2.6882202662866363e-42, 7.265460179153071e-44, 1.911963205040282e-45, 4.902469756513544e-47, 1.2256174391283858e-48};

__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  while (n) { if (n & 1) r *= x; x *= x; n >>= 1; }
  return r;
}

// one warp: lane k takes the terms k, k + 32 of the sum; the partial sums are
// combined by a fixed xor tree (deterministic)
__device__ double swsh_theta_warp(int l, int m, double ch, double sh, int lane) {
  const int a = m, b = 2;
  // sqrt((l+a)!(l-a)!(l+b)!(l-b)!) = 1/sqrt(product of inverse factorials)
  const double root = rsqrt(c_invfact[l + a] * c_invfact[l - a] * c_invfact[l + b] * c_invfact[l - b]);
  double sum = 0.0;
  for (int k = lane; k <= 2 * l; k += 32) {
    const int f0 = l + b - k, f1 = k, f2 = a - b + k, f3 = l - a - k;
    if (f0 < 0 || f2 < 0 || f3 < 0) continue;
    double term = root * (c_invfact[f0] * c_invfact[f1]) * (c_invfact[f2] * c_invfact[f3]);
    term *= ipow(ch, 2 * l + b - a - 2 * k) * ipow(sh, a - b + 2 * k);
    sum += ((a - b + k) & 1) ? -term : term;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  // (-1)^s = +1 for s = -2
  return sqrt((2.0 * l + 1.0) / (2.0 * kTwoPi)) * sum;
}

// one warp per mode (the Wigner-d sums are short dependent FP64 chains: spread
// over lanes they overlap instead of running back to back in one thread)
__device__ __forceinline__ void modes_warp(long long j, int lane, int n_wf, const WfInfo* wf, const DevInputs& in,
                                           int conj, ModeInfo* modes, long long nm_total, int* status) {
  if (j >= nm_total) return;
  int lo = 0, hi = n_wf - 1;     // waveform holding mode j: last w with mo <= j
  while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (wf[mid].mo <= j) lo = mid; else hi = mid - 1; }
  const WfInfo W = wf[lo];
  const int l = in.l[j], m = in.m[j], n = in.n[j];
  ModeInfo M;
  M.wf = lo; M.l = l; M.m = m; M.n = n;
  M.seg_base = W.seg_base + (j - W.mo) * (W.K - 1);
  M.key_base = W.amp_base + (j - W.mo) * W.K;
  M.alpha = 0.0; M.beta = 0.0;
  const bool ok = (l >= 2 && l <= 20 && m >= -l && m <= l && (!conj || m >= 0) && n > -1000000 && n < 1000000);
  const double th = in.theta[lo];
  if (lane == 0 && (!finite(th) || !finite(in.phi[lo]) || !finite(in.prefactor[lo]))) atomicOr(status, ST_NONFINITE);
  if (!ok) {
    if (lane == 0) atomicOr(status, ST_MODE);
  } else {
    // c+ = alpha e^{i m phi}, cx = i beta e^{i m phi} (the e^{i m phi} goes into the phase)
    double sh, ch;
    sincos(0.5 * th, &sh, &ch);
    const double S = swsh_theta_warp(l, m, ch, sh, lane);
    if (conj) {
      const double Sp = swsh_theta_warp(l, -m, ch, sh, lane) * ((l & 1) ? -1.0 : 1.0);
      M.alpha = 0.5 * (S + Sp);
      M.beta = 0.5 * (S - Sp);
    } else {
      M.alpha = 0.5 * S;
      M.beta = 0.5 * S;
    }
  }
  if (lane == 0) {
    const ff a = ff_from_double(M.alpha), b = ff_from_double(M.beta);
    M.af[0] = a.hi; M.af[1] = a.lo; M.bf[0] = b.hi; M.bf[1] = b.lo;
    const bool amaj = alpha_major(M.alpha, M.beta);
    M.scale = amaj ? M.alpha : M.beta;
    M.rho = M.scale != 0.0 ? (amaj ? M.beta : M.alpha) / M.scale : 0.0;   // |rho| <= 1
    modes[j] = M;
  }
}

// --------------------------------------------------------- not-a-knot splines
// Unknowns: knot second derivatives M_0..M_{K-1}.  Interior rows (k=1..K-2):
//   h_{k-1} M_{k-1} + 2(h_{k-1}+h_k) M_k + h_k M_{k+1} = r_k,
//   r_k = 6[(y_{k+1}-y_k)/h_k - (y_k-y_{k-1})/h_{k-1}].
// Not-a-knot (third derivative continuous at t_1 and t_{K-2}) gives
//   M_0 = ((h0+h1) M_1 - h0 M_2)/h1,  M_{K-1} = ((ha+hb) M_{K-2} - hb M_{K-3})/ha
// (ha = h_{K-3}, hb = h_{K-2}); substituting them turns rows 1 and K-2 into
//   (h0 + 2 h1) M_1 + (h1 - h0) M_2 = r_1 h1/(h0+h1),
//   (ha - hb) M_{K-3} + (2 ha + hb) M_{K-2} = r_{K-2} ha/(ha+hb),
// a diagonally dominant tridiagonal system in M_1..M_{K-2}, solved by the
// Thomas algorithm.  The forward-sweep factors depend only on the knot times
// and are computed once per waveform.
__device__ __forceinline__ void tri_row(const double* t, int K, int i, double& a, double& b, double& c, double& scale) {
  double h0 = t[i] - t[i - 1], h1 = t[i + 1] - t[i];
  scale = 1.0;
  if (i == 1) { a = 0.0; b = h0 + 2.0 * h1; c = h1 - h0; scale = h1 / (h0 + h1); if (K == 4) {} }
  else if (i == K - 2) {
    double ha = h0, hb = h1;
    a = ha - hb; b = 2.0 * ha + hb; c = 0.0; scale = ha / (ha + hb);
  } else { a = h0; b = 2.0 * (h0 + h1); c = h1; }
}


// double-double product (Dekker/Knuth error-free transforms), for the knot
// phases Phi/(2 pi) in Q0.64 turns
struct dd { double hi, lo; };
__device__ __forceinline__ dd dd_two_prod(double a, double b) { dd r; r.hi = a * b; r.lo = fma(a, b, -r.hi); return r; }
__device__ __forceinline__ dd dd_fast(double s, double e) { dd r; r.hi = s + e; r.lo = e - (r.hi - s); return r; }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = dd_two_prod(a.hi, b.hi);
  return dd_fast(p.hi, p.lo + (a.hi * b.lo + a.lo * b.hi));
}

// knot frequency of mode (m, n) at knot i: the exact expression shared with
// the ownership rule, evaluated without contraction
__device__ __forceinline__ double knot_freq(int m, int n, double om_phi, double om_r) {
  return __ddiv_rn(__dadd_rn(__dmul_rn((double)m, om_phi), __dmul_rn((double)n, om_r)), kTwoPi);
}

// spline coefficients in u over [t_s, t_s + h]: a + b u + c u^2 + d u^3
__device__ __forceinline__ void ucoef(double y0, double y1, double M0, double M1, double h2, double* c) {
  c[0] = y0;
  c[1] = (y1 - y0) - h2 * (2.0 * M0 + M1) * (1.0 / 6.0);
  c[2] = 0.5 * h2 * M0;
  c[3] = h2 * (M1 - M0) * (1.0 / 6.0);
}

// the same coefficients times sc, with sc folded into the h^2 factors (k6 = sc h^2/6,
// k2 = sc h^2/2) instead of multiplying the four results
__device__ __forceinline__ void ucoef_scaled(double y0, double y1, double M0, double M1, double sc, double k6,
                                             double k2, double* c) {
  c[0] = sc * y0;
  c[1] = fma(-k6, fma(2.0, M0, M1), sc * (y1 - y0));
  c[2] = k2 * M0;
  c[3] = k6 * (M1 - M0);
}

// ---- warp-parallel forms of the two sequential sweeps (GB300's FP64 latency
// makes a 200-step dependent chain per thread slow, so each sweep is written as
// a scan over the warp: every lane composes its stretch of consecutive steps,
// the compositions are combined with a Hillis-Steele scan, and each lane then
// replays its stretch from the prefix).

// scale a pair/matrix by a power of two so that its largest entry is O(1)
__device__ __forceinline__ double pow2_of_max(double m) {
  const long long e = ((__double_as_longlong(m) >> 52) & 0x7FF);
  // 2^-(e-1023), clamped to the normal range
  const long long ee = e < 1 ? 1 : (e > 2045 ? 2045 : e);
  return __longlong_as_double((2046 - ee) << 52);
}

struct M22 { double a, b, c, d; };
__device__ __forceinline__ M22 m22_mul(const M22& X, const M22& Y) {   // X Y
  M22 r;
  r.a = fma(X.a, Y.a, X.b * Y.c); r.b = fma(X.a, Y.b, X.b * Y.d);
  r.c = fma(X.c, Y.a, X.d * Y.c); r.d = fma(X.c, Y.b, X.d * Y.d);
  const double sc = pow2_of_max(fmax(fmax(fabs(r.a), fabs(r.b)), fmax(fabs(r.c), fabs(r.d))));
  r.a *= sc; r.b *= sc; r.c *= sc; r.d *= sc;
  return r;
}
__device__ __forceinline__ M22 m22_shfl_up(const M22& X, int o) {
  M22 r;
  r.a = __shfl_up_sync(0xffffffffu, X.a, o); r.b = __shfl_up_sync(0xffffffffu, X.b, o);
  r.c = __shfl_up_sync(0xffffffffu, X.c, o); r.d = __shfl_up_sync(0xffffffffu, X.d, o);
  return r;
}

// per waveform (one warp): the forward-sweep factors {c'_i, 1/m_i, s_i/m_i, a_i/m_i}
// of the reduced system, and 1/h_k.  With v_i = (N_i, D_i) = M_i v_{i-1},
// M_i = [[0, c_i], [-a_i, b_i]], v_0 = (0, 1): c'_i = N_i / D_i and
// m_i = b_i - a_i c'_{i-1} = D_i / D_{i-1}.
__device__ __forceinline__ void factor_warp(int w, int lane, int n_wf, const WfInfo* wf, const double* tall, dbl4* fac,
                                            double* ih) {
  if (w >= n_wf) return;
  const WfInfo W = wf[w];
  const double* t = tall + W.ko;
  const int K = (int)W.K, n = K - 2;                 // unknowns i = 1..K-2
  for (int k = lane; k < K; k += 32) ih[W.ko + k] = (k + 1 < K) ? rcp_d(t[k + 1] - t[k]) : 0.0;
  if (lane == 0) {
    fac[W.ko] = mk_dbl4(0.0, 0.0, 0.0, 0.0);
    fac[W.ko + K - 1] = mk_dbl4(0.0, 0.0, 0.0, 0.0);
  }
  const int E = (n + 31) / 32;
  const int i0 = 1 + lane * E, i1 = min(i0 + E, n + 1);
  M22 Q = {1.0, 0.0, 0.0, 1.0};
  for (int i = i0; i < i1; i++) {
    double a, b, c, sc;
    tri_row(t, K, i, a, b, c, sc);
    const M22 Mi = {0.0, c, -a, b};
    Q = m22_mul(Mi, Q);
  }
  M22 S = Q;
  for (int o = 1; o < 32; o <<= 1) {
    const M22 X = m22_shfl_up(S, o);
    if (lane >= o) S = m22_mul(S, X);
  }
  M22 P = m22_shfl_up(S, 1);
  if (lane == 0) P = M22{1.0, 0.0, 0.0, 1.0};
  double N = P.b, D = P.d;                           // v_{i0-1} = P (0, 1)
  for (int i = i0; i < i1; i++) {
    double a, b, c, sc;
    tri_row(t, K, i, a, b, c, sc);
    const double Nn = c * D, Dn = fma(-a, N, b * D);
    const double inv = D * rcp_d(Dn);                // 1/m_i = D_{i-1}/D_i
    const double cc = (i == K - 2) ? 0.0 : c * inv;
    fac[W.ko + i] = mk_dbl4(cc, inv, sc * inv, a * inv);
    const double scl = pow2_of_max(fmax(fabs(Nn), fabs(Dn)));
    N = Nn * scl;
    D = Dn * scl;
  }
}

// one launch for the two independent first steps of the preparation: the spline
// factorisation (first fblocks blocks, a warp per waveform) and the per-mode records
// (a warp per mode)
__global__ void k_modes_factor(int n_wf, const WfInfo* wf, DevInputs in, int conj, ModeInfo* modes,
                               long long nm_total, int* status, dbl4* fac, double* ih, int fblocks) {
  const int lane = threadIdx.x & 31;
  if ((int)blockIdx.x < fblocks)
    factor_warp((int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane, n_wf, wf, in.t, fac, ih);
  else
    modes_warp(((blockIdx.x - fblocks) * (long long)blockDim.x + threadIdx.x) >> 5, lane, n_wf, wf, in, conj, modes,
               nm_total, status);
}

// affine map x -> p x + q; compose(g, f) = g after f
struct Aff { double p, q; };
__device__ __forceinline__ Aff aff_after(const Aff& g, const Aff& f) { Aff r; r.p = g.p * f.p; r.q = fma(g.p, f.q, g.q); return r; }

// right-hand side of row i times s_i/m_i: q_i = 6 [(y_{i+1}-y_i)/h_i - (y_i-y_{i-1})/h_{i-1}] s_i/m_i
__device__ __forceinline__ double rhs_q(const double* y, long long ys, const double* ih, const dbl4* fac, int i) {
  const double d1 = (y[(i + 1) * ys] - y[i * ys]) * ih[i];
  const double d0 = (y[i * ys] - y[(i - 1) * ys]) * ih[i - 1];
  return 6.0 * (d1 - d0) * fac[i].z;
}

// one warp per series: forward sweep rp_i = q_i - (a_i/m_i) rp_{i-1}, back
// substitution M_i = rp_i - c'_i M_{i+1}, both as warp scans of affine maps
__device__ void spline_solve_warp(int K, const double* y, long long ys, double* M, long long ms, const dbl4* fac,
                                  const double* ih, int lane) {
  const int n = K - 2;
  const int E = (n + 31) / 32;
  const int i0 = 1 + lane * E, i1 = min(i0 + E, n + 1);
  // forward (the right-hand sides are kept in M for the replay below)
  Aff F = {1.0, 0.0};
  for (int i = i0; i < i1; i++) {
    const double q = rhs_q(y, ys, ih, fac, i);
    M[i * ms] = q;
    const Aff f = {-fac[i].w, q};
    F = aff_after(f, F);
  }
  Aff S = F;
  for (int o = 1; o < 32; o <<= 1) {
    Aff X;
    X.p = __shfl_up_sync(0xffffffffu, S.p, o);
    X.q = __shfl_up_sync(0xffffffffu, S.q, o);
    if (lane >= o) S = aff_after(S, X);
  }
  double x = __shfl_up_sync(0xffffffffu, S.q, 1);   // exclusive prefix applied to rp_0 = 0
  if (lane == 0) x = 0.0;
  for (int i = i0; i < i1; i++) {
    x = fma(-fac[i].w, x, M[i * ms]);
    M[i * ms] = x;
  }
  __syncwarp();
  // backward, in decreasing i: x_i = rp_i - c'_i x_{i+1}, x_{K-1} = 0 (c'_{K-2} = 0)
  const int j0 = n - lane * E, j1 = max(j0 - E, 0);   // lane covers i = j0 .. j1+1 downwards
  Aff B = {1.0, 0.0};
  for (int i = j0; i > j1; i--) {
    const Aff f = {-fac[i].x, M[i * ms]};
    B = aff_after(f, B);
  }
  S = B;
  for (int o = 1; o < 32; o <<= 1) {
    Aff X;
    X.p = __shfl_up_sync(0xffffffffu, S.p, o);
    X.q = __shfl_up_sync(0xffffffffu, S.q, o);
    if (lane >= o) S = aff_after(S, X);
  }
  x = __shfl_up_sync(0xffffffffu, S.q, 1);
  if (lane == 0) x = 0.0;
  __syncwarp();
  for (int i = j0; i > j1; i--) {
    x = fma(-fac[i].x, x, M[i * ms]);
    M[i * ms] = x;
  }
  __syncwarp();
  if (lane == 0) {
    // M_0 = ((h0+h1) M_1 - h0 M_2)/h1 ;  M_{K-1} = ((ha+hb) M_{K-2} - hb M_{K-3})/ha
    const double r01 = ih[1] / ih[0];                      // h0 / h1
    M[0] = (1.0 + r01) * M[ms] - r01 * M[2 * ms];
    const double rba = ih[K - 3] / ih[K - 2];              // hb / ha
    M[(K - 1) * ms] = (1.0 + rba) * M[(K - 2) * ms] - rba * M[(K - 3) * ms];
  }
}

__global__ void k_spline_solve(int n_wf, const WfInfo* wf, const ModeInfo* modes, long long nm_total, DevInputs in,
                               const dbl4* fac, const double* ih, double* fundM, long long K_total, double* ampM,
                               FundSeg* fund) {
  long long sid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  long long nfund = 4LL * n_wf;
  if (sid < nfund) {
    int w = (int)(sid >> 2), which = (int)(sid & 3);
    const WfInfo W = wf[w];
    const double* y = which == 0 ? in.phi_phi : which == 1 ? in.phi_r : which == 2 ? in.omega_phi : in.omega_r;
    const double* ys = y + W.ko;
    const double* Ms = fundM + which * K_total + W.ko;
    spline_solve_warp((int)W.K, ys, 1, fundM + which * K_total + W.ko, 1, fac + W.ko, ih + W.ko, lane);
    __syncwarp();
    // per segment: this series' u-coefficients, and (Phi series) the knot phase in turns
    const double* t = in.t + W.ko;
    for (int s = lane; s + 1 < (int)W.K; s += 32) {
      const double h = t[s + 1] - t[s];
      double c[4];
      ucoef(ys[s], ys[s + 1], Ms[s], Ms[s + 1], h * h, c);
      FundSeg* F = fund + W.ko + s;
      // the fourth slot of the Phi_phi record carries sqrt(h), which every mode's
      // amplitude record of this segment needs (one square root per segment, not per mode)
      F->P[which] = mk_dbl4(c[1], c[2], c[3], which == 0 ? sqrt(h) : 0.0);
      dd x;
      if (which < 2) x = dd_mul(dd{ys[s], 0.0}, dd{kInv2PiHi, kInv2PiLo});
      else if (which == 2) x = dd_mul(dd{in.phi[w], 0.0}, dd{kInv2PiHi, kInv2PiLo});
      else x = dd{0.0, 0.0};
      F->q[which] = q64_of(x.hi) + q64_of(x.lo);
    }
    return;
  }
  sid -= nfund;
  if (sid >= 2 * nm_total) return;
  long long j = sid >> 1;
  int part = (int)(sid & 1);
  const ModeInfo Mi = modes[j];
  const WfInfo W = wf[Mi.wf];
  spline_solve_warp((int)W.K, in.amp + 2 * Mi.key_base + part, 2, ampM + 2 * Mi.key_base + part, 2, fac + W.ko,
                    ih + W.ko, lane);
}

// ------------------------------------------------ per (mode, segment) records
__device__ __forceinline__ void put_ff(float* dst, double x) {
  // hi rounded to nearest; x - hi is exact; lo truncated (|lo| <= |x - hi| <= ulp(hi)/2)
  const float hi = __double2float_rn(x);
  dst[0] = hi;
  dst[1] = d2f_bits(x - f2d_bits(hi));
}

__global__ void k_seg_prep(int n_wf, const WfInfo* wf, const ModeInfo* modes, DevInputs in, const FundSeg* fund, const double* ampM, long long seg_total, SegCore* core,
                           SegAmp64* amp64, SegAmp32* amp32, SegFF* segff, SegCrit* crit, long long* keyF,
                           double* yk) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= seg_total) return;
  int lo = 0, hi = n_wf - 1;
  while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (wf[mid].seg_base <= r) lo = mid; else hi = mid - 1; }
  const WfInfo W = wf[lo];
  long long rr = r - W.seg_base;
  long long Km1 = W.K - 1;
  long long j = W.mo + rr / Km1;
  int s = (int)(rr - (rr / Km1) * Km1);
  const ModeInfo Mi = modes[j];
  const int m = Mi.m, n = Mi.n;
  long long i0 = W.ko + s;
  const double ts = in.t[i0], h = in.t[i0 + 1] - ts, h2 = h * h;
  const FundSeg& Fs = fund[i0];
  const dbl4 cPp = Fs.P[0], cPr = Fs.P[1], cOp = Fs.P[2], cOr = Fs.P[3];
  const double dm = (double)m, dn = (double)n;
  SegCore C;
  C.A = knot_freq(m, n, in.omega_phi[i0], in.omega_r[i0]);
  C.b = fma(dm, cOp.x, dn * cOr.x) * kInv2PiHi;
  C.c = fma(dm, cOp.y, dn * cOr.y) * kInv2PiHi;
  C.d = fma(dm, cOp.z, dn * cOr.z) * kInv2PiHi;
  C.c2 = 2.0 * C.c;
  C.d3 = 3.0 * C.d;
  double P1 = fma(dm, cPp.x, dn * cPr.x) * kInv2PiHi;
  C.Q1 = fma(-C.A, h, P1);
  C.P2 = fma(dm, cPp.y, dn * cPr.y) * kInv2PiHi;
  C.P3 = fma(dm, cPp.z, dn * cPr.z) * kInv2PiHi;
  C.h = h;
  C.ts = ts;
  // theta0 = frac((m Phi_phi_s + n Phi_r_s - m phi)/2pi): integer combination of
  // the Q0.64 knot phases (wraps modulo one turn)
  C.theta0 = (unsigned long long)(long long)m * (Fs.q[0] - Fs.q[2]) + (unsigned long long)(long long)n * Fs.q[1];
  // mixed plans: minus frac(A t_s), exactly from the integer product of the mantissas, so
  // that their output kernel forms the phase from delta t = (g - A) t instead of g t
  if (amp32) C.theta0 -= q64_mul(C.A, ts);
  C.bf = d2f_bits(C.b); C.cf = d2f_bits(C.c); C.df = d2f_bits(C.d);   // truncated: start values only
  {
    const float r = C.bf != 0.f ? 1.f / C.bf : 0.f;   // FP32: it only scales the FP32 start value
    C.rbf = (fabsf(r) < 1e30f && fabsf(r) > 1e-30f) ? r : 0.f;
  }
  core[r] = C;
  if (yk) yk[r] = 0.47746482927568600731 / h;   // 3/(2 pi h), extended SPA

  // amplitude, scaled by prefactor sqrt(h) (the weight is sqrt(h)/sqrt|dF/du|); sqrt(h)
  // from the segment's fundamental record
  double sc = in.prefactor[lo] * cPp.w;
  const double* am = ampM + 2 * (Mi.key_base + s);
  const double* ay = in.amp + 2 * (Mi.key_base + s);
  double cre[4], cim[4];
  if (amp64) {   // FP64 records also carry the mode's polarisation scale
    SegAmp64 A;
    const double sc64 = sc * Mi.scale, sh2 = sc64 * h2, k6 = sh2 * (1.0 / 6.0), k2 = 0.5 * sh2;
    ucoef_scaled(ay[0], ay[2], am[0], am[2], sc64, k6, k2, A.re);
    ucoef_scaled(ay[1], ay[3], am[1], am[3], sc64, k6, k2, A.im);
    amp64[r] = A;
  } else {
    ucoef(ay[0], ay[2], am[0], am[2], h2, cre);
    ucoef(ay[1], ay[3], am[1], am[3], h2, cim);
  }
  if (amp32) {
    SegAmp32 A;
    for (int q = 0; q < 4; q++) { A.re[q] = (float)(sc * cre[q]); A.im[q] = (float)(sc * cim[q]); }
    amp32[r] = A;
  }
  if (segff) {
    SegFF X;
    put_ff(X.A, C.A); put_ff(X.b, C.b); put_ff(X.c, C.c); put_ff(X.d, C.d);
    put_ff(X.c2, C.c2); put_ff(X.d3, C.d3);
    put_ff(X.Q1, C.Q1); put_ff(X.P2, C.P2); put_ff(X.P3, C.P3); put_ff(X.h, h);
    const double sh = cPp.w;   // sqrt(h)
    for (int q = 0; q < 4; q++) { put_ff(X.are[q], sh * cre[q]); put_ff(X.aim[q], sh * cim[q]); }
    segff[r] = X;
  }

  // turnovers: roots of dF/du = b + 2c u + 3d u^2 in (0, 1)
  SegCrit X;
  X.n = 0; X.u[0] = X.u[1] = 0.0; X.F[0] = X.F[1] = 0.0; X.pad[0] = X.pad[1] = X.pad[2] = 0;
  // FP32 pre-check: dF/du = b + c2 u + d3 u^2 keeps one sign on [0, 1] when its end
  // values agree in sign and its vertex is outside [0, 1] or has that sign too
  // (margins of 1e-3 relative cover the FP32 rounding); otherwise solve exactly
  bool maybe = true;
  {
    const float fb = d2f_bits(C.b), fc2 = d2f_bits(C.c2), fd3 = d2f_bits(C.d3);
    const float D0 = fb, D1 = fb + fc2 + fd3;
    const float scl = fabsf(fb) + fabsf(fc2) + fabsf(fd3);
    if (D0 * D1 > 1e-3f * scl * scl) {
      if (fd3 == 0.f) maybe = false;
      else {
        const float uv = -fc2 / (2.f * fd3);
        if (uv < -1e-3f || uv > 1.001f) maybe = false;
        else {
          const float Dv = fb + uv * (fc2 + fd3 * uv);
          if (Dv * D0 > 1e-3f * scl * scl) maybe = false;
        }
      }
    }
  }
  if (maybe) {
    double qa = C.d3, qb = C.c2, qc = C.b;
    double rt[2]; int nr = 0;
    if (qa == 0.0) {
      if (qb != 0.0) rt[nr++] = -qc / qb;
    } else {
      double disc = qb * qb - 4.0 * qa * qc;
      if (disc >= 0.0) {
        double q = -0.5 * (qb + copysign(sqrt(disc), qb));
        if (q != 0.0) { rt[nr++] = q / qa; rt[nr++] = qc / q; }
        else rt[nr++] = 0.0;
      }
    }
    for (int i = 0; i < nr; i++)
      if (rt[i] > 0.0 && rt[i] < 1.0) X.u[X.n++] = rt[i];
    if (X.n == 2 && X.u[1] < X.u[0]) { double tmp = X.u[0]; X.u[0] = X.u[1]; X.u[1] = tmp; }
    if (X.n == 2 && X.u[1] == X.u[0]) X.n = 1;
    for (int i = 0; i < X.n; i++) {
      double u = X.u[i];
      X.F[i] = C.A + u * (C.b + u * (C.c + u * C.d));
    }
  }
  crit[r] = X;
  keyF[Mi.key_base + s] = ordkey(C.A);
  if (s == Km1 - 1) keyF[Mi.key_base + s + 1] = ordkey(knot_freq(m, n, in.omega_phi[i0 + 1], in.omega_r[i0 + 1]));
}

// ------------------------------------------------------------------ runs
// Sub-pieces of segment s: the monotone pieces between 0, its turnovers and 1.
// Their end frequencies are the knot expressions at u = 0, 1 and the cubic at
// turnovers.  A run is a maximal sequence of consecutive sub-pieces with the
// same (non-zero) direction; a flat piece (equal end frequencies) owns no
// frequency and separates runs.
struct SubPieces {
  int n;              // 1..3
  int dir[3];
  double ua[3], ub[3], Fa[3], Fb[3];
};

// (fixed indices and selects: X.n <= 2, so the pieces stay in registers)
__device__ __forceinline__ void sub_pieces(const SegCrit& X, double F0, double F1, SubPieces& P) {
  const bool c1 = X.n > 0, c2 = X.n > 1;
  P.n = X.n + 1;
  P.ua[0] = 0.0;      P.Fa[0] = F0;
  P.ub[0] = c1 ? X.u[0] : 1.0;  P.Fb[0] = c1 ? X.F[0] : F1;
  P.ua[1] = X.u[0];   P.Fa[1] = X.F[0];
  P.ub[1] = c2 ? X.u[1] : 1.0;  P.Fb[1] = c2 ? X.F[1] : F1;
  P.ua[2] = X.u[1];   P.Fa[2] = X.F[1];
  P.ub[2] = 1.0;      P.Fb[2] = F1;
#pragma unroll
  for (int i = 0; i < 3; i++) P.dir[i] = P.Fb[i] > P.Fa[i] ? 1 : (P.Fb[i] < P.Fa[i] ? -1 : 0);
}

// warp per mode; FILL=false counts runs into run_cnt, FILL=true writes them
template <bool FILL>
__global__ void k_runs(const WfInfo* wf, const ModeInfo* modes, long long nm_total, const SegCore* core,
                       const SegCrit* crit, const long long* keyF, const int* run_off, Run* runs, double2* runF, long long run_cap,
                       int* run_cnt, int* status) {
  long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= nm_total) return;
  const ModeInfo Mi = modes[j];
  const WfInfo W = wf[Mi.wf];
  const int nseg = (int)(W.K - 1);
  int carry_dir = 0;          // direction of the last sub-piece before this chunk
  int carry_cnt = 0;          // runs started before this chunk
  long long base = FILL ? (long long)run_off[j] : 0;
  for (int c0 = 0; c0 < nseg; c0 += 32) {
    int s = c0 + lane;
    bool valid = s < nseg;
    SubPieces P; P.n = 0;
    if (valid) {
      const SegCore C = core[Mi.seg_base + s];
      const SegCrit X = crit[Mi.seg_base + s];
      // segment end frequency: the knot expression F_V(t_{s+1}), kept as a key
      double F1 = unordkey(keyF[Mi.key_base + s + 1]);
      sub_pieces(X, C.A, F1, P);
    }
    int first_dir = (valid && P.n > 0) ? P.dir[0] : 0;
    int last_dir = (valid && P.n > 0) ? (P.n == 1 ? P.dir[0] : P.n == 2 ? P.dir[1] : P.dir[2]) : 0;
    int prev_last = __shfl_up_sync(0xffffffffu, last_dir, 1);
    if (lane == 0) prev_last = carry_dir;
    int next_first = __shfl_down_sync(0xffffffffu, first_dir, 1);
    if (lane == 31 || s + 1 >= nseg) next_first = 0;   // next chunk's first handled by its own start test
    int starts = 0;
    int pd = prev_last;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      if (i >= P.n) break;
      if (P.dir[i] != 0 && P.dir[i] != pd) starts++;
      pd = P.dir[i];
    }
    // inclusive warp scan of starts
    int incl = starts;
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int excl = incl - starts;
    int total = __shfl_sync(0xffffffffu, incl, 31);
    if (FILL && valid) {
      int idx = carry_cnt + excl;     // runs started before this segment (within the mode)
      pd = prev_last;
#pragma unroll
      for (int i = 0; i < 3; i++) {
        if (i >= P.n) break;
        int d = P.dir[i];
        if (d != 0 && d != pd) {
          long long rid = base + idx;
          if (rid < run_cap) {
            // start fields only: the end fields may be written by another lane
            runs[rid].mode = (int)j;
            runs[rid].dir = d;
            runs[rid].s0 = s;
            runs[rid].u0 = P.ua[i];
            const ff uu = ff_from_double(P.ua[i]);
            runs[rid].u0f[0] = uu.hi;
            runs[rid].u0f[1] = uu.lo;
            runF[rid].x = P.Fa[i];
          }
          idx++;
        }
        // end of a run: next sub-piece (in this segment or the next) has another direction
        int nd = (i + 1 < P.n) ? P.dir[i < 2 ? i + 1 : 2] : (s + 1 < nseg ? -2 : 0);
        bool ends;
        if (nd == -2) {
          // first sub-piece of segment s+1: taken from the next lane, or re-derived at a chunk edge
          int nf = next_first;
          if (lane == 31) {
            const SegCore C2 = core[Mi.seg_base + s + 1];
            const SegCrit X2 = crit[Mi.seg_base + s + 1];
            double F2 = unordkey(keyF[Mi.key_base + s + 2]);
            SubPieces P2; sub_pieces(X2, C2.A, F2, P2);
            nf = P2.dir[0];
          }
          ends = (d != 0 && nf != d);
        } else {
          ends = (d != 0 && nd != d);
        }
        if (ends) {
          long long rid = base + idx - 1;
          if (rid < run_cap) {
            runs[rid].s1 = s;
            runs[rid].u1 = P.ub[i];
            const ff uu = ff_from_double(P.ub[i]);
            runs[rid].u1f[0] = uu.hi;
            runs[rid].u1f[1] = uu.lo;
            runF[rid].y = P.Fb[i];
          }
        }
        pd = d;
      }
    }
    carry_cnt += total;
    carry_dir = __shfl_sync(0xffffffffu, last_dir, 31);
    if (c0 + 32 > nseg) {
      // the chunk was partial: the true last direction is at lane nseg-1-c0
      carry_dir = __shfl_sync(0xffffffffu, last_dir, (nseg - 1 - c0) & 31);
    }
  }
  if (!FILL && lane == 0) run_cnt[j] = carry_cnt;
  if (FILL && lane == 0 && base + carry_cnt > run_cap) atomicOr(status, ST_CAPACITY);
}

// exclusive scan of cnt[0..n) in place, total written to cnt[n]; one block
__global__ void k_scan(int* cnt, long long n) {
  __shared__ long long part[1024];
  int tid = threadIdx.x;
  long long per = (n + blockDim.x - 1) / blockDim.x;
  long long b = tid * per, e = b + per < n ? b + per : n;
  long long s = 0;
  for (long long i = b; i < e; i++) s += cnt[i];
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    long long v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  long long run = part[tid] - s;
  for (long long i = b; i < e; i++) { long long c = cnt[i]; cnt[i] = (int)run; run += c; }
  if (tid == blockDim.x - 1) cnt[n] = (int)part[tid];
}

__global__ void k_wf_runs(int n_wf, WfInfo* wf, const int* run_off, long long run_cap) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_wf) return;
  long long a = run_off[wf[w].mo], b = run_off[wf[w].mo + wf[w].nm];
  if (a > run_cap) a = run_cap;
  if (b > run_cap) b = run_cap;
  wf[w].run_base = a;
  wf[w].nruns = b - a;
  wf[w].occ_lo = (int)(wf[w].fo + wf[w].nf);   // empty until k_run_bins widens it
  wf[w].occ_hi = (int)wf[w].fo;
}

// Output-bin ranges of each run.  Increasing runs own [F_start, F_end),
// decreasing runs own (F_end, F_start]; the negative-frequency part serves
// bins f with -f in that range (they enter through conj H(-f)).
// One warp per run: four groups of 8 lanes find the four bounds at once, each
// with an 8-way search (8 probes per step, integer keys of the doubles).
// bound of group g: first i in [0, n) with key(f[i]) >= x (strict: > x)
__device__ __forceinline__ long long group_bound(const long long* fk, long long n, long long x, bool strict, int j,
                                                 unsigned gmask) {
  long long lo = 0, hi = n;   // answer in [lo, hi]
  while (hi - lo > 8) {
    const long long span = hi - lo;
    const long long p = lo + (span * (j + 1)) / 9;
    const long long v = fk[p];
    const bool pr = strict ? (v > x) : (v >= x);
    const unsigned bal = __ballot_sync(gmask, pr) & gmask;
    // probes of this group sit at bit offsets (lane & ~7) .. +7
    const unsigned mine = bal >> (threadIdx.x & 24);
    const int first = mine ? __ffs(mine) - 1 : 8;
    const long long pl = first > 0 ? lo + (span * first) / 9 : lo - 1;        // probe before the first true
    const long long ph = first < 8 ? lo + (span * (first + 1)) / 9 : hi;       // first true probe
    lo = (first > 0) ? pl + 1 : lo;
    hi = ph;
  }
  // at most 8 candidates left: lo .. hi-1, answer = first true or hi
  const long long p = lo + j;
  bool pr = false;
  if (p < hi) {
    const long long v = fk[p];
    pr = strict ? (v > x) : (v >= x);
  }
  const unsigned bal = (__ballot_sync(gmask, pr) & gmask) >> (threadIdx.x & 24);
  return bal ? lo + (__ffs(bal) - 1) : hi;
}

__global__ void k_run_bins(WfInfo* wf, const ModeInfo* modes, long long nm_total, const int* run_total,
                           const Run* runs, const double2* runF, long long run_cap, const double* freqs, RunBins* rb,
                           unsigned long long* counters, int* status) {
  const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, grp = lane >> 3, j = lane & 7;
  long long nr = *run_total;
  if (nr > run_cap) nr = run_cap;
  if (r >= nr) return;
  const Run R = runs[r];
  RunBins B;
  // a run whose fields were not all written (cannot happen when the count and
  // fill passes agree) is made empty, so that no later kernel indexes with it
  if (R.mode < 0 || R.mode >= nm_total) {
    if (lane == 0) {
      B.b0p = B.b1p = B.b0n = B.b1n = 0;
      rb[r] = B;
      atomicOr(status, ST_CAPACITY);
    }
    return;
  }
  const int wi = modes[R.mode].wf;
  const WfInfo W = wf[wi];
  if (R.s0 < 0 || R.s1 < R.s0 || R.s1 >= W.K - 1 || R.dir == 0) {
    if (lane == 0) {
      B.b0p = B.b1p = B.b0n = B.b1n = (int)W.fo;
      rb[r] = B;
      atomicOr(status, ST_CAPACITY);
    }
    return;
  }
  const long long* fk = reinterpret_cast<const long long*>(freqs) + W.fo;   // positive: bits are ordered keys
  const double Fs = runF[r].x, Fe = runF[r].y;
  // group 0..3: (b0p, b1p, b0n, b1n); lower bound = first f >= x, upper = first f > x
  double x;
  bool strict;
  if (R.dir > 0) {
    x = grp == 0 ? Fs : grp == 1 ? Fe : grp == 2 ? -Fe : -Fs;
    strict = grp >= 2;
  } else {
    x = grp == 0 ? Fe : grp == 1 ? Fs : grp == 2 ? -Fs : -Fe;
    strict = grp <= 1;
  }
  const unsigned gmask = 0xFFu << (grp * 8);
  const long long v = group_bound(fk, W.nf, ordkey(x), strict, j, gmask);
  const long long b0p = __shfl_sync(0xffffffffu, v, 0), b1p = __shfl_sync(0xffffffffu, v, 8);
  const long long b0n = __shfl_sync(0xffffffffu, v, 16), b1n = __shfl_sync(0xffffffffu, v, 24);
  if (lane == 0) {
    const long long e1p = b1p < b0p ? b0p : b1p, e1n = b1n < b0n ? b0n : b1n;
    B.b0p = (int)(W.fo + b0p); B.b1p = (int)(W.fo + e1p);
    B.b0n = (int)(W.fo + b0n); B.b1n = (int)(W.fo + e1n);
    rb[r] = B;
    unsigned long long cnt = (unsigned long long)((e1p - b0p) + (e1n - b0n));
    if (cnt) atomicAdd(&counters[1], cnt);
    // the waveform's occupied bin range, so that the output kernel skips the run
    // scan for tiles no run reaches
    if (e1p > b0p) { atomicMin(&wf[wi].occ_lo, B.b0p); atomicMax(&wf[wi].occ_hi, B.b1p); }
    if (e1n > b0n) { atomicMin(&wf[wi].occ_lo, B.b0n); atomicMax(&wf[wi].occ_hi, B.b1n); }
  }
}

__global__ void k_table(double2* tab) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kTab64N) return;
  double s, c;
  sincospi((double)k / (double)(kTab64N / 2), &s, &c);
  tab[k] = make_double2(c, s);
}

}  // namespace

void launch_table(double2* tab, cudaStream_t st) { k_table<<<(kTab64N + 255) / 256, 256, 0, st>>>(tab); }

namespace {
__global__ void k_table_ff(const double2* tab, float4* tabf) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kTabN) return;
  static_assert(kTabBits <= kTab64Bits, "the FP32-pair table samples the FP64 table");
  const double2 e = tab[(long long)k << (kTab64Bits - kTabBits)];   // e^{2 pi i k / kTabN}
  const ff c = ff_from_double(e.x), s = ff_from_double(e.y);
  tabf[k] = make_float4(c.hi, c.lo, s.hi, s.lo);
}
}  // namespace

void launch_table_ff(const double2* tab, float4* tabf, cudaStream_t st) {
  k_table_ff<<<(kTabN + 255) / 256, 256, 0, st>>>(tab, tabf);
}

void launch_scan(int* cnt, long long n, cudaStream_t st) { k_scan<<<1, 1024, 0, st>>>(cnt, n); }

// TD comparator: per (mode, segment) FP32 u-coefficients of Re A and Im A
// (unscaled: the prefactor is applied when the samples are stored)
__global__ void k_td_amp(int n_wf, const WfInfo* wf, const ModeInfo* modes, DevInputs in, const double* ampM,
                         long long seg_total, float4* tdamp) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= seg_total) return;
  int lo = 0, hi = n_wf - 1;
  while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (wf[mid].seg_base <= r) lo = mid; else hi = mid - 1; }
  const WfInfo W = wf[lo];
  const long long rr = r - W.seg_base, Km1 = W.K - 1;
  const long long j = W.mo + rr / Km1;
  const int s = (int)(rr - (rr / Km1) * Km1);
  const ModeInfo Mi = modes[j];
  const long long i0 = W.ko + s;
  const double h = in.t[i0 + 1] - in.t[i0], h2 = h * h;
  const double* am = ampM + 2 * (Mi.key_base + s);
  const double* ay = in.amp + 2 * (Mi.key_base + s);
  double cre[4], cim[4];
  ucoef(ay[0], ay[2], am[0], am[2], h2, cre);
  ucoef(ay[1], ay[3], am[1], am[3], h2, cim);
  tdamp[2 * r] = make_float4((float)cre[0], (float)cre[1], (float)cre[2], (float)cre[3]);
  tdamp[2 * r + 1] = make_float4((float)cim[0], (float)cim[1], (float)cim[2], (float)cim[3]);
}

static void launch_modes_factor(const CallShape& cs, const DevInputs& in, const DevScratch& s, cudaStream_t st) {
  const int fblocks = (cs.n_wf * 32 + 255) / 256;
  const long long mblocks = (cs.nm_total * 32 + 255) / 256;
  k_modes_factor<<<(unsigned)(fblocks + mblocks), 256, 0, st>>>(cs.n_wf, s.wf, in, cs.conj, s.modes, cs.nm_total,
                                                                s.status, s.spl_fac, s.spl_ih, fblocks);
}

void launch_prep_td(const CallShape& cs, const DevInputs& in, const DevScratch& s, float4* tdamp, cudaStream_t st) {
  dim3 gk(8, cs.n_wf);
  k_validate_knots<<<gk, 256, 0, st>>>(s.wf, in, s.status);
  k_validate_amp<<<256, 256, 0, st>>>(2 * cs.amp_total, in.amp, s.status);
  launch_modes_factor(cs, in, s, st);
  long long nser = 4LL * cs.n_wf + 2 * cs.nm_total;
  k_spline_solve<<<(unsigned)((nser * 32 + 255) / 256), 256, 0, st>>>(cs.n_wf, s.wf, s.modes, cs.nm_total, in, s.spl_fac,
                                                                 s.spl_ih, s.fundM, cs.K_total, s.ampM, s.fund);
  k_td_amp<<<(unsigned)((cs.seg_total + 127) / 128), 128, 0, st>>>(cs.n_wf, s.wf, s.modes, in, s.ampM, cs.seg_total,
                                                                   tdamp);
}

void launch_prep(const CallShape& cs, const DevInputs& in, const DevScratch& s, cudaStream_t st,
                 cudaEvent_t freqs_ready) {
  dim3 gk(8, cs.n_wf);
  k_validate_knots<<<gk, 256, 0, st>>>(s.wf, in, s.status);
  k_validate_amp<<<256, 256, 0, st>>>(2 * cs.amp_total, in.amp, s.status);
  launch_modes_factor(cs, in, s, st);
  long long nser = 4LL * cs.n_wf + 2 * cs.nm_total;
  k_spline_solve<<<(unsigned)((nser * 32 + 255) / 256), 256, 0, st>>>(cs.n_wf, s.wf, s.modes, cs.nm_total, in, s.spl_fac,
                                                                 s.spl_ih, s.fundM, cs.K_total, s.ampM, s.fund);
  k_seg_prep<<<(unsigned)((cs.seg_total + 127) / 128), 128, 0, st>>>(
      cs.n_wf, s.wf, s.modes, in, s.fund, s.ampM, cs.seg_total, s.core,
      cs.precision == 0 ? s.amp64 : nullptr, cs.precision == 1 ? s.amp32 : nullptr,
      cs.precision == 2 ? s.segff : nullptr, s.crit, s.keyF, cs.ext && cs.precision == 0 ? s.yk : nullptr);
  unsigned wblocks = (unsigned)((cs.nm_total * 32 + 255) / 256);
  k_runs<false><<<wblocks, 256, 0, st>>>(s.wf, s.modes, cs.nm_total, s.core, s.crit, s.keyF, nullptr, nullptr,
                                         nullptr, s.run_cap, s.run_cnt, s.status);
  k_scan<<<1, 1024, 0, st>>>(s.run_cnt, cs.nm_total);
  k_wf_runs<<<(cs.n_wf + 63) / 64, 64, 0, st>>>(cs.n_wf, s.wf, s.run_cnt, s.run_cap);
  cudaMemsetAsync(s.runs, 0xFF, sizeof(Run) * (size_t)s.run_cap, st);
  // the frequency grid is first read here (it may still be arriving on another stream)
  if (freqs_ready) cudaStreamWaitEvent(st, freqs_ready, 0);
  // about one bin per thread per waveform, at most 1216 CTAs (8 per SM of a 152-SM GB300)
  long long gx = (cs.nf_total / (cs.n_wf > 0 ? cs.n_wf : 1) + 255) / 256;
  gx = gx < 1 ? 1 : (gx > 1216 ? 1216 : gx);
  dim3 gf((unsigned)gx, cs.n_wf);
  k_validate_freqs<<<gf, 256, 0, st>>>(s.wf, in, s.status);
  k_runs<true><<<wblocks, 256, 0, st>>>(s.wf, s.modes, cs.nm_total, s.core, s.crit, s.keyF, s.run_cnt, s.runs,
                                        s.runF, s.run_cap, nullptr, s.status);
  k_run_bins<<<(unsigned)((s.run_cap * 32 + 255) / 256), 256, 0, st>>>(s.wf, s.modes, cs.nm_total, s.run_cnt + cs.nm_total,
                                                                  s.runs, s.runF, s.run_cap, in.freqs, s.rbins,
                                                                  s.counters, s.status);
}

}  // namespace emrifd
