// Internal definitions of the GB300 SPA mode-sum library (not part of the C ABI).
//
// Data layout in HBM, per call (all plan-owned scratch, sized at plan creation):
//   WfInfo[n_wf]             per-waveform slice offsets and derived bases
//   ModeInfo[sum N_m]        per-mode numbers, waveform id, polarisation weights
//   spl_fac, spl_ih          per-knot factors of each waveform's not-a-knot system
//   fundM[4][sum K]          knot second derivatives of Phi_phi, Phi_r, Om_phi, Om_r
//   ampM[sum N_m K][2]       knot second derivatives of Re A, Im A
//   SegCore[sum N_m (K-1)]   per (mode, segment): frequency cubic, phase polynomial,
//                            Q0.64 phase offset (112 B, 16-B aligned)
//   SegAmp64/SegAmp32        per (mode, segment): amplitude cubic (FP64 or FP32 copy)
//   SegCrit                  per (mode, segment): turnover points of F_V
//   keyF[sum N_m K]          ordered int64 keys of the knot frequencies F_V(t_k)
//   Run[...]                 monotone branches ("runs") of every voice track,
//   RunBins[...]             and their output-bin ranges (int32, for the tile scan)
//
// Conventions: u = (t - t_s)/h_s is the normalised time inside segment s;
// every per-segment polynomial is in u.  Phases in the hot loop are Q0.64
// fixed-point turns (uint64; wrap-around addition is addition mod 1 turn).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace emrifd {

constexpr int kWarps = 8;                 // warps per CTA of the hot kernel
constexpr int kThreads = 32 * kWarps;
#ifndef EMRI_FD_TABFF_BITS
#define EMRI_FD_TABFF_BITS 16
#endif
constexpr int kTabBits = EMRI_FD_TABFF_BITS;   // FP32-pair table e^{2 pi i k / 2^kTabBits} (FP64X form)
constexpr int kTabN = 1 << kTabBits;
constexpr int kTab64Bits = 16;            // FP64 table e^{2 pi i k / 65536} (FP64 form, adjoint)
constexpr int kTab64N = 1 << kTab64Bits;
constexpr int kListCap = 2048;            // (run, sign) entries buffered per tile pass

// status bits latched in the plan's device status word (no kernel of this library
// waits on a flag, a peer or a barrier it does not own, so none has a timeout bit);
// ST_BOUNDS is latched only by the index checks of checked builds (below)
enum : int {
  ST_KNOTS = 1, ST_FREQ = 2, ST_MODE = 4, ST_NONFINITE = 8, ST_CAPACITY = 16, ST_BOUNDS = 32
};

// Checked builds (-DEMRI_FD_CHECKS=1) test the indices the hot kernels derive from the
// device-built run lists (run, mode, segment, bin) against their arrays.  A failed check
// latches ST_BOUNDS and the access is skipped; nothing traps, so the context stays usable
// and the call reports EMRI_FD_ERR_INTERNAL.  In normal builds the checks compile away.
#ifndef EMRI_FD_CHECKS
#define EMRI_FD_CHECKS 0
#endif
__device__ __forceinline__ bool check_fails(bool ok, const int* status) {
#if EMRI_FD_CHECKS
  if (!ok) {
    atomicOr(const_cast<int*>(status), ST_BOUNDS);
    return true;
  }
#else
  (void)ok;
  (void)status;
#endif
  return false;
}

struct WfInfo {
  long long ko, K;         // knot slice
  long long mo, nm;        // mode slice
  long long fo, nf;        // bin slice
  long long amp_base;      // first amplitude knot (complex index) = sum_{w'<w} N_m K
  long long seg_base;      // first (mode, segment) record = sum_{w'<w} N_m (K-1)
  long long tile_base, ntiles;
  long long run_base, nruns;  // filled on the device
  int occ_lo, occ_hi;         // global bins [occ_lo, occ_hi) some run covers (filled on the device)
};

struct ModeInfo {
  int wf, l, m, n;
  long long seg_base;      // first record of this mode
  long long key_base;      // first knot key / amplitude knot of this mode
  double alpha, beta;      // h+ += alpha Z, hx += i beta Z (positive branch), see spa.cu
  float af[2], bf[2];      // alpha, beta as FP32 pairs (hi, lo)
  // FP64 records: the amplitude is stored times scale, the one of alpha, beta of larger
  // magnitude (alpha_major), and rho = the other over it (0 when both are 0), so that
  // alpha Z and beta Z take one multiply by rho instead of two by alpha and beta
  double scale, rho;
};
static_assert(sizeof(ModeInfo) == 80, "ModeInfo layout");

struct __align__(16) SegCore {
  double A;                // F_V(t_s), knot expression (m*Om_phi_s + n*Om_r_s)/(2 pi)  [Hz]
  double b, c, d;          // F(u) - A = b u + c u^2 + d u^3                           [Hz]
  double c2, d3;           // 2c, 3d  (dF/du = b + c2 u + d3 u^2)
  double Q1, P2, P3;       // phase inside the segment, in turns:
                           //   g t - Phi_V(t)/2pi = g t_s - Phi_V(t_s)/2pi + u (delta h - Q1 - u (P2 + u P3))
                           //   with delta = g - A
  double h;                // segment length [s]
  double ts;               // segment start time [s]
  unsigned long long theta0; // Q0.64 of frac(Phi_V(t_s)/2pi - m phi/2pi)
  float bf, cf, df;        // FP32 copies of b, c, d for the root's initial guess
  float rbf;               // 1/b in FP32 (0 when b is 0 or 1/b is not a finite float)
};
static_assert(sizeof(SegCore) == 112, "SegCore layout");

struct __align__(32) dbl4 { double x, y, z, w; };
__host__ __device__ __forceinline__ dbl4 mk_dbl4(double x, double y, double z, double w) {
  dbl4 r; r.x = x; r.y = y; r.z = z; r.w = w; return r;
}

struct __align__(16) SegAmp64 { double re[4], im[4]; };   // prefactor sqrt(h) A(u), cubic in u
struct __align__(16) SegAmp32 { float re[4], im[4]; };
struct __align__(16) SegCrit { double u[2]; double F[2]; int n; int pad[3]; };  // 48 B

// FP64X records: the SegCore polynomials as FP32 pairs (hi, lo), and the
// amplitude cubic times sqrt(h) (no prefactor, applied at the store)
struct __align__(16) SegFF {
  float A[2], b[2], c[2], d[2];      // frequency cubic [Hz]
  float c2[2], d3[2];                // 2c, 3d
  float Q1[2], P2[2], P3[2], h[2];   // in-segment phase [turns], segment length [s]
  float are[4][2], aim[4][2];        // sqrt(h) A(u)
};
static_assert(sizeof(SegFF) == 144, "SegFF layout");

struct __align__(16) Run {
  int mode, dir, s0, s1;   // global mode index; +1/-1; first/last segment (local)
  double u0, u1;           // start u in s0, end u in s1
  float u0f[2], u1f[2];    // the same as FP32 pairs (hi, lo)
};
struct __align__(16) RunBins { int b0p, b1p, b0n, b1n; };  // global output bins, [b0, b1)

// ----------------------------------------------------------------------------
// small device helpers (integer work only unless stated)
// ----------------------------------------------------------------------------
__device__ __forceinline__ long long ordkey(double x) {
  // monotone map of doubles to signed int64 (non-NaN); -0 < +0
  long long u = __double_as_longlong(x);
  return u ^ ((u >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ double unordkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

__device__ __forceinline__ double abs_bits(double x) {
  // |x| through the sign bit (fabs of a value that is also used bit-wise costs an FP64 add)
  return __hiloint2double(__double2hiint(x) & 0x7FFFFFFF, __double2loint(x));
}

__device__ __forceinline__ bool is_zero_bits(double x) {
  // x == +-0 from the two words (a test on the 64-bit pattern becomes an FP64 compare)
  return ((__double2hiint(x) & 0x7FFFFFFF) | __double2loint(x)) == 0;
}

__device__ __forceinline__ double flip_sign(double x) {
  // -x through the sign bit (an integer operation, not an FP64 instruction)
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// |alpha| >= |beta|, compared through the bits of the magnitudes (integer order is
// numeric order for non-negative doubles); the same test wherever ModeInfo.scale is used
__device__ __forceinline__ bool alpha_major(double alpha, double beta) {
  return (__double_as_longlong(alpha) & 0x7FFFFFFFFFFFFFFFll) >= (__double_as_longlong(beta) & 0x7FFFFFFFFFFFFFFFll);
}

__device__ __forceinline__ float d2f_bits(double x) {
  // double -> float by truncation, through the bit fields (no FP64-pipe conversion);
  // values below the float normal range become 0
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  int e = (int)((u >> 52) & 0x7FF) - 1023 + 127;
  unsigned s = (unsigned)(u >> 32) & 0x80000000u;
  if (e <= 0) return __uint_as_float(s);
  if (e >= 255) return __uint_as_float(s | 0x7F800000u | (unsigned)((u >> 29) & 0x7FFFFF));
  return __uint_as_float(s | ((unsigned)e << 23) | (unsigned)((u >> 29) & 0x7FFFFF));
}

__device__ __forceinline__ double f2d_bits(float x) {
  // exact float -> double through the bit fields; float denormals become 0
  unsigned u = __float_as_uint(x);
  unsigned e = (u >> 23) & 0xFF;
  unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0) return __longlong_as_double((long long)s);
  unsigned long long ed = (e == 255) ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(s | (ed << 52) | ((unsigned long long)(u & 0x7FFFFF) << 29)));
}

// reciprocal of a normal double from an FP32 seed and two FP64 Newton steps
__device__ __forceinline__ double rcp_d(double x) {
  const float xf = d2f_bits(x);
  const float yf = __fdividef(1.f, xf);
  if (!(fabsf(yf) > 0.f && fabsf(yf) < 3.0e38f)) return 1.0 / x;
  double y = f2d_bits(yf);
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// frac(x) in Q0.64 turns (x in turns), by the bit fields of x
__device__ __forceinline__ unsigned long long q64_of(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  int e = (int)((u >> 52) & 0x7FF);
  if (e == 0) return 0ull;
  unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  int sh = e - 1075 + 64;             // value * 2^64 = m * 2^sh
  unsigned long long r;
  if (sh >= 64) r = 0ull;
  else if (sh >= 0) r = m << sh;
  else if (sh > -64) r = m >> (-sh);
  else r = 0ull;
  return (u >> 63) ? (0ull - r) : r;
}

// exact float of a small integer (|v| < 2^22) without a conversion instruction:
// 1.5 * 2^23 + v has v in its low mantissa bits
__device__ __forceinline__ float small_int_to_float(int v) {
  return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}

// frac(a * b) in Q0.64 turns, from the exact 106-bit product of the mantissas
__device__ __forceinline__ unsigned long long q64_mul(double a, double b) {
  unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  int ea = (int)((ua >> 52) & 0x7FF), eb = (int)((ub >> 52) & 0x7FF);
  if (ea == 0 || eb == 0) return 0ull;
  unsigned long long ma = (ua & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  unsigned long long mb = (ub & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  unsigned long long lo = ma * mb, hi = __umul64hi(ma, mb);
  int sh = ea + eb - 2150 + 64;       // product * 2^64 = (hi:lo) * 2^sh
  unsigned long long r;
  if (sh >= 64) r = 0ull;
  else if (sh > 0) r = lo << sh;
  else if (sh == 0) r = lo;
  else if (sh > -64) r = (lo >> (-sh)) | (hi << (64 + sh));
  else if (sh == -64) r = hi;
  else if (sh > -128) r = hi >> (-sh - 64);
  else r = 0ull;
  return ((ua ^ ub) >> 63) ? (0ull - r) : r;
}

// ----------------------------------------------------------------------------
// launchers (defined in prep.cu / spa.cu), all on `st`
// ----------------------------------------------------------------------------
struct Scratch;  // defined in emri_fd.cu

struct DevInputs {
  const double *t, *phi_phi, *phi_r, *omega_phi, *omega_r;
  const int *l, *m, *n;
  const double* amp;
  const double *theta, *phi, *prefactor;
  const double* freqs;
  void *h_plus, *h_cross;
};

// per knot segment of a waveform: the u-coefficients (c1, c2, c3, .) of the four
// fundamental series (Phi_phi, Phi_r, Omega_phi, Omega_r; the fourth slot holds
// sqrt(h) in the Phi_phi record and 0 in the others) and, as Q0.64 turns,
// frac(Phi_phi_s / 2 pi), frac(Phi_r_s / 2 pi) and frac(phi / 2 pi)
struct FundSeg {
  dbl4 P[4];
  unsigned long long q[4];
};
static_assert(sizeof(FundSeg) == 160, "FundSeg layout");

struct DevScratch {
  int* status;
  unsigned long long* counters;   // [0] tile queue, [1] mode-bins, [2] runs total, [3] busy tiles
  WfInfo* wf;
  ModeInfo* modes;
  dbl4* spl_fac;               // [sum K] {c'_i, 1/m_i, s_i/m_i, a_i/m_i} of each waveform's not-a-knot sweep
  double* spl_ih;                 // [sum K] 1/h_k
  double* fundM;                  // [4][sum K]
  FundSeg* fund;                  // [sum K]
  double* ampM;                   // [sum N_m K][2]
  SegCore* core;
  SegAmp64* amp64;
  SegAmp32* amp32;
  SegFF* segff;                   // FP64X plans
  SegCrit* crit;
  double* yk;                     // [sum N_m (K-1)] 3/(2 pi h), extended FP64 plans
  void *wbuf_p, *wbuf_c;          // [sum N_f] unwindowed h+, hx (windowed plans)
  long long* keyF;                // [sum N_m K]
  int* run_cnt;                   // [sum N_m + 1], exclusive-scanned in place
  Run* runs;
  double2* runF;                  // [run_cap] (F at run start, F at run end)
  RunBins* rbins;
  long long run_cap;
  double2* tab;                   // [kTab64N] e^{2 pi i k / kTab64N}
  float4* tabf;                   // [kTabN] the same as FP32 pairs (cos hi, cos lo, sin hi, sin lo), FP64X plans
  // likelihood / adjoint scratch (plans created with likelihood = 1)
  double* hbuf;                   // [2][sum N_f] complex128: h+ then hx
  double* Gbuf;                   // [sum N_f][4] 4 df (d - h)/S, both channels
  double* Lpart;                  // [max_waveforms][kLChunks] partial sums of L
  int* item_off;                  // [run_cap + 1] adjoint items (run, segment), scanned
  void* adj_items;                // [3 seg_cap] AdjItem records (adjoint.cu)
  long long* adj_off;             // [3 seg_cap + 1] bins per item, exclusive-scanned: the adjoint's bin stream
  long long* adj_blk;             // [item blocks + 1] bins per block of kAdjItemBlock items, exclusive-scanned
  double* adj_bnd;                // [adjoint warps][2][16] partial sums of items cut by a warp's range
  int* adj_bnd_id;                // [adjoint warps][2] their items (-1: none, -2: the warp's range is empty)
  long long adj_item_cap;         // 3 seg_cap
  double* slots;                  // [sum N_m (K-1)][3 sub-pieces][16] per-segment gradients
  double* fseg;                   // [sum K][16] fundamental u-coefficient gradients per segment
  double *zf, *za;                // transposed-solve work arrays
};

struct LikeInputs {
  const double *data_plus, *data_cross;   // [sum N_f] complex128
  const double* psd;                      // [sum N_f]
  const double* df;                       // [n_wf]
  double* loglike;                        // [n_wf]
  double *g_phi_phi, *g_phi_r, *g_omega_phi, *g_omega_r;   // [sum K] or null
  double* g_amp;                          // [sum N_m K][2] or null
};

struct CallShape {
  int n_wf;
  long long K_total, nm_total, nf_total, seg_total, tiles_total, amp_total;
  int max_K;
  int tile_bins;
  int tile_split;   // CTAs (a thread-block cluster) sharing each tile: 1, 2 or 4
  int conj;
  int precision;
  int ext;          // 1: extended SPA (Eq. 10)
  int window;       // 1: Hann window applied to the outputs (Sec. 2.3)
};

constexpr int kLChunks = 512;      // per-waveform chunks of the likelihood's partial sums
constexpr int kPrepKernels = 11;   // kernels launched by launch_prep (memsets excluded)
constexpr int kAdjointKernels = 9; // kernels launched by launch_adjoint
constexpr int kAdjCtasPerSm = 2;     // resident CTAs of the adjoint kernel per SM (128 registers, 8 warps)
constexpr int kAdjWarpsPerCta = 8;
constexpr int kAdjItemBlock = 256;   // items per CTA of the item kernel (its local scan)
size_t adjoint_item_bytes();        // sizeof(AdjItem)

// freqs_ready (optional): an event the kernels that read in.freqs must wait for
void launch_prep(const CallShape& cs, const DevInputs& in, const DevScratch& s, cudaStream_t st,
                 cudaEvent_t freqs_ready = nullptr);
void launch_spa(const CallShape& cs, const DevInputs& in, const DevScratch& s, int num_sms, cudaStream_t st);
void launch_prep_td(const CallShape& cs, const DevInputs& in, const DevScratch& s, float4* tdamp, cudaStream_t st);
void launch_td_sum(const CallShape& cs, const DevInputs& in, const DevScratch& s, const float4* tdamp,
                   const double* dt, float* hp, float* hc, int num_sms, cudaStream_t st);
long long td_tile_samples();
void launch_td_pack(const float* hp, const float* hc, long long N, int hann, float2* z, int num_sms,
                    cudaStream_t st);
void launch_td_unpack(const float2* Z, long long N, double dt, double t0, float2* Hp, float2* Hc, int num_sms,
                      cudaStream_t st);
size_t select_smem_bytes(long long max_modes);
void launch_select(const DevScratch& s, int n_wf, int max_K, long long max_nm, const double* amp, double eps,
                   int* keep, long long nm_total, cudaStream_t st);
void launch_window(const CallShape& cs, const DevScratch& s, const double* freqs, const void* in_p, const void* in_c,
                   void* out_p, void* out_c, int num_sms, cudaStream_t st);
void launch_table(double2* tab, cudaStream_t st);
void launch_table_ff(const double2* tab, float4* tabf, cudaStream_t st);
void launch_scan(int* cnt, long long n, cudaStream_t st);
void launch_loglike(const CallShape& cs, const LikeInputs& li, const DevScratch& s, cudaStream_t st);
void launch_adjoint(const CallShape& cs, const DevInputs& in, const LikeInputs& li, const DevScratch& s, int num_sms,
                    cudaStream_t st);

}  // namespace emrifd
