// Time-domain comparator (arXiv 2307.12585, Sec. 2.3 and Sec. 3.2: the TD
// waveform of Eq. 2 and its DFT, against which the FD waveform is compared
// and timed).
//
// k_td_sum: h(t_j) = prefactor sum_modes [A Y_lm e^{-i Phi} + partner] at
// t_j = t_0 + j dt.  With psi = m Phi_phi + n Phi_r - m phi and w = A e^{-i psi},
//   h+ = 2 prefactor sum alpha Re w,   hx = -2 prefactor sum beta Im w,
// alpha, beta = [S_lm +- (-1)^l S_{l,-m}]/2 (the polarisation weights of the FD
// path).  FP32 arithmetic with an integer phase:
//   - per sample (shared by all modes): the segment, u, and frac(Phi_phi/2pi),
//     frac(Phi_r/2pi) as Q0.64 turns (knot value in Q0.64 from preparation plus
//     the in-segment cubic in FP64), rounded to Q0.32;
//   - per mode-sample: psi = m a + n b in wrapping 32-bit integers (error
//     <= (|m| + |n|)/2 units of 2^-32 turn), e^{-i psi} from the hardware FP32
//     sin/cos of psi in [-pi, pi) (about 4e-7 absolute), the amplitude cubics in
//     FP32, and FP32 sums over chunks of 32 modes carried in FP32 pairs.
// Persistent CTAs take tiles of kTdTile consecutive samples of one waveform
// from an atomic queue; a tile spans at most a few spline segments and is
// swept once per segment it touches, each sample accumulating only in its own.
//
// k_td_unpack: the spectrum from one complex FFT of z = h+ + i hx per
// waveform (cuFFT, inverse direction: sum_j z_j e^{+2 pi i jk/N}, the Fourier
// sign of Eq. 3): H+[k] = (Z[k] + conj Z[N-k])/2, Hx[k] = (Z[k] - conj Z[N-k])/(2i),
// times dt e^{2 pi i f_k t_0}, f_k = k/(N dt), for k = 1 .. N/2 - 1.
#include <cufft.h>

#include "common.cuh"
#include "ff.cuh"

namespace emrifd {
namespace {

constexpr int kTdSpt = 8;                       // samples per thread
constexpr int kTdTile = kTdSpt * kThreads;      // samples per tile

struct TdParams {
  const WfInfo* wf;
  int n_wf;
  const ModeInfo* modes;
  const float4* tdamp;
  const FundSeg* fund;
  const double* t;
  const double* dt;
  const double* prefactor;
  float* hp;
  float* hc;
  unsigned long long* counters;
  const int* status;
  long long tiles_total;
};

__device__ __forceinline__ int knot_segment(const double* t, int K, double x) {
  int a = 0, b = K - 2;   // last segment index with t[s] <= x
  while (a < b) {
    const int c = (a + b + 1) >> 1;
    if (t[c] <= x) a = c; else b = c - 1;
  }
  return a;
}

__global__ void __launch_bounds__(kThreads) k_td_sum(TdParams P) {
  __shared__ long long s_tile;
  const int tid = threadIdx.x;
  if (*P.status != 0) return;
  for (;;) {
    if (tid == 0) s_tile = (long long)atomicAdd(&P.counters[0], 1ull);
    __syncthreads();
    const long long tile = s_tile;
    __syncthreads();
    if (tile >= P.tiles_total) break;
    int lo = 0, hi = P.n_wf - 1;
    while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (P.wf[mid].tile_base <= tile) lo = mid; else hi = mid - 1; }
    const WfInfo W = P.wf[lo];
    const double* t = P.t + W.ko;
    const int K = (int)W.K;
    const double t0 = t[0], tlast = t[K - 1], dt = P.dt[lo];
    const long long j0 = (tile - W.tile_base) * kTdTile;
    const long long jend = min(j0 + kTdTile, W.nf);
    // segments touched by the tile's samples inside the trajectory
    const double ta = t0 + dt * (double)j0;
    double tb = t0 + dt * (double)(jend - 1);
    if (tb > tlast) tb = tlast;
    const int seg_lo = ta <= tlast ? knot_segment(t, K, ta) : K - 1;
    const int seg_hi = ta <= tlast ? knot_segment(t, K, tb) : K - 2;

    int seg[kTdSpt];
    unsigned pa[kTdSpt], pb[kTdSpt];
    float uf[kTdSpt];
    ff acc_p[kTdSpt], acc_c[kTdSpt];
#pragma unroll
    for (int q = 0; q < kTdSpt; q++) {
      const long long j = j0 + (long long)tid * kTdSpt + q;
      const double tj = t0 + dt * (double)j;
      seg[q] = -1;
      pa[q] = pb[q] = 0u;
      uf[q] = 0.f;
      acc_p[q] = acc_c[q] = ff_make(0.f, 0.f);
      if (j < jend && tj <= tlast) {
        const int s = knot_segment(t, K, tj);
        const double u = (tj - t[s]) / (t[s + 1] - t[s]);
        const FundSeg& F = P.fund[W.ko + s];
        const double dpp = u * fma(u, fma(u, F.P[0].z, F.P[0].y), F.P[0].x);
        const double dpr = u * fma(u, fma(u, F.P[1].z, F.P[1].y), F.P[1].x);
        const unsigned long long qa = F.q[0] - F.q[2] + q64_of(dpp * 0.15915494309189535);
        const unsigned long long qb = F.q[1] + q64_of(dpr * 0.15915494309189535);
        pa[q] = (unsigned)((qa + 0x80000000ull) >> 32);
        pb[q] = (unsigned)((qb + 0x80000000ull) >> 32);
        uf[q] = (float)u;
        seg[q] = s;
      }
    }
    for (int s = seg_lo; s <= seg_hi; s++) {
      const float4* amp_s = P.tdamp + 2 * (W.seg_base + s);
      for (long long m0 = 0; m0 < W.nm; m0 += 32) {
        float cp[kTdSpt], cc[kTdSpt];
#pragma unroll
        for (int q = 0; q < kTdSpt; q++) cp[q] = cc[q] = 0.f;
        const long long m1 = min(m0 + 32, W.nm);
        for (long long jm = m0; jm < m1; jm++) {
          const ModeInfo& M = P.modes[W.mo + jm];
          const int mm = M.m, nn = M.n;
          const float al = M.af[0], be = M.bf[0];
          const float4 ar = __ldg(amp_s + 2 * jm * (W.K - 1)), ai = __ldg(amp_s + 2 * jm * (W.K - 1) + 1);
          // every sample is evaluated with segment s's coefficients; the chunk sums of
          // samples in another segment (tiles that straddle a knot) are dropped below
#pragma unroll
          for (int q = 0; q < kTdSpt; q++) {
            const unsigned th = (unsigned)mm * pa[q] + (unsigned)nn * pb[q];   // psi in 2^-32 turns
            // psi in [-pi, pi) as FP32 radians; the hardware sin/cos approximations are
            // accurate to about 4e-7 absolute there, ample for an FP32 comparator
            const float x = (float)(int)th * 1.4629180792671596e-09f;           // 2 pi / 2^32
            float sn, cs;
            __sincosf(x, &sn, &cs);
            const float u = uf[q];
            const float are = fmaf(fmaf(fmaf(ar.w, u, ar.z), u, ar.y), u, ar.x);
            const float aim = fmaf(fmaf(fmaf(ai.w, u, ai.z), u, ai.y), u, ai.x);
            // w = A e^{-i psi}
            const float wr = fmaf(are, cs, aim * sn);
            const float wi = fmaf(aim, cs, -are * sn);
            cp[q] = fmaf(al, wr, cp[q]);
            cc[q] = fmaf(be, wi, cc[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < kTdSpt; q++) {
          if (seg[q] != s) continue;
          acc_p[q] = ff_add_f(acc_p[q], cp[q]);
          acc_c[q] = ff_add_f(acc_c[q], cc[q]);
        }
      }
    }
    const float pf = (float)(2.0 * P.prefactor[lo]);
#pragma unroll
    for (int q = 0; q < kTdSpt; q++) {
      const long long j = j0 + (long long)tid * kTdSpt + q;
      if (j < jend) {
        P.hp[W.fo + j] = pf * (acc_p[q].hi + acc_p[q].lo);
        P.hc[W.fo + j] = -pf * (acc_c[q].hi + acc_c[q].lo);
      }
    }
  }
}

// z = (h+ + i hx) w_j for one waveform (w_j = sin^2(pi j/N) with the Hann window, else 1)
__global__ void k_td_pack(const float* hp, const float* hc, long long N, double inv_n, int hann, float2* z) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
    float w = 1.f;
    if (hann) {
      const float sj = sinpif((float)((double)j * inv_n));
      w = sj * sj;
    }
    z[j] = make_float2(w * hp[j], w * hc[j]);
  }
}

__global__ void k_td_unpack(const float2* Z, long long N, double dt, double t0, float2* Hp, float2* Hc) {
  const long long nk = N / 2 - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nk; i += (long long)gridDim.x * blockDim.x) {
    const long long k = i + 1;
    const float2 a = Z[k], b = Z[N - k];
    // H+ = (a + conj b)/2, Hx = (a - conj b)/(2i)
    double pr = 0.5 * ((double)a.x + (double)b.x), pi = 0.5 * ((double)a.y - (double)b.y);
    double cr = 0.5 * ((double)a.y + (double)b.y), ci = -0.5 * ((double)a.x - (double)b.x);
    double er = dt, ei = 0.0;
    if (t0 != 0.0) {
      double sn, cs;
      sincospi(2.0 * fmod((double)k * (t0 / (dt * (double)N)), 1.0), &sn, &cs);
      er = dt * cs;
      ei = dt * sn;
    }
    Hp[i] = make_float2((float)(pr * er - pi * ei), (float)(pr * ei + pi * er));
    Hc[i] = make_float2((float)(cr * er - ci * ei), (float)(cr * ei + ci * er));
  }
}

}  // namespace

void launch_td_sum(const CallShape& cs, const DevInputs& in, const DevScratch& s, const float4* tdamp,
                   const double* dt, float* hp, float* hc, int num_sms, cudaStream_t st) {
  TdParams p;
  p.wf = s.wf; p.n_wf = cs.n_wf; p.modes = s.modes; p.tdamp = tdamp; p.fund = s.fund; p.t = in.t; p.dt = dt;
  p.prefactor = in.prefactor; p.hp = hp; p.hc = hc; p.counters = s.counters; p.status = s.status;
  p.tiles_total = cs.tiles_total;
  cudaMemsetAsync(s.counters, 0, sizeof(unsigned long long), st);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_td_sum, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)num_sms * per_sm;
  if (grid > cs.tiles_total) grid = cs.tiles_total > 0 ? cs.tiles_total : 1;
  k_td_sum<<<(unsigned)grid, kThreads, 0, st>>>(p);
}

long long td_tile_samples() { return kTdTile; }

void launch_td_pack(const float* hp, const float* hc, long long N, int hann, float2* z, int num_sms,
                    cudaStream_t st) {
  long long b = (N + 255) / 256;
  if (b > 32LL * num_sms) b = 32LL * num_sms;
  if (b < 1) b = 1;
  k_td_pack<<<(unsigned)b, 256, 0, st>>>(hp, hc, N, 1.0 / (double)N, hann, z);
}

void launch_td_unpack(const float2* Z, long long N, double dt, double t0, float2* Hp, float2* Hc, int num_sms,
                      cudaStream_t st) {
  long long b = (N / 2 + 255) / 256;
  if (b > 32LL * num_sms) b = 32LL * num_sms;
  if (b < 1) b = 1;
  k_td_unpack<<<(unsigned)b, 256, 0, st>>>(Z, N, dt, t0, Hp, Hc);
}

}  // namespace emrifd
