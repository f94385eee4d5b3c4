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
//
// Work decomposition: a persistent grid takes tiles of 32*BPL consecutive bins
// from a queue.  A tile's (run, sign) entries are collected in shared memory
// in ascending run order; warp w handles entries w, w+8, ... for all bins of
// the tile (BPL per lane) and the 8 warp partials are summed in warp order,
// so every bin's sum has a fixed order (no atomics on the outputs).
#include "spa_math.cuh"

namespace emrifd {
namespace {

struct SpaParams {
  const WfInfo* wf;
  int n_wf;
  const ModeInfo* modes;
  const SegCore* core;
  const SegAmp64* amp64;
  const SegAmp32* amp32;
  const long long* keyF;
  const Run* runs;
  const RunBins* rb;
  const double* freqs;
  void* hp;
  void* hc;
  const double2* tab;
  unsigned long long* counters;
  const int* status;
  long long tiles_total;
};

template <int BPL, int PREC>
struct Smem {
  double2 tab[PREC == 0 ? kTabN : 1];
  int list[kListCap];
  int wsum[kWarps + 1];
  long long tile;
  double red[kWarps][32 * BPL][4];
};

template <int BPL, int PREC>
__global__ void __launch_bounds__(kThreads, 2) k_spa(SpaParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<BPL, PREC>& S = *reinterpret_cast<Smem<BPL, PREC>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int TB = 32 * BPL;
  if (*P.status != 0) return;
  if (PREC == 0)
    for (int i = tid; i < kTabN; i += kThreads) S.tab[i] = P.tab[i];
  __syncthreads();

  for (;;) {
    if (tid == 0) S.tile = (long long)atomicAdd(&P.counters[0], 1ull);
    __syncthreads();
    const long long tile = S.tile;
    if (tile >= P.tiles_total) break;
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
      kn[q] = ordkey(-fq[q]);
    }
    double acc[BPL][4];
    float accf[BPL][4], cmp[BPL][4];
#pragma unroll
    for (int q = 0; q < BPL; q++)
#pragma unroll
      for (int c = 0; c < 4; c++) { acc[q][c] = 0.0; accf[q][c] = 0.f; cmp[q][c] = 0.f; }

    long long rcur = 0;
    const long long nruns = W.nruns;
    while (rcur < nruns || rcur == 0) {
      // ---- collect (run, sign) entries overlapping [bin0, binEnd), ascending
      int cnt = 0;
      while (rcur < nruns && cnt + 2 * kThreads <= kListCap) {
        long long r = rcur + tid;
        int fp = 0, fn = 0;
        if (r < nruns) {
          const RunBins B = P.rb[W.run_base + r];
          fp = (B.b0p < binEnd && B.b1p > bin0) ? 1 : 0;
          fn = (B.b0n < binEnd && B.b1n > bin0) ? 1 : 0;
        }
        int c = fp + fn, incl = c;
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
        if (fp) S.list[pos++] = (int)(r << 1);
        if (fn) S.list[pos] = (int)((r << 1) | 1);
        cnt += total;
        rcur += kThreads;
        __syncthreads();
      }
      if (rcur == 0) rcur = 1;   // no runs at all: leave the loop after this pass

      // ---- evaluate: warp w takes entries w, w + kWarps, ...
      for (int e = warp; e < cnt; e += kWarps) {
        const int ent = S.list[e];
        const long long r = W.run_base + (ent >> 1);
        const bool neg = ent & 1;
        const Run R = P.runs[r];
        const RunBins B = P.rb[r];
        const int b0 = neg ? B.b0n : B.b0p, b1 = neg ? B.b1n : B.b1p;
        const ModeInfo M = P.modes[R.mode];
        const double sa = M.alpha, sb = neg ? -M.beta : M.beta;   // h+ += alpha Z~, hx += i sb Z~
#pragma unroll
        for (int q = 0; q < BPL; q++) {
          const long long bin = bin0 + lane + 32 * q;
          if (bin < b0 || bin >= b1) continue;
          const double g = neg ? -fq[q] : fq[q];
          const long long key = neg ? kn[q] : kp[q];
          // a5: segment holding the root
          const int s = run_segment(R, P.keyF, M.key_base, key);
          const double ulo = (s == R.s0) ? R.u0 : 0.0, uhi = (s == R.s1) ? R.u1 : 1.0;
          const SegCore C = P.core[M.seg_base + s];
          // a6: root
          const double delta = g - C.A;
          float uf, Df;
          const double u = solve_root(C, delta, ulo, uhi, R.dir, uf, Df);
          // a8: dF/du and the weight sqrt(h)/sqrt|dF/du| (sqrt(h) is in the amplitude)
          const double Dd = fma(u, fma(u, C.d3, C.c2), C.b);
          const long long Dbits = __double_as_longlong(Dd);
          if ((Dbits & 0x7FFFFFFFFFFFFFFFLL) == 0) continue;   // Fdot == 0: no contribution
          const bool pos_slope = Dbits >= 0;
          // a7: phase in Q0.64 turns
          const unsigned long long Th = phase_q64(C, g, delta, u, pos_slope);
          if (PREC == 0) {
            const double wgt = rsqrt_abs(Dd);
            double er, ei;
            cis_q64(Th, S.tab, er, ei);
            // a9-a10
            const SegAmp64 Am = P.amp64[M.seg_base + s];
            double are = fma(u, fma(u, fma(u, Am.re[3], Am.re[2]), Am.re[1]), Am.re[0]);
            double aim = fma(u, fma(u, fma(u, Am.im[3], Am.im[2]), Am.im[1]), Am.im[0]);
            are *= wgt;
            aim *= wgt;
            const double zr = fma(are, er, -aim * ei);
            const double zi = fma(are, ei, aim * er);
            // a11: positive branch h+ += alpha Z, hx += i beta Z;
            //      negative branch h+ += alpha conj Z, hx += -i beta conj Z
            acc[q][0] = fma(sa, zr, acc[q][0]);
            acc[q][1] = fma(neg ? -sa : sa, zi, acc[q][1]);
            acc[q][2] = fma(-M.beta, zi, acc[q][2]);
            acc[q][3] = fma(sb, zr, acc[q][3]);
          } else {
            const float wgt = rsqrtf(fabsf(Df));
            const float th = (float)(int)(Th >> 32) * 4.656612873077393e-10f;   // half-turns in [-1, 1)
            float sn, cs;
            sincospif(th, &sn, &cs);
            const SegAmp32 Am = P.amp32[M.seg_base + s];
            float are = ((Am.re[3] * uf + Am.re[2]) * uf + Am.re[1]) * uf + Am.re[0];
            float aim = ((Am.im[3] * uf + Am.im[2]) * uf + Am.im[1]) * uf + Am.im[0];
            are *= wgt;
            aim *= wgt;
            const float zr = are * cs - aim * sn;
            const float zi = are * sn + aim * cs;
            const float fa = (float)sa, fb = (float)M.beta;
            float v[4] = {fa * zr, (neg ? -fa : fa) * zi, -fb * zi, (neg ? -fb : fb) * zr};
#pragma unroll
            for (int c = 0; c < 4; c++) {   // Kahan-compensated accumulation
              float y = v[c] - cmp[q][c];
              float t2 = accf[q][c] + y;
              cmp[q][c] = (t2 - accf[q][c]) - y;
              accf[q][c] = t2;
            }
          }
        }
      }
      __syncthreads();
      if (rcur >= nruns) break;
    }

    // ---- fixed-order reduction over warps, one store per bin
#pragma unroll
    for (int q = 0; q < BPL; q++)
#pragma unroll
      for (int c = 0; c < 4; c++)
        S.red[warp][lane + 32 * q][c] = PREC == 0 ? acc[q][c] : ((double)accf[q][c] - (double)cmp[q][c]);
    __syncthreads();
    for (int i = tid; i < TB; i += kThreads) {
      const long long bin = bin0 + i;
      if (bin < binEnd) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w2 = 0; w2 < kWarps; w2++)
#pragma unroll
          for (int c = 0; c < 4; c++) v[c] += S.red[w2][i][c];
        if (PREC == 0) {
          reinterpret_cast<double2*>(P.hp)[bin] = make_double2(v[0], v[1]);
          reinterpret_cast<double2*>(P.hc)[bin] = make_double2(v[2], v[3]);
        } else {
          reinterpret_cast<float2*>(P.hp)[bin] = make_float2((float)v[0], (float)v[1]);
          reinterpret_cast<float2*>(P.hc)[bin] = make_float2((float)v[2], (float)v[3]);
        }
      }
    }
    __syncthreads();
  }
}

template <int BPL, int PREC>
void launch_one(const SpaParams& p, int num_sms, cudaStream_t st) {
  size_t sm = sizeof(Smem<BPL, PREC>);
  cudaFuncSetAttribute(k_spa<BPL, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spa<BPL, PREC>, kThreads, sm);
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)num_sms * per_sm;
  if (grid > p.tiles_total) grid = p.tiles_total > 0 ? p.tiles_total : 1;
  k_spa<BPL, PREC><<<(unsigned)grid, kThreads, sm, st>>>(p);
}

}  // namespace

void launch_spa(const CallShape& cs, const DevInputs& in, const DevScratch& s, int num_sms, cudaStream_t st) {
  SpaParams p;
  p.wf = s.wf; p.n_wf = cs.n_wf; p.modes = s.modes; p.core = s.core; p.amp64 = s.amp64; p.amp32 = s.amp32;
  p.keyF = s.keyF; p.runs = s.runs; p.rb = s.rbins; p.freqs = in.freqs; p.hp = in.h_plus; p.hc = in.h_cross;
  p.tab = s.tab; p.counters = s.counters; p.status = s.status; p.tiles_total = cs.tiles_total;
  cudaMemsetAsync(s.counters, 0, sizeof(unsigned long long), st);
  const int bpl = cs.tile_bins / 32;
  if (cs.precision == 0) {
    if (bpl == 1) launch_one<1, 0>(p, num_sms, st);
    else if (bpl == 4) launch_one<4, 0>(p, num_sms, st);
    else launch_one<2, 0>(p, num_sms, st);
  } else {
    if (bpl == 1) launch_one<1, 1>(p, num_sms, st);
    else if (bpl == 4) launch_one<4, 1>(p, num_sms, st);
    else launch_one<2, 1>(p, num_sms, st);
  }
}

}  // namespace emrifd
