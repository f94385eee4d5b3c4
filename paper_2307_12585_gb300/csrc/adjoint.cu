// Whittle log-likelihood (arXiv 2307.12585, Eq. 13-14) and its adjoint with
// respect to every knot value of Phi_phi, Phi_r, Omega_phi, Omega_r and the
// complex mode amplitudes.
//
// L_w = -1/2 sum_alpha <d - h|d - h>_alpha = -2 df sum_i |d_i - h_i|^2 / S_i,
// G_i = dL/dRe h_i + i dL/dIm h_i = 4 df (d_i - h_i) / S_i  (per channel).
// One output-kernel contribution Z (see spa.cu) enters h+ and hx as
// alpha Z, i beta Z (F > 0) or alpha conj Z, -i beta conj Z (F < 0), so
// dL = Re[Q dZ] with Q = alpha conj G+ + i beta conj Gx (F > 0) or
// alpha G+ + i beta Gx (F < 0).  With Z = A(u) E, E = |dF/du|^{-1/2} e^{i psi},
// dZ/Z = dA/A - dD/(2D) + i dpsi (D = dF/du), and the root moving as
// du = -(dF/dcoef)/D at fixed frequency (the branch and segment assignment of
// every bin is held fixed), the per-bin derivatives with respect to the
// segment's u-polynomial coefficients are (QE = Q E, QZ = Q Z):
//   amplitude a_k:      u^k Re QE,  u^k (-Im QE)           (d/dRe, d/dIm)
//   phase phi_k (rad):  u^k Im QZ
//   frequency F_k (Hz): -T u^k / D - (1/2) Re QZ k u^(k-1) / D,
//   T = Re(QE A'(u)) - (1/2) Re QZ D'(u)/D - Im QZ (2 pi g h - Phi_V'(u)).
// The roots are recomputed here with exactly the arithmetic of the output
// kernel (spa_math.cuh), not stored.  Sums run in a fixed order: a warp tree per
// (run, segment), slots per (mode, segment, sub-piece), a block tree over the
// modes of each segment, then the transposed not-a-knot solve to knot values.
#include "spa_math.cuh"

namespace emrifd {
namespace {

constexpr double kTwoPi = 6.283185307179586;
constexpr double kInv2Pi = 0.15915494309189535;

// ------------------------------------------------------------ residual and L
__global__ void k_residual(const WfInfo* wf, const double2* hp, const double2* hc, const double2* dp,
                           const double2* dc, const double* psd, const double* dfs, dbl4* G, double* Lpart,
                           int* status) {
  __shared__ double red[256];
  const WfInfo W = wf[blockIdx.y];
  const long long len = (W.nf + kLChunks - 1) / kLChunks;
  const long long b0 = W.fo + blockIdx.x * len, b1 = min(b0 + len, W.fo + W.nf);
  const double df = dfs[blockIdx.y];
  double acc = 0.0;
  int bad = 0;
  const double c4 = 4.0 * df;
  for (long long b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
    const double S = psd[b];
    // S positive and finite, tested on its bits as a signed integer (0 < bits < +inf's)
    // so that the test takes no FP64-pipe slots
    const long long sb = __double_as_longlong(S);
    if (!(sb > 0 && sb < 0x7ff0000000000000LL)) bad = ST_NONFINITE;
    const double2 a = hp[b], c = hc[b], x = dp[b], y = dc[b];
    const double rpr = x.x - a.x, rpi = x.y - a.y, rcr = y.x - c.x, rci = y.y - c.y;
    const double w = c4 * rcp_d(S);
    acc = fma(rpr * rpr + rpi * rpi + rcr * rcr + rci * rci, w, acc);
    G[b] = mk_dbl4(w * rpr, w * rpi, w * rcr, w * rci);
  }
  if (bad) atomicOr(status, bad);
  // -1/2 once per thread: a power of two, so every partial is the same as with -w/2
  // applied per bin
  red[threadIdx.x] = -0.5 * acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) Lpart[blockIdx.y * kLChunks + blockIdx.x] = red[0];
}

// one CTA of 256 threads per waveform: chunk partials summed in a fixed tree order
__global__ void k_loglike_final(int n_wf, const double* Lpart, double* L) {
  __shared__ double red[256];
  const int w = blockIdx.x, tid = threadIdx.x;
  double s = 0.0;
  for (int c = tid; c < kLChunks; c += 256) s += Lpart[(long long)w * kLChunks + c];
  red[tid] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0) L[w] = red[0];
}

// ---------------------------------------------------------- adjoint items
__global__ void k_item_len(const int* run_total, const Run* runs, long long run_cap, int* len) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= run_cap) return;
  long long nr = min((long long)*run_total, run_cap);
  int v = 0;
  if (r < nr) {
    const Run R = runs[r];
    if (R.mode >= 0 && R.s1 >= R.s0) v = R.s1 - R.s0 + 1;
  }
  len[r] = v;
}

// One adjoint item: a (run, segment) pair, with the bins of both branch signs that it
// covers and per-segment constants of its derivatives
struct __align__(16) AdjItem {
  int run, s, piece, pad;
  int lo_p, hi_p, lo_n, hi_n;            // global bins [lo, hi) of the positive / negative branch
  double a3r, a2r, a3i, a2i;             // 3 re_3, 2 re_2, 3 im_3, 2 im_2 of the amplitude record (dA/du)
  double d2c, p2c, p3c, pad2;            // 2 (3d) = d^2F/du^2 slope, 2 P2, 3 P3 (dPhi_V/du)
};
static_assert(sizeof(AdjItem) == 96, "AdjItem layout");

struct AdjParams {
  const WfInfo* wf;
  const ModeInfo* modes;
  const SegCore* core;
  const SegAmp64* amp64;
  const SegCrit* crit;
  const long long* keyF;
  const Run* runs;
  const RunBins* rb;
  const double* freqs;
  const dbl4* G;
  const int* item_off;     // exclusive scan of items per run, total at [run_cap]
  long long run_cap;
  AdjItem* items;          // [item_cap]
  long long* adj_off;      // [item_cap + 1] exclusive scan of the items' bin counts (the bin stream)
  long long* adj_blk;      // [item blocks + 1] bins per block of kAdjItemBlock items, scanned
  long long item_cap;
  double* bnd;             // [warps][2][16]
  int* bnd_id;             // [warps][2]
  const double2* tab;      // e^{2 pi i k/65536}
  double* slots;           // [3 * seg_total][16]
  const int* status;
  long long nm_total, seg_total, nf_total;   // array sizes (checked builds)
};

// last r in [0, n) with off[r] <= it, for ascending off with off[0] <= it (one thread)
template <typename T>
__device__ __forceinline__ long long last_le(const T* off, long long n, long long it) {
  long long lo = 0, hi = n - 1;
  while (lo < hi) {
    const long long mid = (lo + hi + 1) >> 1;
    if ((long long)off[mid] <= it) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// one item slot: the run and segment of the item, the bins it covers (knot s passed
// for s > s0, knot s + 1 not passed for s < s1, as the output kernel assigns them), its
// sub-piece and the per-segment constants.  Returns the item's bin count; slots past
// the item count, and every slot after a failed input check (the run lists are then
// not valid), get zero bins.
__device__ __forceinline__ long long adj_item(const AdjParams& P, long long it) {
  const long long nitems = P.item_off[P.run_cap];
  if (it >= nitems || *P.status != 0) return 0;
  const long long r = last_le(P.item_off, P.run_cap, it);
  const Run R = P.runs[r];
  const int s = R.s0 + (int)(it - P.item_off[r]);
  const RunBins B = P.rb[r];
  const ModeInfo M = P.modes[R.mode];
  AdjItem I;
  I.run = (int)r; I.s = s; I.pad = 0;
  // the bins of each branch sign, cut at knot s (for s > s0) and knot s + 1 (for
  // s < s1): the first bin at which "knot passed" flips, found by binary search.  The
  // (up to) four searches q = 2 sign + (0: knot s, 1: knot s + 1) advance in lockstep so
  // that their loads overlap.
  long long b0s[2], b1s[2], slo[4], shi[4], kk[4];
  bool sneg[4], ssuf[4];
#pragma unroll
  for (int sg = 0; sg < 2; sg++) {
    b0s[sg] = sg ? B.b0n : B.b0p;
    b1s[sg] = sg ? B.b1n : B.b1p;
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int sg = q >> 1, k = s + (q & 1);
    const bool want = (b0s[sg] < b1s[sg]) && ((q & 1) ? (s < R.s1) : (s > R.s0));
    slo[q] = b0s[sg];
    shi[q] = want ? b1s[sg] : b0s[sg];   // an empty range: not searched
    sneg[q] = sg == 1;
    ssuf[q] = (R.dir > 0) != (sg == 1);   // "passed" holds on a suffix of the bins
    kk[q] = want ? P.keyF[M.key_base + k] : 0;
  }
  for (;;) {
    bool any = false;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (slo[q] < shi[q]) {
        const long long c = (slo[q] + shi[q]) >> 1;
        const double f = P.freqs[c];
        const long long key = ordkey(sneg[q] ? flip_sign(f) : f);
        const bool passed = R.dir > 0 ? (kk[q] <= key) : (kk[q] >= key);
        if (passed == ssuf[q]) shi[q] = c; else slo[q] = c + 1;
        any = true;
      }
    }
    if (!any) break;
  }
  int lo[2], hi[2];
#pragma unroll
  for (int sg = 0; sg < 2; sg++) {
    long long lo_b = b0s[sg], hi_b = b1s[sg];
    if (lo_b < hi_b) {
      const bool suffix = ssuf[2 * sg];
      if (s > R.s0) { const long long x = slo[2 * sg]; if (suffix) lo_b = x; else hi_b = x; }
      if (s < R.s1) { const long long x = slo[2 * sg + 1]; if (suffix) hi_b = min(hi_b, x); else lo_b = max(lo_b, x); }
    }
    if (hi_b < lo_b) hi_b = lo_b;
    lo[sg] = (int)lo_b;
    hi[sg] = (int)hi_b;
  }
  I.lo_p = lo[0]; I.hi_p = hi[0]; I.lo_n = lo[1]; I.hi_n = hi[1];
  // sub-piece of segment s that this run covers
  int piece = 0;
  if (s == R.s0) {
    const SegCrit X = P.crit[M.seg_base + s];   // at most two critical points
    piece = (X.n > 0 && X.u[0] <= R.u0) + (X.n > 1 && X.u[1] <= R.u0);
  }
  I.piece = piece;
  const SegAmp64 Am = P.amp64[M.seg_base + s];
  const SegCore C = P.core[M.seg_base + s];
  I.a3r = 3.0 * Am.re[3]; I.a2r = 2.0 * Am.re[2]; I.a3i = 3.0 * Am.im[3]; I.a2i = 2.0 * Am.im[2];
  I.d2c = 2.0 * C.d3; I.p2c = 2.0 * C.P2; I.p3c = 3.0 * C.P3; I.pad2 = 0.0;
  P.items[it] = I;
  return (long long)(hi[0] - lo[0]) + (hi[1] - lo[1]);
}

// exclusive scan over the 256 threads of a CTA (int64); *total gets the CTA's sum
__device__ __forceinline__ long long cta_exclusive_scan(long long v, long long* wsum, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  long long before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kAdjItemBlock / 32; w++) {
    const long long t = wsum[w];
    if (w < warp) before += t;
    all += t;
  }
  *total = all;
  return before + x - v;
}

// items, one thread per item slot, kAdjItemBlock slots per CTA: each slot's record
// and bin count; the counts are scanned within the CTA (adj_off gets the offset of
// the item inside its block) and the block's total goes to adj_blk
__global__ void __launch_bounds__(kAdjItemBlock) k_adj_items(AdjParams P) {
  __shared__ long long wsum[kAdjItemBlock / 32];
  const long long it = blockIdx.x * (long long)kAdjItemBlock + threadIdx.x;
  const long long n = it < P.item_cap ? adj_item(P, it) : 0;
  long long total;
  const long long e = cta_exclusive_scan(n, wsum, &total);
  if (it < P.item_cap) P.adj_off[it] = e;
  if (threadIdx.x == 0) P.adj_blk[blockIdx.x] = total;
}

// the bin stream's offsets: adj_off[i] += the scanned total of the blocks before i's
// block; adj_off[item_cap] = the stream's length
__global__ void k_adj_offsets(long long* adj_off, const long long* blk, long long item_cap) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < item_cap) adj_off[i] += blk[i / kAdjItemBlock];
  else if (i == item_cap) adj_off[i] = blk[(item_cap + kAdjItemBlock - 1) / kAdjItemBlock];
}

// exclusive scan of cnt[0..n) in place (int64), total written to cnt[n]; one block of
// 1024 threads stepping through the array 4096 entries at a time (each thread four
// consecutive entries, so the loads and stores are coalesced), carrying the running total
__global__ void __launch_bounds__(1024) k_scan64(long long* cnt, long long n) {
  __shared__ long long wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long carry = 0;
  for (long long base = 0; base < n; base += 4096) {
    long long v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const long long i = base + 4 * tid + k;
      v[k] = i < n ? cnt[i] : 0;
      s += v[k];
    }
    long long x = s;   // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    long long e = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - s;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const long long i = base + 4 * tid + k;
      if (i < n) cnt[i] = e;
      e += v[k];
    }
    carry += wsum[31];
    __syncthreads();
  }
  if (tid == 0) cnt[n] = carry;
}

// the adjoint's per-lane state of one item
struct AdjLane {
  Run R;
  SegCore C;
  SegAmp64 Am;
  AdjItem I;
  double ap, bp;           // alpha, beta over the record's scale (one of them is 1)
  double ulo, uhi;
  long long seg;           // global (mode, segment) record
};

__device__ __forceinline__ bool adj_load(const AdjParams& P, long long it, AdjLane& L) {
  L.I = P.items[it];
  if (check_fails(L.I.run >= 0 && L.I.run < P.run_cap, P.status)) return false;
  L.R = P.runs[L.I.run];
  if (check_fails(L.R.mode >= 0 && L.R.mode < P.nm_total, P.status)) return false;
  const ModeInfo M = P.modes[L.R.mode];
  L.seg = M.seg_base + L.I.s;
  if (check_fails(L.I.s >= L.R.s0 && L.I.s <= L.R.s1 && L.seg < P.seg_total && L.I.lo_p >= 0 &&
                      L.I.hi_p <= P.nf_total && L.I.lo_n >= 0 && L.I.hi_n <= P.nf_total,
                  P.status))
    return false;
  L.C = P.core[L.seg];
  L.Am = P.amp64[L.seg];   // times M.scale
  const bool amaj = alpha_major(M.alpha, M.beta);
  L.ap = amaj ? 1.0 : M.rho;
  L.bp = amaj ? M.rho : 1.0;
  L.ulo = (L.I.s == L.R.s0) ? L.R.u0 : 0.0;
  L.uhi = (L.I.s == L.R.s1) ? L.R.u1 : 1.0;
  return true;
}

// The adjoint's bin stream: the bins of every item, item after item (positive branch
// first), adj_off[i] the position of item i's first bin.  Lane g of the G lanes of the
// grid takes the contiguous positions [N g/G, N (g + 1)/G), so every lane has the same
// number of bins (no lane idles at the end of an item) and a lane's bins mostly belong
// to one item.  Per bin the lane recomputes the forward's root, phase, weight and
// amplitude (spa_math.cuh) and accumulates the item's 16 coefficient sums in
// registers.  An item that starts and ends inside a lane is written to its slot by
// that lane; the first and last item of each lane (which may continue in its
// neighbours) go to shared memory, where 16 lanes of the warp sum them per item in
// lane order; items that continue past the warp's range go to the warp's two boundary
// records, summed in warp order by k_adj_fixup.  Every sum has a fixed order.
__global__ void __launch_bounds__(32 * kAdjWarpsPerCta, kAdjCtasPerSm) k_adjoint(AdjParams P) {
  extern __shared__ __align__(16) double adj_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* rows = adj_smem + (size_t)wib * 64 * 16;                              // [64][16]
  int* ids = reinterpret_cast<int*>(adj_smem + (size_t)kAdjWarpsPerCta * 64 * 16) + wib * 64;  // [64]
  const long long nw = (long long)gridDim.x * kAdjWarpsPerCta;
  const long long gw = (long long)blockIdx.x * kAdjWarpsPerCta + wib;
  if (*P.status != 0) {
    if (lane < 2) P.bnd_id[2 * gw + lane] = -2;
    return;
  }
  const long long N = P.adj_off[P.item_cap];
  const long long G = 32 * nw, g = 32 * gw + lane;
  const long long p0 = N / G * g + (N % G) * g / G, p1 = N / G * (g + 1) + (N % G) * (g + 1) / G;
  const long long wp0 = N / G * (32 * gw) + (N % G) * (32 * gw) / G;
  const long long wp1 = N / G * (32 * gw + 32) + (N % G) * (32 * gw + 32) / G;
  ids[2 * lane] = -1;
  ids[2 * lane + 1] = -1;
  if (p0 < p1) {
    // the item holding position p0: the last i with adj_off[i] <= p0 (empty items
    // before it have the same offset and are skipped by taking the last)
    long long it = last_le(P.adj_off, P.item_cap, p0);
    long long it_end = P.adj_off[it + 1];
    AdjLane L;
    if (!adj_load(P, it, L)) return;
    bool first_open = true;
    double acc[16], hsum[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 16; q++) acc[q] = 0.0;
    for (long long pos = p0; pos < p1; pos++) {
      if (pos >= it_end) {
        // item it is finished for this lane: its frequency sums combined, then kept for
        // the warp's combination (the lane's first item) or written (an inner item)
        acc[1] += hsum[0];
        acc[2] = fma(2.0, hsum[1], acc[2]);
        acc[3] = fma(3.0, hsum[2], acc[3]);
        double* dst;
        if (first_open) {
          dst = rows + 2 * lane * 16;
          ids[2 * lane] = (int)it;
          first_open = false;
        } else {
          dst = P.slots + (L.seg * 3 + L.I.piece) * 16;
        }
#pragma unroll
        for (int q = 0; q < 16; q++) dst[q] = acc[q];
        do { it++; it_end = P.adj_off[it + 1]; } while (it_end <= pos);
        if (!adj_load(P, it, L)) return;
#pragma unroll
        for (int q = 0; q < 16; q++) acc[q] = 0.0;
        hsum[0] = hsum[1] = hsum[2] = 0.0;
      }
      const long long k = pos - P.adj_off[it];
      const long long np = L.I.hi_p - L.I.lo_p;
      const bool neg = k >= np;
      const long long b = neg ? L.I.lo_n + (k - np) : L.I.lo_p + k;
      const SegCore& C = L.C;
      const SegAmp64& Am = L.Am;
      const double g0 = P.freqs[b];
      const double gg = neg ? flip_sign(g0) : g0;
      const double delta = gg - C.A;
      float uf, Df;
      const double u = solve_root<6>(C, delta, L.ulo, L.uhi, L.I.s == L.R.s0 ? L.R.u0f[0] : 0.f,
                                     L.I.s == L.R.s1 ? L.R.u1f[0] : 1.f, L.R.dir, uf, Df);
      const double Dd = fma(u, fma(u, C.d3, C.c2), C.b);
      const long long Dbits = __double_as_longlong(Dd);
      if (is_zero_bits(Dd)) continue;
      const unsigned long long Th = phase_q64(C, gg, delta, u, Dbits >= 0);
      const double wgt = rsqrt_abs(Dd);
      double Er, Ei;
      cis_w_q64(Th, P.tab, wgt, Er, Ei);                    // E = |D|^{-1/2} e^{i psi}
      const double Ar = fma(u, fma(u, fma(u, Am.re[3], Am.re[2]), Am.re[1]), Am.re[0]);
      const double Ai = fma(u, fma(u, fma(u, Am.im[3], Am.im[2]), Am.im[1]), Am.im[0]);
      const double dAr = fma(u, fma(u, L.I.a3r, L.I.a2r), Am.re[1]);
      const double dAi = fma(u, fma(u, L.I.a3i, L.I.a2i), Am.im[1]);
      const dbl4 Gb = P.G[b];
      double Qr, Qi;
      if (!neg) { Qr = L.ap * Gb.x + L.bp * Gb.w; Qi = -L.ap * Gb.y + L.bp * Gb.z; }
      else { Qr = L.ap * Gb.x - L.bp * Gb.w; Qi = L.ap * Gb.y + L.bp * Gb.z; }
      const double QEr = Qr * Er - Qi * Ei, QEi = Qr * Ei + Qi * Er;
      const double QZr = QEr * Ar - QEi * Ai, QZi = QEr * Ai + QEi * Ar;
      const double Dp = fma(L.I.d2c, u, C.c2);              // d^2F/du^2
      const double dpsi = kTwoPi * fma(-u, fma(L.I.p3c, u, L.I.p2c), fma(delta, C.h, -C.Q1));  // 2 pi g h - Phi_V'(u)
      const double w2 = wgt * wgt;                          // 1/|dF/du| from the weight: no FP64 division
      const double invD = Dbits >= 0 ? w2 : flip_sign(w2);
      const double hD = -0.5 * QZr * invD;
      const double T = fma(QEr, dAr, fma(-QEi, dAi, fma(hD, Dp, -QZi * dpsi)));
      const double tD = -T * invD;
      const double u2 = u * u, u3 = u2 * u;
      acc[0] += tD;
      acc[1] = fma(tD, u, acc[1]);
      acc[2] = fma(tD, u2, acc[2]);
      acc[3] = fma(tD, u3, acc[3]);
      hsum[0] += hD;
      hsum[1] = fma(hD, u, hsum[1]);
      hsum[2] = fma(hD, u2, hsum[2]);
      acc[4] += QZi;
      acc[5] = fma(u, QZi, acc[5]);
      acc[6] = fma(u2, QZi, acc[6]);
      acc[7] = fma(u3, QZi, acc[7]);
      acc[8] += QEr;
      acc[9] = fma(u, QEr, acc[9]);
      acc[10] = fma(u2, QEr, acc[10]);
      acc[11] = fma(u3, QEr, acc[11]);
      acc[12] -= QEi;
      acc[13] = fma(-u, QEi, acc[13]);
      acc[14] = fma(-u2, QEi, acc[14]);
      acc[15] = fma(-u3, QEi, acc[15]);
    }
    acc[1] += hsum[0];
    acc[2] = fma(2.0, hsum[1], acc[2]);
    acc[3] = fma(3.0, hsum[2], acc[3]);
    double* dst = rows + (2 * lane + 1) * 16;
#pragma unroll
    for (int q = 0; q < 16; q++) dst[q] = acc[q];
    ids[2 * lane + 1] = (int)it;
  }
  __syncwarp();
  // per item, the lanes' first and last partials in lane order; an item inside the
  // warp's range is complete, one cut by its start or end goes to a boundary record
  if (lane < 16) {
    int cur = -1, nb0 = -1, nb1 = -1;
    double sum = 0.0;
    for (int row = 0; row <= 64; row++) {
      const int id = row < 64 ? ids[row] : -1;
      if (row < 64 && id < 0) continue;
      if (id != cur) {
        if (cur >= 0) {
          const long long a = P.adj_off[cur], e = P.adj_off[cur + 1];
          if (a < wp0) {
            P.bnd[(2 * gw) * 16 + lane] = sum;
            nb0 = cur;
          } else if (e > wp1) {
            P.bnd[(2 * gw + 1) * 16 + lane] = sum;
            nb1 = cur;
          } else {
            const AdjItem I = P.items[cur];
            const Run R = P.runs[I.run];
            const long long seg = P.modes[R.mode].seg_base + I.s;
            P.slots[(seg * 3 + I.piece) * 16 + lane] = sum;
          }
        }
        cur = id;
        if (row < 64) sum = rows[row * 16 + lane];
      } else {
        sum += rows[row * 16 + lane];
      }
    }
    if (lane == 0) {
      P.bnd_id[2 * gw] = wp0 < wp1 ? nb0 : -2;
      P.bnd_id[2 * gw + 1] = wp0 < wp1 ? nb1 : -2;
    }
  }
}

// items cut by warp ranges: the warp where an item starts holds its first partial in
// its second boundary record; the following warps hold the rest in their first
// records; one thread per warp sums a chain in warp order and writes the item's slot
__global__ void k_adj_fixup(AdjParams P, long long nw) {
  const long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (w >= nw || *P.status != 0) return;
  const int it = P.bnd_id[2 * w + 1];
  if (it < 0) return;
  double sum[16];
#pragma unroll
  for (int q = 0; q < 16; q++) sum[q] = P.bnd[(2 * w + 1) * 16 + q];
  for (long long w2 = w + 1; w2 < nw; w2++) {
    const int id = P.bnd_id[2 * w2];
    if (id == -2) continue;          // a warp with no positions
    if (id != it) break;
#pragma unroll
    for (int q = 0; q < 16; q++) sum[q] += P.bnd[(2 * w2) * 16 + q];
  }
  const AdjItem I = P.items[it];
  const Run R = P.runs[I.run];
  const long long seg = P.modes[R.mode].seg_base + I.s;
#pragma unroll
  for (int q = 0; q < 16; q++) P.slots[(seg * 3 + I.piece) * 16 + q] = sum[q];
}

// per (mode, segment): sum the sub-piece slots into slot 0 and scale the
// amplitude part to the unscaled spline coefficients (the record holds
// prefactor sqrt(h) scale times them, and the sums were formed with alpha and
// beta over the mode's scale)
// one coefficient of a (mode, segment) record's gradient: its three sub-piece slots summed
__device__ __forceinline__ double slot_sum(const double* a, int q) { return a[q] + a[16 + q] + a[32 + q]; }

// u-coefficient gradients (a, b, c, d) of segment s -> gradients of
// (y_s, y_{s+1}, M_s, M_{s+1}), with a = y_s, b = y_{s+1} - y_s - h^2 (2 M_s + M_{s+1})/6,
// c = h^2 M_s / 2, d = h^2 (M_{s+1} - M_s)/6; accumulated per knot
// (1/3 and 1/6 as products with their nearest doubles: no FP64 divisions)
__device__ __forceinline__ void ucoef_adj(const double* gq, double h2, int side, double& gy, double& gM) {
  constexpr double kThird = 1.0 / 3.0, kSixth = 1.0 / 6.0;
  const double ga = gq[0], gb = gq[1], gc = gq[2], gd = gq[3];
  if (side == 0) {   // the segment starting at this knot
    gy += ga - gb;
    gM += h2 * (-gb * kThird + 0.5 * gc - gd * kSixth);
  } else {           // the segment ending at this knot
    gy += gb;
    gM += h2 * ((gd - gb) * kSixth);
  }
}

// fundamental series: per (waveform, segment) block, fixed-order tree over the
// waveform's modes; writes u-coefficient gradients of Phi_phi, Phi_r (rad) and
// Om_phi, Om_r (rad/s) for that segment: [4 series][4]
__global__ void k_fund_seg(const WfInfo* wf, const ModeInfo* modes, const double* slots, double* fseg) {
  __shared__ double red[256][17];   // a 17-double row stride: no shared-memory bank conflicts
  const WfInfo W = wf[blockIdx.y];
  const int s = blockIdx.x;
  if (s >= W.K - 1) return;
  double acc[16];
  for (int q = 0; q < 16; q++) acc[q] = 0.0;
  for (long long j = threadIdx.x; j < W.nm; j += blockDim.x) {
    const ModeInfo M = modes[W.mo + j];
    const double* a = slots + (M.seg_base + s) * 3 * 16;
    const double dm = (double)M.m, dn = (double)M.n;
    for (int k = 0; k < 4; k++) {
      const double gp = slot_sum(a, 4 + k), gf = slot_sum(a, k);
      acc[k] += dm * gp;                       // Phi_phi
      acc[4 + k] += dn * gp;                   // Phi_r
      acc[8 + k] += dm * kInv2Pi * gf;         // Om_phi
      acc[12 + k] += dn * kInv2Pi * gf;        // Om_r
    }
  }
  for (int q = 0; q < 16; q++) red[threadIdx.x][q] = acc[q];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 16; q++) red[threadIdx.x][q] += red[threadIdx.x + o][q];
    __syncthreads();
  }
  if (threadIdx.x < 16) fseg[(W.ko + s) * 16 + threadIdx.x] = red[0][threadIdx.x];
}

// Transpose of the not-a-knot map y -> M (the forward solve of the preparation)
// applied to gM, added to gY: out = gY + (dM/dy)^T gM.  One warp per series; the
// two triangular sweeps of the transposed factorisation are warp scans of affine
// maps, as in the forward solve.  On entry out[i os] holds gY_i and z[i os] gM_i,
// each written by lane i mod 32.
struct AffT { double p, q; };
__device__ __forceinline__ AffT afft_after(const AffT& g, const AffT& f) {
  AffT r; r.p = g.p * f.p; r.q = fma(g.p, f.q, g.q); return r;
}
// exclusive prefix (over lanes) of the composition of per-lane maps, applied to 0
__device__ __forceinline__ double afft_scan_exclusive(AffT S, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    AffT X;
    X.p = __shfl_up_sync(0xffffffffu, S.p, o);
    X.q = __shfl_up_sync(0xffffffffu, S.q, o);
    if (lane >= o) S = afft_after(S, X);
  }
  const double x = __shfl_up_sync(0xffffffffu, S.q, 1);
  return lane == 0 ? 0.0 : x;
}

__device__ void spline_adjoint_warp(const double* t, const double* ih, int K, const dbl4* fac, double* out,
                                    long long os, double* z, int lane) {
  __syncwarp();
  if (lane == 0) {
    // adjoint of M_0 = (1 + h0/h1) M_1 - (h0/h1) M_2 and of its mirror at the far end
    const double r01 = ih[1] / ih[0], z0 = z[0];
    z[os] += z0 * (1.0 + r01);
    z[2 * os] += -z0 * r01;
    const double rba = ih[K - 3] / ih[K - 2], zl = z[(K - 1) * os];
    z[(K - 2) * os] += zl * (1.0 + rba);
    z[(K - 3) * os] += -zl * rba;
  }
  __syncwarp();
  const int n = K - 2, E = (n + 31) / 32;
  // Tri = L U (L lower bidiagonal: diag m_i, sub a_i; U unit upper: super c'_i);
  // Tri^T lam = g  <=>  U^T w = g, then L^T lam = w.
  // U^T w = g: w_i = g_i - c'_{i-1} w_{i-1}, i = 1 .. K-2 (c'_0 = 0)
  {
    const int i0 = 1 + lane * E, i1 = min(i0 + E, n + 1);
    AffT F = {1.0, 0.0};
    for (int i = i0; i < i1; i++) F = afft_after(AffT{-fac[i - 1].x, z[i * os]}, F);
    double x = afft_scan_exclusive(F, lane);
    for (int i = i0; i < i1; i++) {
      x = fma(-fac[i - 1].x, x, z[i * os]);
      z[i * os] = x;
    }
  }
  __syncwarp();
  // L^T lam = w: lam_i = (w_i - a_{i+1} lam_{i+1}) / m_i, i = K-2 .. 1 (lam_{K-1} = 0)
  {
    const int j0 = n - lane * E, j1 = max(j0 - E, 0);
    auto map = [&](int i) {
      double a = 0.0;                                   // a_{i+1}: sub-diagonal of row i + 1
      if (i + 1 == K - 2) a = (t[K - 2] - t[K - 3]) - (t[K - 1] - t[K - 2]);
      else if (i + 1 < K - 2) a = t[i + 1] - t[i];
      const double y = fac[i].y;                        // 1/m_i
      return AffT{-a * y, z[i * os] * y};
    };
    AffT B = {1.0, 0.0};
    for (int i = j0; i > j1; i--) B = afft_after(map(i), B);
    double x = afft_scan_exclusive(B, lane);
    __syncwarp();
    for (int i = j0; i > j1; i--) {
      const AffT g = map(i);
      x = fma(g.p, x, g.q);
      z[i * os] = x;
    }
  }
  __syncwarp();
  // lam -> y through rhs_i = s_i 6 [(y_{i+1} - y_i)/h_i - (y_i - y_{i-1})/h_{i-1}], rows i = 1 .. K-2
  auto srow = [&](int i) {       // s_i: 1 except the not-a-knot rows
    if (i == 1) return (t[2] - t[1]) / (t[2] - t[0]);
    if (i == K - 2) return (t[K - 2] - t[K - 3]) / (t[K - 1] - t[K - 3]);
    return 1.0;
  };
  for (int j = lane; j < K; j += 32) {
    double v = out[j * os];   // gY_j, written by this lane
    if (j - 1 >= 1 && j - 1 <= K - 2) v += 6.0 * z[(j - 1) * os] * srow(j - 1) * ih[j - 1];
    if (j >= 1 && j <= K - 2) v -= 6.0 * z[j * os] * srow(j) * (ih[j] + ih[j - 1]);
    if (j + 1 <= K - 2) v += 6.0 * z[(j + 1) * os] * srow(j + 1) * ih[j];
    out[j * os] = v;
  }
}

// One warp per series: the four fundamental series of each waveform, then the real and
// imaginary amplitude series of each mode.  Each lane first maps the u-coefficient
// gradients of the segments on either side of its knots to (y, M) gradients (for an
// amplitude series: the record's three sub-piece slots summed, scaled by
// prefactor sqrt(h) scale), then the warp applies the transposed not-a-knot solve.
__global__ void k_spline_adj(int n_wf, const WfInfo* wf, const ModeInfo* modes, long long nm_total, const double* t,
                             const dbl4* fac, const double* ihall, const FundSeg* fund, const double* pref,
                             const double* slots, const double* fseg, long long K_total, double* zf, double* za,
                             double* g_pp, double* g_pr, double* g_op, double* g_or, double* g_amp) {
  long long sid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  long long nfund = 4LL * n_wf;
  if (sid < nfund) {
    int w = (int)(sid >> 2), q = (int)(sid & 3);
    const WfInfo W = wf[w];
    double* outp = q == 0 ? g_pp : q == 1 ? g_pr : q == 2 ? g_op : g_or;
    if (!outp) return;
    double* out = outp + W.ko;
    double* z = zf + q * K_total + W.ko;
    const double* tw = t + W.ko;
    for (int i = lane; i < W.K; i += 32) {
      double gy = 0.0, gM = 0.0;
      if (i < W.K - 1) {
        const double h = tw[i + 1] - tw[i];
        ucoef_adj(fseg + (W.ko + i) * 16 + 4 * q, h * h, 0, gy, gM);
      }
      if (i > 0) {
        const double h = tw[i] - tw[i - 1];
        ucoef_adj(fseg + (W.ko + i - 1) * 16 + 4 * q, h * h, 1, gy, gM);
      }
      out[i] = gy;
      z[i] = gM;
    }
    spline_adjoint_warp(tw, ihall + W.ko, (int)W.K, fac + W.ko, out, 1, z, lane);
    return;
  }
  sid -= nfund;
  if (sid >= 2 * nm_total || !g_amp) return;
  long long j = sid >> 1;
  int part = (int)(sid & 1);
  const ModeInfo M = modes[j];
  const WfInfo W = wf[M.wf];
  double* out = g_amp + 2 * M.key_base + part;
  double* z = za + 2 * M.key_base + part;
  const double* tw = t + W.ko;
  const double pw = pref[M.wf];
  // the amplitude u-coefficient gradients of segment s, summed over its sub-pieces and
  // scaled (sqrt(h) is the fourth entry of the knot segment's Phi_phi record)
  auto seg_coef = [&](int s, double* g) {
    const double* a = slots + (M.seg_base + s) * 3 * 16 + 8 + 4 * part;
    const double sc = pw * fund[W.ko + s].P[0].w * M.scale;
#pragma unroll
    for (int c = 0; c < 4; c++) g[c] = slot_sum(a, c) * sc;
  };
  for (int i = lane; i < W.K; i += 32) {
    double gy = 0.0, gM = 0.0, g[4];
    if (i < W.K - 1) {
      const double h = tw[i + 1] - tw[i];
      seg_coef(i, g);
      ucoef_adj(g, h * h, 0, gy, gM);
    }
    if (i > 0) {
      const double h = tw[i] - tw[i - 1];
      seg_coef(i - 1, g);
      ucoef_adj(g, h * h, 1, gy, gM);
    }
    out[2 * i] = gy;
    z[2 * i] = gM;
  }
  spline_adjoint_warp(tw, ihall + W.ko, (int)W.K, fac + W.ko, out, 2, z, lane);
}

}  // namespace

void launch_loglike(const CallShape& cs, const LikeInputs& li, const DevScratch& s, cudaStream_t st) {
  dim3 g(kLChunks, cs.n_wf);
  k_residual<<<g, 256, 0, st>>>(s.wf, reinterpret_cast<const double2*>(s.hbuf),
                                reinterpret_cast<const double2*>(s.hbuf) + cs.nf_total,
                                reinterpret_cast<const double2*>(li.data_plus),
                                reinterpret_cast<const double2*>(li.data_cross), li.psd, li.df,
                                reinterpret_cast<dbl4*>(s.Gbuf), s.Lpart, s.status);
  k_loglike_final<<<cs.n_wf, 256, 0, st>>>(cs.n_wf, s.Lpart, li.loglike);
}

size_t adjoint_item_bytes() { return sizeof(AdjItem); }

void launch_adjoint(const CallShape& cs, const DevInputs& in, const LikeInputs& li, const DevScratch& s, int num_sms,
                    cudaStream_t st) {
  k_item_len<<<(unsigned)((s.run_cap + 255) / 256), 256, 0, st>>>(s.run_cnt + cs.nm_total, s.runs, s.run_cap,
                                                                  s.item_off);
  launch_scan(s.item_off, s.run_cap, st);
  cudaMemsetAsync(s.slots, 0, sizeof(double) * 48 * (size_t)cs.seg_total, st);
  AdjParams p;
  p.wf = s.wf; p.modes = s.modes; p.core = s.core; p.amp64 = s.amp64; p.crit = s.crit; p.keyF = s.keyF;
  p.runs = s.runs; p.rb = s.rbins; p.freqs = in.freqs; p.G = reinterpret_cast<const dbl4*>(s.Gbuf);
  p.item_off = s.item_off; p.run_cap = s.run_cap; p.tab = s.tab; p.slots = s.slots; p.status = s.status;
  p.items = static_cast<AdjItem*>(s.adj_items); p.adj_off = s.adj_off; p.adj_blk = s.adj_blk; p.bnd = s.adj_bnd; p.bnd_id = s.adj_bnd_id;
  p.nm_total = cs.nm_total; p.seg_total = cs.seg_total; p.nf_total = cs.nf_total;
  // the item slots of this call's segments (at most three runs touch a segment)
  p.item_cap = 3 * cs.seg_total;
  // the bin stream: per-block scans of the items' bin counts, a scan of the block
  // totals, then each item's offset
  const long long nblk = (p.item_cap + kAdjItemBlock - 1) / kAdjItemBlock;
  k_adj_items<<<(unsigned)nblk, kAdjItemBlock, 0, st>>>(p);
  k_scan64<<<1, 1024, 0, st>>>(s.adj_blk, nblk);
  k_adj_offsets<<<(unsigned)((p.item_cap + 256) / 256), 256, 0, st>>>(s.adj_off, s.adj_blk, p.item_cap);
  const size_t smem = (size_t)kAdjWarpsPerCta * 64 * (16 * sizeof(double) + sizeof(int));
  cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long nw = (long long)num_sms * kAdjCtasPerSm * kAdjWarpsPerCta;
  k_adjoint<<<(unsigned)(num_sms * kAdjCtasPerSm), 32 * kAdjWarpsPerCta, smem, st>>>(p);
  k_adj_fixup<<<(unsigned)((nw + 127) / 128), 128, 0, st>>>(p, nw);
  dim3 gs(cs.max_K, cs.n_wf);
  k_fund_seg<<<gs, 256, 0, st>>>(s.wf, s.modes, s.slots, s.fseg);
  long long nser = 4LL * cs.n_wf + 2 * cs.nm_total;
  k_spline_adj<<<(unsigned)((nser * 32 + 255) / 256), 256, 0, st>>>(
      cs.n_wf, s.wf, s.modes, cs.nm_total, in.t, s.spl_fac, s.spl_ih, s.fund, in.prefactor, s.slots, s.fseg,
      cs.K_total, s.zf, s.za, li.g_phi_phi, li.g_phi_r, li.g_omega_phi, li.g_omega_r, li.g_amp);
}

}  // namespace emrifd
