// Hann window applied in the frequency domain (arXiv 2307.12585, Sec. 2.3):
// the time-domain signal is multiplied by w(t) = sin^2(pi t df) on [0, 1/df],
// i.e. w = 1/2 - e^{2 pi i t df}/4 - e^{-2 pi i t df}/4, so with the Fourier
// sign of Eq. 3 its transform is the three-term convolution
//   h_w(f) = h(f)/2 - h(f + df)/4 - h(f - df)/4
// on a uniform grid of spacing df.  Bins outside the waveform's grid count as 0.
//
// One thread per output bin; the neighbours are read through L1/L2 (each input
// is read about once from HBM).  Grid: x over bins, y over waveforms.  A grid
// whose spacing differs from its mean by more than 1e-6 relative is flagged
// with the ST_FREQ status bit.  (GB300's FP64 rate, not HBM, bounds this
// kernel: the FP64 stencil takes 12 FP64 operations per bin.)
#include "common.cuh"

namespace emrifd {
namespace {

template <typename C>
struct CplxOps;
template <>
struct CplxOps<double2> {
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ double2 hann(double2 a, double2 lo, double2 hi) {
    return make_double2(fma(0.5, a.x, -0.25 * (lo.x + hi.x)), fma(0.5, a.y, -0.25 * (lo.y + hi.y)));
  }
};
template <>
struct CplxOps<float2> {
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 hann(float2 a, float2 lo, float2 hi) {
    return make_float2(fmaf(0.5f, a.x, -0.25f * (lo.x + hi.x)), fmaf(0.5f, a.y, -0.25f * (lo.y + hi.y)));
  }
};

template <typename C>
__global__ void k_hann(const WfInfo* wf, const double* freqs, const C* __restrict__ inp, const C* __restrict__ inc,
                       C* __restrict__ outp, C* __restrict__ outc, int* status) {
  const WfInfo W = wf[blockIdx.y];
  const long long nf = W.nf, fo = W.fo;
  // spacing check without a division: |(f[i+1] - f[i]) (n - 1) - (f[n-1] - f[0])| <= 1e-6 (f[n-1] - f[0])
  const double span = nf > 1 ? freqs[fo + nf - 1] - freqs[fo] : 0.0, nm1 = (double)(nf - 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    const long long b = fo + i;
    const C z = CplxOps<C>::zero();
    const bool has_lo = i > 0, has_hi = i + 1 < nf;
    outp[b] = CplxOps<C>::hann(inp[b], has_lo ? inp[b - 1] : z, has_hi ? inp[b + 1] : z);
    outc[b] = CplxOps<C>::hann(inc[b], has_lo ? inc[b - 1] : z, has_hi ? inc[b + 1] : z);
    if (has_hi && fabs(fma(freqs[b + 1] - freqs[b], nm1, -span)) > 1e-6 * span) atomicOr(status, ST_FREQ);
  }
}

}  // namespace

void launch_window(const CallShape& cs, const DevScratch& s, const double* freqs, const void* in_p, const void* in_c,
                   void* out_p, void* out_c, int num_sms, cudaStream_t st) {
  if (cs.n_wf <= 0 || cs.nf_total <= 0) return;
  const long long per_wf = (cs.nf_total + cs.n_wf - 1) / cs.n_wf;
  long long bx = (per_wf + 255) / 256;
  const long long cap = 64LL * num_sms;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  const dim3 grid((unsigned)bx, (unsigned)cs.n_wf);
  if (cs.precision == 1)   // mixed plans: complex64 outputs
    k_hann<float2><<<grid, 256, 0, st>>>(s.wf, freqs, static_cast<const float2*>(in_p), static_cast<const float2*>(in_c),
                                         static_cast<float2*>(out_p), static_cast<float2*>(out_c), s.status);
  else
    k_hann<double2><<<grid, 256, 0, st>>>(s.wf, freqs, static_cast<const double2*>(in_p),
                                          static_cast<const double2*>(in_c), static_cast<double2*>(out_p),
                                          static_cast<double2*>(out_c), s.status);
}

}  // namespace emrifd
