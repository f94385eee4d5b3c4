// Power-based mode selection on the GPU (arXiv 2307.12585, Sec. 2.1).
//
// At each knot t_k the modes' powers P_j = |A_j(t_k)|^2 are ordered by
// decreasing power (equal powers: increasing mode index); their cumulative
// sums S_i are taken in that order one FP64 addition at a time, and the mode
// at position i is kept when S_{i-1} < (1 - eps) S_N.  The selection is the
// union over knots.
//
// One CTA per (knot, waveform): the powers (contraction-free products and
// sums, so that they are the same doubles everywhere) are loaded into shared
// memory with their indices, bitonic-sorted on the key (~bits(P), index)
// (for P >= 0 the bit pattern orders like the value), summed in order by one
// thread (the FP64 additions of the definition, in its order), and every
// thread then marks its positions below the threshold with atomicOr (skipped
// when the flag is already set), which makes the union independent of the
// order in which CTAs finish.
#include "common.cuh"

namespace emrifd {
namespace {

__global__ void __launch_bounds__(1024) k_select(const WfInfo* wf, const double* amp, double eps, int* keep,
                                                  int* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WfInfo W = wf[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= W.K) return;
  const int nm = (int)W.nm;
  int n2 = 1;
  while (n2 < nm) n2 <<= 1;
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem);
  int* idx = reinterpret_cast<int*>(key + n2);
  double* S = reinterpret_cast<double*>(smem) + n2 + (n2 + 1) / 2;   // after key and idx (8-byte aligned)
  __shared__ double thr;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n2; i += nt) {
    if (i < nm) {
      const double* a = amp + 2 * (W.amp_base + (long long)i * W.K + k);
      const double P = __dadd_rn(__dmul_rn(a[0], a[0]), __dmul_rn(a[1], a[1]));
      if (!(fabs(P) < INFINITY)) atomicOr(status, ST_NONFINITE);
      key[i] = ~(unsigned long long)__double_as_longlong(P);
      idx[i] = i;
    } else {
      key[i] = ~0ull;
      idx[i] = 0x7FFFFFFF;
    }
  }
  __syncthreads();
  // bitonic sort, ascending on (key, idx)
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < n2 / 2; i += nt) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long ka = key[lo], kb = key[hi];
        const int ia = idx[lo], ib = idx[hi];
        const bool gt = ka > kb || (ka == kb && ia > ib);
        if (gt == up) {
          key[lo] = kb; key[hi] = ka;
          idx[lo] = ib; idx[hi] = ia;
        }
      }
      __syncthreads();
    }
  }
  // cumulative sums in the sorted order, one addition at a time
  if (tid == 0) {
    // the keys are read 16 at a time ahead of the additions, so that the chain
    // of dependent FP64 additions is not also serialised behind shared-memory
    // stores to S (which the compiler must assume may alias the keys)
    double s = 0.0;
    for (int i0 = 0; i0 < nm; i0 += 16) {
      double v[16];
#pragma unroll
      for (int q = 0; q < 16; q++) v[q] = i0 + q < nm ? __longlong_as_double((long long)~key[i0 + q]) : 0.0;
      double b[16];
#pragma unroll
      for (int q = 0; q < 16; q++) {
        b[q] = s;                                          // power before position i0 + q
        s = __dadd_rn(s, v[q]);
      }
#pragma unroll
      for (int q = 0; q < 16; q++)
        if (i0 + q < nm) S[i0 + q] = b[q];
    }
    thr = __dmul_rn(__dsub_rn(1.0, eps), s);
  }
  __syncthreads();
  // a mode kept at many knots is set once: the plain read skips the atomic when an
  // earlier CTA has already set it (a stale 0 only costs a redundant atomicOr)
  for (int i = tid; i < nm; i += nt) {
    int* dst = keep + W.mo + idx[i];
    if (S[i] < thr && *reinterpret_cast<volatile int*>(dst) == 0) atomicOr(dst, 1);
  }
}

}  // namespace

size_t select_smem_bytes(long long max_modes) {
  long long n2 = 1;
  while (n2 < max_modes) n2 <<= 1;
  return (size_t)(8 * n2 + 8 * ((n2 + 1) / 2) + 8 * n2);
}

void launch_select(const DevScratch& s, int n_wf, int max_K, long long max_nm, const double* amp, double eps,
                   int* keep, long long nm_total, cudaStream_t st) {
  cudaMemsetAsync(keep, 0, sizeof(int) * (size_t)(nm_total > 0 ? nm_total : 1), st);
  const size_t sm = select_smem_bytes(max_nm);
  cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_select<<<dim3((unsigned)max_K, (unsigned)n_wf), 1024, sm, st>>>(s.wf, amp, eps, keep, s.status);
}

}  // namespace emrifd
