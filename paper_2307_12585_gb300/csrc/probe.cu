// Peak-rate probe of the FP64 and FP32 fused multiply-add pipes.
//
// Not part of the paper's method: it measures the denominator that the SPA
// kernels' FP64 (and FP32) roofline fractions are quoted against.  Every thread
// runs kChains independent FMA recurrences x <- x a + b, so that each SM
// sub-partition always has independent FMAs to issue (16 resident warps x 8
// chains per sub-partition against a pipe latency of a few cycles); the chains'
// sum is stored only under a condition that never holds for these values, which
// keeps the compiler from removing them.  The caller times a launch with CUDA
// events on `stream`.
#include "../../include/emri_fd.h"
#include <cuda_runtime.h>

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;   // FMAs per chain per loop iteration

__device__ double g_probe_sink;   // written only if the impossible test below holds

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) x[j] = (T)(threadIdx.x + 1 + j) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < kUnroll; r++)
#pragma unroll
      for (int j = 0; j < kChains; j++) x[j] = fma(x[j], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += x[j];
  if (s == (T)-1) g_probe_sink = (double)s;   // x stays positive: never true
}

}  // namespace

extern "C" emri_fd_status emri_fd_fma_probe(int precision, int iters, int blocks_per_sm, void* stream,
                                            long long* fma_per_launch) {
  if ((precision != 0 && precision != 1) || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64)
    return EMRI_FD_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return EMRI_FD_ERR_CUDA;
  }
  const long long grid = (long long)sms * blocks_per_sm;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a = 1 - 2^-20 and b = 2^-30 keep every chain positive and bounded (it tends to b/(1 - a))
  if (precision == 0)
    k_fma_probe<double><<<(unsigned)grid, kProbeThreads, 0, st>>>(iters, 1.0 - 0x1p-20, 0x1p-30);
  else
    k_fma_probe<float><<<(unsigned)grid, kProbeThreads, 0, st>>>(iters, 1.0f - 0x1p-20f, 0x1p-30f);
  if (cudaGetLastError() != cudaSuccess) return EMRI_FD_ERR_CUDA;
  if (fma_per_launch) *fma_per_launch = grid * kProbeThreads * (long long)iters * kUnroll * kChains;
  return EMRI_FD_OK;
}
