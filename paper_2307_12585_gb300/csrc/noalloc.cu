// emri_fd_sum_modes_noalloc: the SPA mode sum of one waveform without any
// device allocation.
//
// Some callers cannot allocate device memory: code that runs while another
// component (for example a framework's caching allocator) already holds the
// device's memory, so that cudaMalloc can fail; latency-critical code for
// which cudaMalloc / cudaFree, which may synchronise the device, are not
// acceptable; and plug-ins or callbacks that are not allowed to call the
// allocator at all.  For them this entry point runs the same kernels as
// emri_fd_sum_modes, but with all scratch in one file-scope device array of
// fixed size (below), which every GPU that loads the library holds until the
// process exits.  The caller passes device inputs and outputs.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/emri_fd.h"
#include "common.cuh"

using namespace emrifd;

namespace {

constexpr long long kNaMaxK = EMRI_FD_NOALLOC_MAX_KNOTS;
constexpr long long kNaMaxModes = EMRI_FD_NOALLOC_MAX_MODES;
constexpr long long kNaMaxSeg = kNaMaxModes * (kNaMaxK - 1);
constexpr long long kNaMaxAmp = kNaMaxModes * kNaMaxK;
constexpr long long kNaRunCap = 12 * kNaMaxModes + 64;

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets of the sub-arrays inside the scratch array
constexpr size_t kOffStatus = 0;
constexpr size_t kOffCounters = kOffStatus + al256(sizeof(int));
constexpr size_t kOffWf = kOffCounters + al256(8 * sizeof(unsigned long long));
constexpr size_t kOffAngles = kOffWf + al256(sizeof(WfInfo));
constexpr size_t kOffModes = kOffAngles + al256(3 * sizeof(double));
constexpr size_t kOffFac = kOffModes + al256(kNaMaxModes * sizeof(ModeInfo));
constexpr size_t kOffIh = kOffFac + al256(kNaMaxK * sizeof(dbl4));
constexpr size_t kOffFundM = kOffIh + al256(kNaMaxK * sizeof(double));
constexpr size_t kOffFund = kOffFundM + al256(4 * kNaMaxK * sizeof(double));
constexpr size_t kOffAmpM = kOffFund + al256(kNaMaxK * sizeof(FundSeg));
constexpr size_t kOffCore = kOffAmpM + al256(2 * kNaMaxAmp * sizeof(double));
constexpr size_t kOffAmp64 = kOffCore + al256(kNaMaxSeg * sizeof(SegCore));
constexpr size_t kOffCrit = kOffAmp64 + al256(kNaMaxSeg * sizeof(SegAmp64));
constexpr size_t kOffKeyF = kOffCrit + al256(kNaMaxSeg * sizeof(SegCrit));
constexpr size_t kOffRunCnt = kOffKeyF + al256(kNaMaxAmp * sizeof(long long));
constexpr size_t kOffRuns = kOffRunCnt + al256((kNaMaxModes + 1) * sizeof(int));
constexpr size_t kOffRunF = kOffRuns + al256(kNaRunCap * sizeof(Run));
constexpr size_t kOffRbins = kOffRunF + al256(kNaRunCap * sizeof(double2));
constexpr size_t kOffTab = kOffRbins + al256(kNaRunCap * sizeof(RunBins));
constexpr size_t kNaBytes = kOffTab + al256(kTab64N * sizeof(double2));
static_assert(kNaBytes == 7555328, "the size stated in include/emri_fd.h");

// The scratch.  In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_dev_ptr[kNaMaxDevices] = {};

// writes the per-call waveform descriptor and the per-waveform scalars
__global__ void k_noalloc_set(WfInfo w, double theta, double phi, double pref, WfInfo* dst, double* ang) {
  *dst = w;
  ang[0] = theta;
  ang[1] = phi;
  ang[2] = pref;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// once per device, with that device current: the scratch's device address and
// the e^{2 pi i k/65536} table the output kernel reads
emri_fd_status setup(int dev, cudaStream_t st, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_dev_ptr[dev]) { *out = g_dev_ptr[dev]; return EMRI_FD_OK; }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return EMRI_FD_ERR_CUDA;
  }
  unsigned char* base = static_cast<unsigned char*>(p);
  launch_table(reinterpret_cast<double2*>(base + kOffTab), st);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return EMRI_FD_ERR_CUDA;
  g_dev_ptr[dev] = base;
  *out = base;
  return EMRI_FD_OK;
}

}  // namespace

extern "C" emri_fd_status emri_fd_sum_modes_noalloc(int conj_partners, long long n_knots, long long n_modes,
                                                    long long n_freqs, const double* t, const double* phi_phi,
                                                    const double* phi_r, const double* omega_phi,
                                                    const double* omega_r, const int* l, const int* m, const int* n,
                                                    const double* amp, double theta, double phi, double prefactor,
                                                    const double* freqs, void* h_plus, void* h_cross, void* stream) {
  if (conj_partners != 0 && conj_partners != 1) return EMRI_FD_ERR_ARG;
  if (n_knots < 4) return EMRI_FD_ERR_KNOTS;
  if (n_modes < 1 || n_freqs < 1) return EMRI_FD_ERR_ARG;
  if (n_knots > kNaMaxK || n_modes > kNaMaxModes || n_freqs > EMRI_FD_NOALLOC_MAX_BINS) return EMRI_FD_ERR_CAPACITY;
  const void* dptrs[] = {t, phi_phi, phi_r, omega_phi, omega_r, l, m, n, amp, freqs, h_plus, h_cross};
  for (const void* q : dptrs)
    if (q == nullptr || !on_device(q)) return EMRI_FD_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  if (dev < 0 || dev >= kNaMaxDevices) return EMRI_FD_ERR_CUDA;
  unsigned char* base = nullptr;
  emri_fd_status s0 = setup(dev, st, &base);
  if (s0 != EMRI_FD_OK) return s0;

  DevScratch s{};
  s.status = reinterpret_cast<int*>(base + kOffStatus);
  s.counters = reinterpret_cast<unsigned long long*>(base + kOffCounters);
  s.wf = reinterpret_cast<WfInfo*>(base + kOffWf);
  s.modes = reinterpret_cast<ModeInfo*>(base + kOffModes);
  s.spl_fac = reinterpret_cast<dbl4*>(base + kOffFac);
  s.spl_ih = reinterpret_cast<double*>(base + kOffIh);
  s.fundM = reinterpret_cast<double*>(base + kOffFundM);
  s.fund = reinterpret_cast<FundSeg*>(base + kOffFund);
  s.ampM = reinterpret_cast<double*>(base + kOffAmpM);
  s.core = reinterpret_cast<SegCore*>(base + kOffCore);
  s.amp64 = reinterpret_cast<SegAmp64*>(base + kOffAmp64);
  s.amp32 = nullptr;
  s.crit = reinterpret_cast<SegCrit*>(base + kOffCrit);
  s.keyF = reinterpret_cast<long long*>(base + kOffKeyF);
  s.run_cnt = reinterpret_cast<int*>(base + kOffRunCnt);
  s.runs = reinterpret_cast<Run*>(base + kOffRuns);
  s.runF = reinterpret_cast<double2*>(base + kOffRunF);
  s.rbins = reinterpret_cast<RunBins*>(base + kOffRbins);
  s.run_cap = kNaRunCap;
  s.tab = reinterpret_cast<double2*>(base + kOffTab);
  double* ang = reinterpret_cast<double*>(base + kOffAngles);

  const int TB = 128;
  WfInfo W{};
  W.ko = 0; W.K = n_knots; W.mo = 0; W.nm = n_modes; W.fo = 0; W.nf = n_freqs;
  W.amp_base = 0; W.seg_base = 0; W.tile_base = 0; W.ntiles = (n_freqs + TB - 1) / TB;
  CallShape cs{};
  cs.n_wf = 1; cs.K_total = n_knots; cs.nm_total = n_modes; cs.nf_total = n_freqs;
  cs.seg_total = n_modes * (n_knots - 1); cs.amp_total = n_modes * n_knots; cs.tiles_total = W.ntiles;
  cs.max_K = (int)n_knots; cs.tile_bins = TB; cs.conj = conj_partners; cs.precision = EMRI_FD_FP64;
  DevInputs in{};
  in.t = t; in.phi_phi = phi_phi; in.phi_r = phi_r; in.omega_phi = omega_phi; in.omega_r = omega_r;
  in.l = l; in.m = m; in.n = n; in.amp = amp; in.theta = ang; in.phi = ang + 1; in.prefactor = ang + 2;
  in.freqs = freqs; in.h_plus = h_plus; in.h_cross = h_cross;

  // the array keeps the previous call's contents: reset the status word and
  // counters (everything else is fully rewritten before it is read)
  cudaMemsetAsync(s.status, 0, sizeof(int), st);
  cudaMemsetAsync(s.counters, 0, 8 * sizeof(unsigned long long), st);
  k_noalloc_set<<<1, 1, 0, st>>>(W, theta, phi, prefactor, s.wf, ang);
  launch_prep(cs, in, s, st);
  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return EMRI_FD_ERR_CUDA;
  }
  launch_spa(cs, in, s, num_sms, st);
  if (cudaGetLastError() != cudaSuccess) return EMRI_FD_ERR_CUDA;
  int hs = 0;
  if (cudaMemcpyAsync(&hs, s.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return EMRI_FD_ERR_CUDA;
  }
  if (hs & ST_KNOTS) return EMRI_FD_ERR_KNOTS;
  if (hs & ST_FREQ) return EMRI_FD_ERR_FREQ;
  if (hs & ST_MODE) return EMRI_FD_ERR_MODE;
  if (hs & ST_NONFINITE) return EMRI_FD_ERR_NONFINITE;
  if (hs & ST_CAPACITY) return EMRI_FD_ERR_CAPACITY;
  if (hs & ST_BOUNDS) return EMRI_FD_ERR_INTERNAL;
  return EMRI_FD_OK;
}
