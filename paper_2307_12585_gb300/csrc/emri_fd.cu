// C ABI of the GB300 SPA mode sum: plan lifetime, host-side validation,
// host-pointer staging and the launch sequence (see include/emri_fd.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cufft.h>
#include <nvtx3/nvToolsExt.h>   // header-only NVTX: ranges are no-ops unless a profiler attaches

#include "../../include/emri_fd.h"
#include "common.cuh"

using namespace emrifd;

struct emri_fd_plan_s {
  emri_fd_desc desc;
  cudaStream_t stream;
  int device = 0, num_sms = 0;
  long long cap_K = 0, cap_nm = 0, cap_nf = 0, cap_seg = 0, cap_amp = 0;
  DevScratch s{};
  WfInfo* wf_pinned = nullptr;       // host copy uploaded each call
  cudaEvent_t wf_done = nullptr;     // guards reuse of wf_pinned
  // host frequency grids of emri_fd_sum_modes are copied on a side stream while the
  // preparation kernels that do not read them run
  cudaStream_t side = nullptr;
  cudaEvent_t ev_main = nullptr, ev_freqs = nullptr;
  bool freqs_side = false;           // the next run_forward waits for ev_freqs
  unsigned long long* cnt_pinned = nullptr;
  int* st_pinned = nullptr;          // the status word read back by synchronising calls
  // staging for host-memory inputs / outputs
  void* stage[32] = {};
  size_t stage_sz[32] = {};
  // last call's shape (for stats)
  long long last_tiles = 0, last_nm = 0;
  // optional event timing of the output kernel and of the preparation kernels
  bool profiling = false;
  std::vector<cudaEvent_t> ev;       // triples (prep start, spa start, spa end) per call
  int ev_used = 0;
  long long launches = 0;            // kernels launched by calls since the last profile reset
  std::vector<void*> allocs;
  // time-domain comparator: per-(mode, segment) FP32 amplitude coefficients,
  // and FFT plans and buffer (made on first use)
  float4* tdamp = nullptr;
  std::vector<std::pair<long long, cufftHandle>> fft_plans;
  float2* zbuf = nullptr;
  long long zcap = 0;
};

namespace {


template <typename T>
emri_fd_status dalloc(emri_fd_plan_s* p, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_OOM; }
  p->allocs.push_back(q);
  *ptr = static_cast<T*>(q);
  return EMRI_FD_OK;
}

bool is_device_ptr(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// returns a device pointer holding `bytes` of src (staged through a plan buffer if src is host memory)
emri_fd_status stage_in(emri_fd_plan_s* p, int slot, const void* src, size_t bytes, const void** out) {
  if (bytes == 0 || is_device_ptr(src)) { *out = src; return EMRI_FD_OK; }
  if (p->stage_sz[slot] < bytes) {
    if (p->stage[slot]) cudaFree(p->stage[slot]);
    p->stage[slot] = nullptr;
    p->stage_sz[slot] = 0;
    if (cudaMalloc(&p->stage[slot], bytes) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_OOM; }
    p->stage_sz[slot] = bytes;
  }
  if (cudaMemcpyAsync(p->stage[slot], src, bytes, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
    return EMRI_FD_ERR_CUDA;
  *out = p->stage[slot];
  return EMRI_FD_OK;
}

}  // namespace

extern "C" {

const char* emri_fd_strerror(emri_fd_status s) {
  switch (s) {
    case EMRI_FD_OK: return "ok";
    case EMRI_FD_ERR_ARG: return "invalid argument";
    case EMRI_FD_ERR_KNOTS: return "knots: fewer than 4 or times not strictly increasing";
    case EMRI_FD_ERR_FREQ: return "frequencies not strictly increasing or not positive";
    case EMRI_FD_ERR_MODE: return "invalid mode numbers";
    case EMRI_FD_ERR_NONFINITE: return "non-finite input value";
    case EMRI_FD_ERR_CAPACITY: return "size above the plan's capacity";
    case EMRI_FD_ERR_CUDA: return "CUDA runtime error";
    case EMRI_FD_ERR_OOM: return "device allocation failed";
    case EMRI_FD_ERR_TIMEOUT: return "bounded device wait timed out (reserved; not returned by this version)";
    case EMRI_FD_ERR_INTERNAL: return "a device-side index check failed (checked builds)";
  }
  return "unknown status";
}

void emri_fd_plan_destroy(emri_fd_plan_t p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  for (void* q : p->allocs) cudaFree(q);
  for (int i = 0; i < 32; i++) if (p->stage[i]) cudaFree(p->stage[i]);
  if (p->wf_pinned) cudaFreeHost(p->wf_pinned);
  if (p->cnt_pinned) cudaFreeHost(p->cnt_pinned);
  if (p->st_pinned) cudaFreeHost(p->st_pinned);
  if (p->wf_done) cudaEventDestroy(p->wf_done);
  if (p->side) { cudaStreamSynchronize(p->side); cudaStreamDestroy(p->side); }
  if (p->ev_main) cudaEventDestroy(p->ev_main);
  if (p->ev_freqs) cudaEventDestroy(p->ev_freqs);
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  for (auto& fp : p->fft_plans) cufftDestroy(fp.second);
  if (p->zbuf) cudaFree(p->zbuf);
  cudaGetLastError();
  delete p;
}

emri_fd_status emri_fd_plan(emri_fd_plan_t* out, const emri_fd_desc* d, void* stream) {
  if (!out || !d) return EMRI_FD_ERR_ARG;
  *out = nullptr;
  if ((d->precision != EMRI_FD_FP64 && d->precision != EMRI_FD_MIXED && d->precision != EMRI_FD_FP64X) || (d->conj_partners != 0 && d->conj_partners != 1) ||
      d->max_waveforms < 1 || d->max_waveforms > 65535 || d->max_knots < 4 || d->max_modes_total < 1 || d->max_bins_total < 1 ||
      d->max_bins_total > 2000000000LL || d->max_knots_total < 0 ||
      !(d->tile_bins == 0 || d->tile_bins == 32 || d->tile_bins == 64 || d->tile_bins == 128))
    return EMRI_FD_ERR_ARG;
  for (int i = 0; i < 2; i++) if (d->reserved[i] != 0) return EMRI_FD_ERR_ARG;
  if (!(d->tile_split == 0 || d->tile_split == 1 || d->tile_split == 2 || d->tile_split == 4)) return EMRI_FD_ERR_ARG;
  if (d->tile_split > 1 && !(d->tile_bins == 32 || d->tile_bins == 64)) return EMRI_FD_ERR_ARG;
  if (d->time_domain != 0 && d->time_domain != 1) return EMRI_FD_ERR_ARG;
  if (d->window != EMRI_FD_WINDOW_NONE && d->window != EMRI_FD_WINDOW_HANN) return EMRI_FD_ERR_ARG;
  if (d->window != EMRI_FD_WINDOW_NONE && d->likelihood) return EMRI_FD_ERR_ARG;
  if (d->spa_form != EMRI_FD_SPA_STANDARD && d->spa_form != EMRI_FD_SPA_EXTENDED) return EMRI_FD_ERR_ARG;
  if (d->likelihood != 0 &&
      (d->likelihood != 1 || d->precision != EMRI_FD_FP64 || d->spa_form != EMRI_FD_SPA_STANDARD))
    return EMRI_FD_ERR_ARG;
  emri_fd_plan_s* p = new emri_fd_plan_s();
  p->desc = *d;
  if (p->desc.tile_bins == 0) p->desc.tile_bins = 128;
  p->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    cudaGetLastError(); delete p; return EMRI_FD_ERR_CUDA;
  }
  p->cap_K = d->max_knots_total > 0 ? d->max_knots_total : (long long)d->max_waveforms * d->max_knots;
  p->cap_nm = d->max_modes_total;
  p->cap_nf = d->max_bins_total;
  p->cap_seg = d->max_modes_total * (long long)(d->max_knots - 1);
  p->cap_amp = d->max_modes_total * (long long)d->max_knots;
  DevScratch& s = p->s;
  s.run_cap = 12 * d->max_modes_total + 64;
  emri_fd_status st = EMRI_FD_OK;
#define AL(ptr, n) if (st == EMRI_FD_OK) st = dalloc(p, &(ptr), (size_t)(n))
  AL(s.status, 1);
  AL(s.counters, 8);
  AL(s.wf, d->max_waveforms);
  AL(s.modes, p->cap_nm);
  AL(s.spl_fac, p->cap_K);
  AL(s.spl_ih, p->cap_K);
  AL(s.fundM, 4 * p->cap_K);
  AL(s.fund, p->cap_K);
  AL(s.ampM, 2 * p->cap_amp);
  AL(s.core, p->cap_seg);
  if (d->precision == EMRI_FD_FP64) { AL(s.amp64, p->cap_seg); }
  else if (d->precision == EMRI_FD_MIXED) { AL(s.amp32, p->cap_seg); }
  else { AL(s.segff, p->cap_seg); AL(s.tabf, kTabN); }
  AL(s.crit, p->cap_seg);
  if (d->spa_form == EMRI_FD_SPA_EXTENDED && d->precision == EMRI_FD_FP64) { AL(s.yk, p->cap_seg); }
  if (d->time_domain) {
    float4* ta = nullptr;
    AL(ta, 2 * p->cap_seg);
    p->tdamp = ta;
  }
  if (d->window == EMRI_FD_WINDOW_HANN) {
    unsigned char *wp = nullptr, *wc = nullptr;
    const long long ob = (d->precision == EMRI_FD_MIXED ? 8 : 16) * p->cap_nf;
    AL(wp, ob);
    AL(wc, ob);
    s.wbuf_p = wp;
    s.wbuf_c = wc;
  }
  AL(s.keyF, p->cap_amp);
  AL(s.run_cnt, p->cap_nm + 1);
  AL(s.runs, s.run_cap);
  AL(s.runF, s.run_cap);
  AL(s.rbins, s.run_cap);
  AL(s.tab, kTab64N);
  if (d->likelihood) {
    AL(s.hbuf, 4 * p->cap_nf);
    AL(s.Gbuf, 4 * p->cap_nf);
    AL(s.Lpart, (long long)kLChunks * d->max_waveforms);
    AL(s.item_off, s.run_cap + 1);
    s.adj_item_cap = 3 * p->cap_seg;
    {
      unsigned char* ai = nullptr;
      AL(ai, adjoint_item_bytes() * (size_t)s.adj_item_cap);
      s.adj_items = ai;
    }
    AL(s.adj_off, s.adj_item_cap + 1);
    AL(s.adj_blk, (s.adj_item_cap + kAdjItemBlock - 1) / kAdjItemBlock + 1);
    AL(s.adj_bnd, 32LL * kAdjCtasPerSm * kAdjWarpsPerCta * p->num_sms);
    AL(s.adj_bnd_id, 2LL * kAdjCtasPerSm * kAdjWarpsPerCta * p->num_sms);
    AL(s.slots, 48 * p->cap_seg);
    AL(s.za, 2 * p->cap_amp);
    AL(s.zf, 4 * p->cap_K);
    AL(s.fseg, 16 * p->cap_K);
  }
#undef AL
  if (st == EMRI_FD_OK && (cudaMallocHost(&p->wf_pinned, sizeof(WfInfo) * d->max_waveforms) != cudaSuccess ||
                           cudaMallocHost(&p->cnt_pinned, sizeof(unsigned long long) * 8) != cudaSuccess ||
                           cudaMallocHost(&p->st_pinned, sizeof(int)) != cudaSuccess ||
                           cudaEventCreateWithFlags(&p->wf_done, cudaEventDisableTiming) != cudaSuccess ||
                           cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
                           cudaEventCreateWithFlags(&p->ev_main, cudaEventDisableTiming) != cudaSuccess ||
                           cudaEventCreateWithFlags(&p->ev_freqs, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    st = EMRI_FD_ERR_OOM;
  }
  if (st == EMRI_FD_OK) {
    cudaMemsetAsync(s.status, 0, sizeof(int), p->stream);
    cudaMemsetAsync(s.counters, 0, 8 * sizeof(unsigned long long), p->stream);
    launch_table(s.tab, p->stream);
    if (s.tabf) launch_table_ff(s.tab, s.tabf, p->stream);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess) st = EMRI_FD_ERR_CUDA;
  }
  if (st != EMRI_FD_OK) { emri_fd_plan_destroy(p); return st; }
  *out = p;
  return EMRI_FD_OK;
}

}  // extern "C"

namespace {

// host-side shape checks, per-waveform table, input staging (shared by the
// two computing entry points); on success the waveform table is uploaded
emri_fd_status prepare_call(emri_fd_plan_s* p, int n_wf, const long long* knot_off, const long long* mode_off,
                            const long long* freq_off, const double* t, const double* phi_phi, const double* phi_r,
                            const double* omega_phi, const double* omega_r, const int* l, const int* m, const int* n,
                            const double* amp, const double* theta, const double* phi, const double* prefactor,
                            const double* freqs, CallShape& cs, DevInputs& in, bool freqs_on_side = false) {
  if (!p || n_wf < 1 || !knot_off || !mode_off || !freq_off) return EMRI_FD_ERR_ARG;
  if (n_wf > p->desc.max_waveforms) return EMRI_FD_ERR_CAPACITY;
  if (knot_off[0] != 0 || mode_off[0] != 0 || freq_off[0] != 0) return EMRI_FD_ERR_ARG;
  const int TB = p->desc.tile_bins;
  // the pinned table may still be read by the previous call's copy
  if (cudaEventSynchronize(p->wf_done) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  cs = CallShape{};
  cs.n_wf = n_wf;
  cs.tile_bins = TB;
  cs.tile_split = p->desc.tile_split > 1 ? p->desc.tile_split : 1;
  cs.conj = p->desc.conj_partners;
  cs.precision = p->desc.precision;
  cs.ext = p->desc.spa_form;
  cs.window = p->desc.window;
  long long amp_base = 0, seg_base = 0, tiles = 0;
  int maxK = 0;
  for (int w = 0; w < n_wf; w++) {
    long long K = knot_off[w + 1] - knot_off[w], nm = mode_off[w + 1] - mode_off[w], nf = freq_off[w + 1] - freq_off[w];
    if (K < 0 || nm < 0 || nf < 0) return EMRI_FD_ERR_ARG;
    if (K < 4) return EMRI_FD_ERR_KNOTS;
    if (K > p->desc.max_knots) return EMRI_FD_ERR_CAPACITY;
    WfInfo& W = p->wf_pinned[w];
    W.ko = knot_off[w]; W.K = K; W.mo = mode_off[w]; W.nm = nm; W.fo = freq_off[w]; W.nf = nf;
    W.amp_base = amp_base; W.seg_base = seg_base;
    W.tile_base = tiles; W.ntiles = (nf + TB - 1) / TB;
    W.run_base = 0; W.nruns = 0;
    amp_base += nm * K;
    seg_base += nm * (K - 1);
    tiles += W.ntiles;
    if (K > maxK) maxK = (int)K;
  }
  cs.K_total = knot_off[n_wf];
  cs.nm_total = mode_off[n_wf];
  cs.nf_total = freq_off[n_wf];
  cs.seg_total = seg_base;
  cs.amp_total = amp_base;
  cs.tiles_total = tiles;
  cs.max_K = maxK;
  if (cs.K_total > p->cap_K || cs.nm_total > p->cap_nm || cs.nf_total > p->cap_nf || cs.seg_total > p->cap_seg ||
      cs.amp_total > p->cap_amp)
    return EMRI_FD_ERR_CAPACITY;
  if (!t || !phi_phi || !phi_r || !omega_phi || !omega_r || !theta || !phi || !prefactor) return EMRI_FD_ERR_ARG;
  if (cs.nm_total > 0 && (!l || !m || !n || !amp)) return EMRI_FD_ERR_ARG;
  if (cs.nf_total > 0 && !freqs) return EMRI_FD_ERR_ARG;

  in = DevInputs{};
  emri_fd_status st = EMRI_FD_OK;
  const size_t kb = sizeof(double) * cs.K_total;
  const void* q;
#define STG(slot, ptr, bytes, field, type)                            \
  if (st == EMRI_FD_OK) {                                               \
    st = stage_in(p, slot, ptr, bytes, &q);                             \
    in.field = static_cast<type>(q);                                    \
  }
  STG(0, t, kb, t, const double*);
  STG(1, phi_phi, kb, phi_phi, const double*);
  STG(2, phi_r, kb, phi_r, const double*);
  STG(3, omega_phi, kb, omega_phi, const double*);
  STG(4, omega_r, kb, omega_r, const double*);
  STG(5, l, sizeof(int) * cs.nm_total, l, const int*);
  STG(6, m, sizeof(int) * cs.nm_total, m, const int*);
  STG(7, n, sizeof(int) * cs.nm_total, n, const int*);
  STG(8, amp, 2 * sizeof(double) * cs.amp_total, amp, const double*);
  STG(9, theta, sizeof(double) * n_wf, theta, const double*);
  STG(10, phi, sizeof(double) * n_wf, phi, const double*);
  STG(11, prefactor, sizeof(double) * n_wf, prefactor, const double*);
  if (freqs_on_side && cs.nf_total > 0 && !is_device_ptr(freqs)) {
    // staged on the side stream after the main stream's earlier readers of the buffer
    const size_t fb = sizeof(double) * cs.nf_total;
    if (p->stage_sz[12] < fb) {
      if (p->stage[12]) { cudaStreamSynchronize(p->stream); cudaFree(p->stage[12]); }
      p->stage[12] = nullptr;
      p->stage_sz[12] = 0;
      if (cudaMalloc(&p->stage[12], fb) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_OOM; }
      p->stage_sz[12] = fb;
    }
    if (cudaEventRecord(p->ev_main, p->stream) != cudaSuccess || cudaStreamWaitEvent(p->side, p->ev_main, 0) != cudaSuccess ||
        cudaMemcpyAsync(p->stage[12], freqs, fb, cudaMemcpyHostToDevice, p->side) != cudaSuccess ||
        cudaEventRecord(p->ev_freqs, p->side) != cudaSuccess)
      return EMRI_FD_ERR_CUDA;
    in.freqs = static_cast<const double*>(p->stage[12]);
    p->freqs_side = true;
  } else {
    STG(12, freqs, sizeof(double) * cs.nf_total, freqs, const double*);
  }
#undef STG
  if (st != EMRI_FD_OK) return st;
  if (cudaMemcpyAsync(p->s.wf, p->wf_pinned, sizeof(WfInfo) * n_wf, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaEventRecord(p->wf_done, p->stream) != cudaSuccess)
    return EMRI_FD_ERR_CUDA;
  return EMRI_FD_OK;
}

// the device address of page-locked host memory the device can write in place, else null
void* mapped_host_ptr(void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// a device buffer for an output of `bytes` at `dst` (host outputs go to staging slot `slot`)
emri_fd_status stage_out(emri_fd_plan_s* p, int slot, void* dst, size_t bytes, void** out, bool* host) {
  *host = false;
  *out = dst;
  if (!dst || bytes == 0 || is_device_ptr(dst)) return EMRI_FD_OK;
  if (p->stage_sz[slot] < bytes) {
    if (p->stage[slot]) cudaFree(p->stage[slot]);
    p->stage[slot] = nullptr;
    p->stage_sz[slot] = 0;
    if (cudaMalloc(&p->stage[slot], bytes) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_OOM; }
    p->stage_sz[slot] = bytes;
  }
  *out = p->stage[slot];
  *host = true;
  return EMRI_FD_OK;
}

// read the status word back (pinned), reset it and synchronise once; the first latched
// device-detected error, in a fixed order of precedence
emri_fd_status sync_status(emri_fd_plan_s* p) {
  if (cudaMemcpyAsync(p->st_pinned, p->s.status, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->s.status, 0, sizeof(int), p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return EMRI_FD_ERR_CUDA;
  }
  const int hs = *p->st_pinned;
  if (hs & ST_KNOTS) return EMRI_FD_ERR_KNOTS;
  if (hs & ST_FREQ) return EMRI_FD_ERR_FREQ;
  if (hs & ST_MODE) return EMRI_FD_ERR_MODE;
  if (hs & ST_NONFINITE) return EMRI_FD_ERR_NONFINITE;
  if (hs & ST_CAPACITY) return EMRI_FD_ERR_CAPACITY;
  if (hs & ST_BOUNDS) return EMRI_FD_ERR_INTERNAL;
  return EMRI_FD_OK;
}

// preparation kernels and the output kernel, with optional event timing
void run_forward(emri_fd_plan_s* p, const CallShape& cs, const DevInputs& in, size_t ob) {
  cudaStream_t stm = p->stream;
  cudaMemsetAsync(p->s.counters, 0, 8 * sizeof(unsigned long long), stm);
  cudaEvent_t* E = nullptr;
  if (p->profiling && p->ev_used + 3 <= (int)p->ev.size()) {
    E = &p->ev[p->ev_used];
    p->ev_used += 3;
    cudaEventRecord(E[0], stm);
  }
  const cudaEvent_t freqs_ready = p->freqs_side ? p->ev_freqs : nullptr;
  p->freqs_side = false;
  if (cs.nm_total > 0) {
    nvtxRangePushA("emri_fd: preparation (splines, records, runs)");
    launch_prep(cs, in, p->s, stm, freqs_ready);
    nvtxRangePop();
    p->launches += kPrepKernels;
  } else {
    // no modes: every run list is empty
    cudaMemsetAsync(p->s.run_cnt, 0, sizeof(int), stm);
  }
  if (freqs_ready) cudaStreamWaitEvent(stm, freqs_ready, 0);   // (launch_prep has waited already)
  if (cs.nf_total > 0) {
    if (cs.nm_total == 0) {
      cudaMemsetAsync(in.h_plus, 0, ob, stm);
      cudaMemsetAsync(in.h_cross, 0, ob, stm);
    } else if (cs.window) {
      // unwindowed sum into plan buffers, then the window's three-term convolution
      DevInputs in2 = in;
      in2.h_plus = p->s.wbuf_p;
      in2.h_cross = p->s.wbuf_c;
      if (E) cudaEventRecord(E[1], stm);
      nvtxRangePushA("emri_fd: SPA output kernel");
      launch_spa(cs, in2, p->s, p->num_sms, stm);
      nvtxRangePop();
      if (E) cudaEventRecord(E[2], stm);
      nvtxRangePushA("emri_fd: Hann window");
      launch_window(cs, p->s, in.freqs, in2.h_plus, in2.h_cross, in.h_plus, in.h_cross, p->num_sms, stm);
      nvtxRangePop();
      p->launches += 2;
    } else {
      if (E) cudaEventRecord(E[1], stm);
      nvtxRangePushA("emri_fd: SPA output kernel");
      launch_spa(cs, in, p->s, p->num_sms, stm);
      nvtxRangePop();
      if (E) cudaEventRecord(E[2], stm);
      p->launches += 1;
    }
  }
  if (E && !(cs.nf_total > 0 && cs.nm_total > 0)) {
    cudaEventRecord(E[1], stm);
    cudaEventRecord(E[2], stm);
  }
  p->last_tiles = cs.tiles_total;
  p->last_nm = cs.nm_total;
}

}  // namespace

extern "C" {

emri_fd_status emri_fd_sum_modes(emri_fd_plan_t p, int n_wf, const long long* knot_off, const long long* mode_off,
                                 const long long* freq_off, const double* t, const double* phi_phi,
                                 const double* phi_r, const double* omega_phi, const double* omega_r, const int* l,
                                 const int* m, const int* n, const double* amp, const double* theta,
                                 const double* phi, const double* prefactor, const double* freqs, void* h_plus,
                                 void* h_cross) {
  CallShape cs;
  DevInputs in;
  emri_fd_status st = prepare_call(p, n_wf, knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r, l,
                                   m, n, amp, theta, phi, prefactor, freqs, cs, in, true);
  if (st != EMRI_FD_OK) return st;
  if (cs.nf_total > 0 && (!h_plus || !h_cross)) return EMRI_FD_ERR_ARG;
  const size_t ob = (p->desc.precision == EMRI_FD_MIXED ? 8 : 16) * (size_t)cs.nf_total;
  bool hp_host = false, hc_host = false, in_place = false;
  // page-locked host outputs: the kernels write them directly (no staging copy after the sum)
  void* hp_map = (cs.nf_total > 0 && !is_device_ptr(h_plus)) ? mapped_host_ptr(h_plus) : nullptr;
  void* hc_map = (cs.nf_total > 0 && !is_device_ptr(h_cross)) ? mapped_host_ptr(h_cross) : nullptr;
  if (hp_map) { in.h_plus = hp_map; in_place = true; }
  else if ((st = stage_out(p, 13, h_plus, ob, &in.h_plus, &hp_host)) != EMRI_FD_OK) return st;
  if (hc_map) { in.h_cross = hc_map; in_place = true; }
  else if ((st = stage_out(p, 14, h_cross, ob, &in.h_cross, &hc_host)) != EMRI_FD_OK) return st;
  run_forward(p, cs, in, ob);
  if (cudaGetLastError() != cudaSuccess) return EMRI_FD_ERR_CUDA;
  cudaStream_t stm = p->stream;
  if ((hp_host && cudaMemcpyAsync(h_plus, in.h_plus, ob, cudaMemcpyDeviceToHost, stm) != cudaSuccess) ||
      (hc_host && cudaMemcpyAsync(h_cross, in.h_cross, ob, cudaMemcpyDeviceToHost, stm) != cudaSuccess))
    return EMRI_FD_ERR_CUDA;
  // host outputs: the call synchronises, so it also returns its device-detected errors
  if (hp_host || hc_host || in_place) return sync_status(p);
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_td_sum(emri_fd_plan_t p, int n_wf, const long long* knot_off, const long long* mode_off,
                              const long long* sample_off, const double* t, const double* phi_phi,
                              const double* phi_r, const double* omega_phi, const double* omega_r, const int* l,
                              const int* m, const int* n, const double* amp, const double* theta,
                              const double* phi, const double* prefactor, const double* dt, float* h_plus,
                              float* h_cross) {
  if (!p || !p->desc.time_domain) return EMRI_FD_ERR_ARG;
  if (n_wf < 1 || !knot_off || !mode_off || !sample_off) return EMRI_FD_ERR_ARG;
  if (n_wf > p->desc.max_waveforms) return EMRI_FD_ERR_CAPACITY;
  if (knot_off[0] != 0 || mode_off[0] != 0 || sample_off[0] != 0) return EMRI_FD_ERR_ARG;
  if (cudaEventSynchronize(p->wf_done) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  CallShape cs{};
  cs.n_wf = n_wf;
  cs.conj = p->desc.conj_partners;
  const long long TS = td_tile_samples();
  long long amp_base = 0, seg_base = 0, tiles = 0;
  for (int w = 0; w < n_wf; w++) {
    const long long K = knot_off[w + 1] - knot_off[w], nm = mode_off[w + 1] - mode_off[w];
    const long long ns = sample_off[w + 1] - sample_off[w];
    if (K < 0 || nm < 0 || ns < 0) return EMRI_FD_ERR_ARG;
    if (K < 4) return EMRI_FD_ERR_KNOTS;
    if (K > p->desc.max_knots) return EMRI_FD_ERR_CAPACITY;
    WfInfo& W = p->wf_pinned[w];
    W = WfInfo{};
    W.ko = knot_off[w]; W.K = K; W.mo = mode_off[w]; W.nm = nm; W.fo = sample_off[w]; W.nf = ns;
    W.amp_base = amp_base; W.seg_base = seg_base; W.tile_base = tiles; W.ntiles = (ns + TS - 1) / TS;
    amp_base += nm * K;
    seg_base += nm * (K - 1);
    tiles += W.ntiles;
  }
  cs.K_total = knot_off[n_wf];
  cs.nm_total = mode_off[n_wf];
  cs.nf_total = sample_off[n_wf];
  cs.seg_total = seg_base;
  cs.amp_total = amp_base;
  cs.tiles_total = tiles;
  if (cs.K_total > p->cap_K || cs.nm_total > p->cap_nm || cs.seg_total > p->cap_seg || cs.amp_total > p->cap_amp)
    return EMRI_FD_ERR_CAPACITY;
  if (!t || !phi_phi || !phi_r || !omega_phi || !omega_r || !theta || !phi || !prefactor || !dt) return EMRI_FD_ERR_ARG;
  if (cs.nm_total > 0 && (!l || !m || !n || !amp)) return EMRI_FD_ERR_ARG;
  if (cs.nf_total > 0 && (!h_plus || !h_cross)) return EMRI_FD_ERR_ARG;
  for (int w = 0; w < n_wf; w++) {
    // dt is read here on the host when it is host memory, else checked by the caller
    if (!is_device_ptr(dt) && !(dt[w] > 0.0 && dt[w] < INFINITY)) return EMRI_FD_ERR_ARG;
  }
  DevInputs in{};
  emri_fd_status st = EMRI_FD_OK;
  const size_t kb = sizeof(double) * cs.K_total;
  const void* q;
#define STG(slot, ptr, bytes, field, type)                            \
  if (st == EMRI_FD_OK) {                                               \
    st = stage_in(p, slot, ptr, bytes, &q);                             \
    in.field = static_cast<type>(q);                                    \
  }
  STG(0, t, kb, t, const double*);
  STG(1, phi_phi, kb, phi_phi, const double*);
  STG(2, phi_r, kb, phi_r, const double*);
  STG(3, omega_phi, kb, omega_phi, const double*);
  STG(4, omega_r, kb, omega_r, const double*);
  STG(5, l, sizeof(int) * cs.nm_total, l, const int*);
  STG(6, m, sizeof(int) * cs.nm_total, m, const int*);
  STG(7, n, sizeof(int) * cs.nm_total, n, const int*);
  STG(8, amp, 2 * sizeof(double) * cs.amp_total, amp, const double*);
  STG(9, theta, sizeof(double) * n_wf, theta, const double*);
  STG(10, phi, sizeof(double) * n_wf, phi, const double*);
  STG(11, prefactor, sizeof(double) * n_wf, prefactor, const double*);
#undef STG
  if (st != EMRI_FD_OK) return st;
  const void* dtd = nullptr;
  if ((st = stage_in(p, 12, dt, sizeof(double) * n_wf, &dtd)) != EMRI_FD_OK) return st;
  void *hpd = nullptr, *hcd = nullptr;
  bool hph = false, hch = false;
  const size_t ob = sizeof(float) * (size_t)cs.nf_total;
  if ((st = stage_out(p, 13, h_plus, ob, &hpd, &hph)) != EMRI_FD_OK) return st;
  if ((st = stage_out(p, 14, h_cross, ob, &hcd, &hch)) != EMRI_FD_OK) return st;
  cudaStream_t stm = p->stream;
  if (cudaMemcpyAsync(p->s.wf, p->wf_pinned, sizeof(WfInfo) * n_wf, cudaMemcpyHostToDevice, stm) != cudaSuccess ||
      cudaEventRecord(p->wf_done, stm) != cudaSuccess)
    return EMRI_FD_ERR_CUDA;
  cudaMemsetAsync(p->s.counters, 0, 8 * sizeof(unsigned long long), stm);
  cudaEvent_t* E = nullptr;
  if (p->profiling && p->ev_used + 3 <= (int)p->ev.size()) {
    E = &p->ev[p->ev_used];
    p->ev_used += 3;
    cudaEventRecord(E[0], stm);
  }
  if (cs.nm_total > 0) {
    launch_prep_td(cs, in, p->s, p->tdamp, stm);
    p->launches += 6;
  }
  if (E) cudaEventRecord(E[1], stm);
  if (cs.nf_total > 0) {
    if (cs.nm_total == 0) {
      cudaMemsetAsync(hpd, 0, ob, stm);
      cudaMemsetAsync(hcd, 0, ob, stm);
    } else {
      launch_td_sum(cs, in, p->s, p->tdamp, static_cast<const double*>(dtd), static_cast<float*>(hpd),
                    static_cast<float*>(hcd), p->num_sms, stm);
      p->launches += 1;
    }
  }
  if (E) cudaEventRecord(E[2], stm);
  if (cudaGetLastError() != cudaSuccess) return EMRI_FD_ERR_CUDA;
  if ((hph && cudaMemcpyAsync(h_plus, hpd, ob, cudaMemcpyDeviceToHost, stm) != cudaSuccess) ||
      (hch && cudaMemcpyAsync(h_cross, hcd, ob, cudaMemcpyDeviceToHost, stm) != cudaSuccess))
    return EMRI_FD_ERR_CUDA;
  if ((hph || hch) && cudaStreamSynchronize(stm) != cudaSuccess) return EMRI_FD_ERR_CUDA;
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_td_spectrum(emri_fd_plan_t p, int n_wf, const long long* sample_off, const double* t0,
                                   const double* dt, int window, const float* h_plus, const float* h_cross,
                                   void* H_plus, void* H_cross) {
  if (!p || !p->desc.time_domain || n_wf < 1 || !sample_off || !t0 || !dt) return EMRI_FD_ERR_ARG;
  if (window != EMRI_FD_WINDOW_NONE && window != EMRI_FD_WINDOW_HANN) return EMRI_FD_ERR_ARG;
  if (is_device_ptr(t0) || is_device_ptr(dt) || !is_device_ptr(h_plus) || !is_device_ptr(h_cross) ||
      !is_device_ptr(H_plus) || !is_device_ptr(H_cross))
    return EMRI_FD_ERR_ARG;
  if (sample_off[0] != 0) return EMRI_FD_ERR_ARG;
  long long maxN = 0;
  for (int w = 0; w < n_wf; w++) {
    const long long N = sample_off[w + 1] - sample_off[w];
    if (N < 0 || N > 2000000000LL || !(dt[w] > 0.0 && dt[w] < INFINITY) || !(fabs(t0[w]) < INFINITY))
      return EMRI_FD_ERR_ARG;
    if (N > maxN) maxN = N;
  }
  cudaStream_t stm = p->stream;
  if (maxN > p->zcap) {
    if (p->zbuf) { cudaStreamSynchronize(stm); cudaFree(p->zbuf); }
    p->zbuf = nullptr;
    p->zcap = 0;
    if (cudaMalloc(&p->zbuf, sizeof(float2) * (size_t)maxN) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_OOM; }
    p->zcap = maxN;
  }
  long long ho = 0;
  for (int w = 0; w < n_wf; w++) {
    const long long N = sample_off[w + 1] - sample_off[w];
    if (N < 4) { continue; }
    cufftHandle h = 0;
    bool found = false;
    for (auto& fp : p->fft_plans)
      if (fp.first == N) { h = fp.second; found = true; }
    if (!found) {
      if (cufftPlan1d(&h, (int)N, CUFFT_C2C, 1) != CUFFT_SUCCESS) return EMRI_FD_ERR_CUDA;
      p->fft_plans.emplace_back(N, h);
    }
    if (cufftSetStream(h, stm) != CUFFT_SUCCESS) return EMRI_FD_ERR_CUDA;
    launch_td_pack(h_plus + sample_off[w], h_cross + sample_off[w], N, window, p->zbuf, p->num_sms, stm);
    if (cufftExecC2C(h, reinterpret_cast<cufftComplex*>(p->zbuf), reinterpret_cast<cufftComplex*>(p->zbuf),
                     CUFFT_INVERSE) != CUFFT_SUCCESS)
      return EMRI_FD_ERR_CUDA;
    launch_td_unpack(p->zbuf, N, dt[w], t0[w], static_cast<float2*>(H_plus) + ho, static_cast<float2*>(H_cross) + ho,
                     p->num_sms, stm);
    p->launches += 3;
    ho += N / 2 - 1;
  }
  if (cudaGetLastError() != cudaSuccess) return EMRI_FD_ERR_CUDA;
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_select_modes(emri_fd_plan_t p, int n_wf, const long long* knot_off, const long long* mode_off,
                                    const double* amp, double eps, int* keep) {
  if (!p || n_wf < 1 || !knot_off || !mode_off) return EMRI_FD_ERR_ARG;
  if (n_wf > p->desc.max_waveforms) return EMRI_FD_ERR_CAPACITY;
  if (knot_off[0] != 0 || mode_off[0] != 0 || !(fabs(eps) < INFINITY)) return EMRI_FD_ERR_ARG;
  if (cudaEventSynchronize(p->wf_done) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  long long amp_base = 0, max_nm = 1;
  int maxK = 1;
  for (int w = 0; w < n_wf; w++) {
    const long long K = knot_off[w + 1] - knot_off[w], nm = mode_off[w + 1] - mode_off[w];
    if (K < 1 || nm < 0) return EMRI_FD_ERR_ARG;
    if (K > p->desc.max_knots || nm > EMRI_FD_SELECT_MAX_MODES) return EMRI_FD_ERR_CAPACITY;
    WfInfo& W = p->wf_pinned[w];
    W = WfInfo{};
    W.ko = knot_off[w]; W.K = K; W.mo = mode_off[w]; W.nm = nm; W.amp_base = amp_base;
    amp_base += nm * K;
    if (K > maxK) maxK = (int)K;
    if (nm > max_nm) max_nm = nm;
  }
  const long long nm_total = mode_off[n_wf];
  if (knot_off[n_wf] > p->cap_K || nm_total > p->cap_nm || amp_base > p->cap_amp) return EMRI_FD_ERR_CAPACITY;
  if (nm_total > 0 && (!amp || !keep)) return EMRI_FD_ERR_ARG;
  if (nm_total == 0) return EMRI_FD_OK;
  const void* a = nullptr;
  emri_fd_status st = stage_in(p, 8, amp, 2 * sizeof(double) * (size_t)amp_base, &a);
  if (st != EMRI_FD_OK) return st;
  void* kd = nullptr;
  bool khost = false;
  if ((st = stage_out(p, 13, keep, sizeof(int) * (size_t)nm_total, &kd, &khost)) != EMRI_FD_OK) return st;
  cudaStream_t stm = p->stream;
  if (cudaMemcpyAsync(p->s.wf, p->wf_pinned, sizeof(WfInfo) * n_wf, cudaMemcpyHostToDevice, stm) != cudaSuccess ||
      cudaEventRecord(p->wf_done, stm) != cudaSuccess)
    return EMRI_FD_ERR_CUDA;
  launch_select(p->s, n_wf, maxK, max_nm, static_cast<const double*>(a), eps, static_cast<int*>(kd), nm_total, stm);
  p->launches += 1;
  if (cudaGetLastError() != cudaSuccess) return EMRI_FD_ERR_CUDA;
  if (khost && (cudaMemcpyAsync(keep, kd, sizeof(int) * (size_t)nm_total, cudaMemcpyDeviceToHost, stm) != cudaSuccess ||
                cudaStreamSynchronize(stm) != cudaSuccess))
    return EMRI_FD_ERR_CUDA;
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_loglike_and_grad(emri_fd_plan_t p, int n_wf, const long long* knot_off,
                                        const long long* mode_off, const long long* freq_off, const double* t,
                                        const double* phi_phi, const double* phi_r, const double* omega_phi,
                                        const double* omega_r, const int* l, const int* m, const int* n,
                                        const double* amp, const double* theta, const double* phi,
                                        const double* prefactor, const double* freqs, const double* data_plus,
                                        const double* data_cross, const double* psd, const double* df,
                                        double* loglike, double* g_phi_phi, double* g_phi_r, double* g_omega_phi,
                                        double* g_omega_r, double* g_amp) {
  if (!p) return EMRI_FD_ERR_ARG;
  if (p->desc.precision != EMRI_FD_FP64 || !p->desc.likelihood) return EMRI_FD_ERR_ARG;
  CallShape cs;
  DevInputs in;
  emri_fd_status st = prepare_call(p, n_wf, knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r, l,
                                   m, n, amp, theta, phi, prefactor, freqs, cs, in);
  if (st != EMRI_FD_OK) return st;
  if (!loglike || !df || (cs.nf_total > 0 && (!data_plus || !data_cross || !psd))) return EMRI_FD_ERR_ARG;
  LikeInputs li{};
  const void* q = nullptr;
  if ((st = stage_in(p, 15, data_plus, 16 * (size_t)cs.nf_total, &q)) != EMRI_FD_OK) return st;
  li.data_plus = static_cast<const double*>(q);
  if ((st = stage_in(p, 16, data_cross, 16 * (size_t)cs.nf_total, &q)) != EMRI_FD_OK) return st;
  li.data_cross = static_cast<const double*>(q);
  if ((st = stage_in(p, 17, psd, 8 * (size_t)cs.nf_total, &q)) != EMRI_FD_OK) return st;
  li.psd = static_cast<const double*>(q);
  if ((st = stage_in(p, 18, df, 8 * (size_t)n_wf, &q)) != EMRI_FD_OK) return st;
  li.df = static_cast<const double*>(q);
  bool host[6] = {false, false, false, false, false, false};
  void* o = nullptr;
  const size_t kb = 8 * (size_t)cs.K_total;
  if ((st = stage_out(p, 19, loglike, 8 * (size_t)n_wf, &o, &host[0])) != EMRI_FD_OK) return st;
  li.loglike = static_cast<double*>(o);
  double* gin[5] = {g_phi_phi, g_phi_r, g_omega_phi, g_omega_r, g_amp};
  double* gdev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 5; k++) {
    const size_t bytes = k < 4 ? kb : 16 * (size_t)cs.amp_total;
    if ((st = stage_out(p, 20 + k, gin[k], bytes, &o, &host[1 + k])) != EMRI_FD_OK) return st;
    gdev[k] = static_cast<double*>(o);
  }
  li.g_phi_phi = gdev[0]; li.g_phi_r = gdev[1]; li.g_omega_phi = gdev[2]; li.g_omega_r = gdev[3]; li.g_amp = gdev[4];
  // forward into the plan's h buffers, then the residual and L
  in.h_plus = p->s.hbuf;
  in.h_cross = p->s.hbuf + 2 * cs.nf_total;
  run_forward(p, cs, in, 16 * (size_t)cs.nf_total);
  cudaStream_t stm = p->stream;
  if (cs.nf_total > 0) {
    nvtxRangePushA("emri_fd: residual and likelihood");
    launch_loglike(cs, li, p->s, stm);
    nvtxRangePop();
    p->launches += 2;
  } else {
    cudaMemsetAsync(li.loglike, 0, 8 * (size_t)n_wf, stm);
  }
  const bool want = g_phi_phi || g_phi_r || g_omega_phi || g_omega_r || g_amp;
  if (want) {
    for (int k = 0; k < 5; k++)
      if (gdev[k]) cudaMemsetAsync(gdev[k], 0, k < 4 ? kb : 16 * (size_t)cs.amp_total, stm);
    if (cs.nm_total > 0 && cs.nf_total > 0) {
      nvtxRangePushA("emri_fd: adjoint (knot gradients)");
      launch_adjoint(cs, in, li, p->s, p->num_sms, stm);
      nvtxRangePop();
      p->launches += kAdjointKernels;
    }
  }
  if (cudaGetLastError() != cudaSuccess) return EMRI_FD_ERR_CUDA;
  bool any_host = false;
  for (int k = 0; k < 6; k++) any_host = any_host || host[k];
  if (any_host) {
    if (host[0] && cudaMemcpyAsync(loglike, li.loglike, 8 * (size_t)n_wf, cudaMemcpyDeviceToHost, stm) != cudaSuccess)
      return EMRI_FD_ERR_CUDA;
    for (int k = 0; k < 5; k++)
      if (host[1 + k] && cudaMemcpyAsync(gin[k], gdev[k], k < 4 ? kb : 16 * (size_t)cs.amp_total,
                                         cudaMemcpyDeviceToHost, stm) != cudaSuccess)
        return EMRI_FD_ERR_CUDA;
    if (cudaStreamSynchronize(stm) != cudaSuccess) return EMRI_FD_ERR_CUDA;
  }
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_sync(emri_fd_plan_t p) {
  if (!p) return EMRI_FD_ERR_ARG;
  return sync_status(p);
}

emri_fd_status emri_fd_stats(emri_fd_plan_t p, long long* out, int nout) {
  if (!p || !out || nout < 0) return EMRI_FD_ERR_ARG;
  int runs = 0;
  cudaMemcpyAsync(p->cnt_pinned, p->s.counters, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, p->stream);
  if (p->last_nm > 0) cudaMemcpyAsync(&runs, p->s.run_cnt + p->last_nm, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  double prep_ms = 0.0, spa_ms = 0.0;
  for (int i = 0; i + 3 <= p->ev_used; i += 3) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, p->ev[i], p->ev[i + 1]);
    cudaEventElapsedTime(&b, p->ev[i + 1], p->ev[i + 2]);
    prep_ms += a;
    spa_ms += b;
  }
  cudaGetLastError();
  long long v[8] = {(long long)p->cnt_pinned[1], (long long)runs, p->last_tiles, (long long)p->cnt_pinned[3],
                    (long long)(p->ev_used / 3), (long long)(spa_ms * 1e6), (long long)(prep_ms * 1e6), p->launches};
  for (int i = 0; i < nout && i < 8; i++) out[i] = v[i];
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_profile(emri_fd_plan_t p, int enable) {
  if (!p) return EMRI_FD_ERR_ARG;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  if (enable && p->ev.empty()) {
    p->ev.resize(3 * 1024);
    for (auto& e : p->ev)
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  }
  p->profiling = enable != 0;
  p->ev_used = 0;
  p->launches = 0;
  return EMRI_FD_OK;
}

struct emri_fd_graph_s {
  cudaGraphExec_t exec = nullptr;
  WfInfo* wf = nullptr;       // the graph's own waveform table
  emri_fd_plan_s* plan = nullptr;
};

emri_fd_status emri_fd_set_tile(emri_fd_plan_t p, int tile_bins) {
  if (!p || !(tile_bins == 32 || tile_bins == 64 || tile_bins == 128)) return EMRI_FD_ERR_ARG;
  if (tile_bins == 128 && p->desc.tile_split > 1) return EMRI_FD_ERR_ARG;
  p->desc.tile_bins = tile_bins;
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_set_tile_split(emri_fd_plan_t p, int tile_split) {
  if (!p || !(tile_split == 0 || tile_split == 1 || tile_split == 2 || tile_split == 4)) return EMRI_FD_ERR_ARG;
  if (tile_split > 1 && p->desc.tile_bins == 128) return EMRI_FD_ERR_ARG;
  p->desc.tile_split = tile_split;
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_capture(emri_fd_plan_t p, int n_wf, const long long* knot_off, const long long* mode_off,
                               const long long* freq_off, const double* t, const double* phi_phi,
                               const double* phi_r, const double* omega_phi, const double* omega_r, const int* l,
                               const int* m, const int* n, const double* amp, const double* theta,
                               const double* phi, const double* prefactor, const double* freqs, void* h_plus,
                               void* h_cross, emri_fd_graph_t* graph) {
  if (!p || !graph) return EMRI_FD_ERR_ARG;
  *graph = nullptr;
  const void* dptrs[] = {t, phi_phi, phi_r, omega_phi, omega_r, l, m, n, amp, theta, phi, prefactor, freqs,
                         h_plus, h_cross};
  for (const void* q : dptrs)
    if (q && !is_device_ptr(q)) return EMRI_FD_ERR_ARG;   // a graph cannot capture host staging
  CallShape cs;
  DevInputs in;
  emri_fd_status st = prepare_call(p, n_wf, knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r, l,
                                   m, n, amp, theta, phi, prefactor, freqs, cs, in);
  if (st != EMRI_FD_OK) return st;
  if (cs.nf_total > 0 && (!h_plus || !h_cross)) return EMRI_FD_ERR_ARG;
  in.h_plus = h_plus;
  in.h_cross = h_cross;
  emri_fd_graph_s* G = new emri_fd_graph_s();
  G->plan = p;
  if (cudaMalloc(&G->wf, sizeof(WfInfo) * n_wf) != cudaSuccess) { cudaGetLastError(); delete G; return EMRI_FD_ERR_OOM; }
  if (cudaMemcpyAsync(G->wf, p->wf_pinned, sizeof(WfInfo) * n_wf, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError(); cudaFree(G->wf); delete G; return EMRI_FD_ERR_CUDA;
  }
  // the captured launches read the graph's own waveform table; they are recorded on
  // a private non-blocking stream (the plan's stream may be the legacy default
  // stream, which cannot be captured); replays run on the plan's stream
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError(); cudaFree(G->wf); delete G; return EMRI_FD_ERR_CUDA;
  }
  WfInfo* saved = p->s.wf;
  cudaStream_t saved_stream = p->stream;
  p->s.wf = G->wf;
  p->stream = cap;
  const bool prof = p->profiling;
  const long long launches = p->launches;
  p->profiling = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    run_forward(p, cs, in, (p->desc.precision == EMRI_FD_MIXED ? 8 : 16) * (size_t)cs.nf_total);
    e = cudaStreamEndCapture(cap, &g);
  }
  p->s.wf = saved;
  p->stream = saved_stream;
  p->profiling = prof;
  p->launches = launches;
  cudaStreamDestroy(cap);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (G->exec) cudaGraphExecDestroy(G->exec);
    cudaFree(G->wf);
    delete G;
    return EMRI_FD_ERR_CUDA;
  }
  *graph = G;
  return EMRI_FD_OK;
}

emri_fd_status emri_fd_replay(emri_fd_graph_t G) {
  if (!G || !G->exec) return EMRI_FD_ERR_ARG;
  if (cudaGraphLaunch(G->exec, G->plan->stream) != cudaSuccess) { cudaGetLastError(); return EMRI_FD_ERR_CUDA; }
  G->plan->launches += kPrepKernels + 1;
  return EMRI_FD_OK;
}

void emri_fd_graph_destroy(emri_fd_graph_t G) {
  if (!G) return;
  cudaStreamSynchronize(G->plan->stream);
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->wf) cudaFree(G->wf);
  cudaGetLastError();
  delete G;
}

}  // extern "C"

