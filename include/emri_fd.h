/*
 * emri_fd.h -- C ABI of the GB300 (sm_103a) frequency-domain EMRI mode sum.
 *
 * Method: arXiv 2307.12585 ("Fast and Fourier"), Sec. 2.2.  The strain is a
 * sum of voices h = h+ - i hx = sum_V H_V(t) exp(-i Phi_V(t)) (Eq. 1-2), one
 * per (l, m, n) harmonic of a Schwarzschild eccentric inspiral, with
 * H_V = prefactor A_lmn(t) -2Y_lm(theta, phi) and Phi_V = m Phi_phi + n Phi_r.
 * Its Fourier transform (sign convention of Eq. 3) is evaluated on an
 * arbitrary ascending frequency grid by the stationary-phase approximation:
 * for every voice and frequency bin, t(f) is obtained by inverting the
 * voice's cubic-spline frequency track F_V(t) = (m Omega_phi + n Omega_r)/2pi
 * segment by segment (Eq. 6), on each monotone branch (voices whose dF/dt
 * vanishes are split at the turnover, Sec. 2.2), and each root contributes
 * H_V(t) exp(i[2 pi f t - Phi_V(t) - sgn(Fdot) pi/4]) / sqrt|Fdot|  (the
 * standard-SPA limit of Eq. 10).
 *
 * Conventions shared by every entry point
 *  - Units: seconds, rad, rad/s, Hz.  The caller converts the paper's
 *    dimensionless Omega/M (Sec. 2.1) to rad/s.
 *  - Every series is interpolated by an independent not-a-knot cubic spline
 *    in t over the waveform's knots (Sec. 2.1).
 *  - With conj_partners = 1, each mode (l, m, n) (m >= 0) also stands for the
 *    voice (l, -m, -n) with amplitude (-1)^l conj(A) (Schwarzschild reflection
 *    symmetry); callers list one mode of each pair.  With conj_partners = 0
 *    every listed mode is one voice, any m in [-l, l].
 *  - Output bins f > 0 receive h+(f) = [H(f) + conj H(-f)]/2 and
 *    hx(f) = i [H(f) - conj H(-f)]/2, H(g) the voice-sum transform at signed
 *    frequency g, so voices whose frequency is negative contribute through
 *    conj H(-f).
 *  - Batches: n_waveforms independent waveforms share one call.  Their
 *    arrays are concatenated; knot_off, mode_off and freq_off (int64,
 *    [n_waveforms + 1], HOST memory, starting at 0, non-decreasing) give each
 *    waveform's slice.
 *  - Data pointers may be device memory (the fast path; required while a
 *    stream is being captured into a CUDA graph) or host memory, in which
 *    case the call stages them through plan-owned device buffers and, for
 *    host outputs, synchronises the stream before returning (emri_fd_sum_modes
 *    then also returns the device-detected errors, reading and resetting the
 *    status word as emri_fd_sync does).  The h_plus and
 *    h_cross outputs of emri_fd_sum_modes are written in place, by the
 *    kernels, when they are page-locked host memory the device can address
 *    (cudaHostAlloc / cudaHostRegister; on GB300 over NVLink-C2C), so their
 *    transfer overlaps the computation; pageable host outputs are staged.
 *  - Ownership: the caller owns every array passed in; the plan owns its
 *    scratch (spline coefficients, branch lists, work counters), sized at plan
 *    creation from the descriptor's maxima and never reallocated by a call on
 *    device data.
 *  - Errors: calls return an emri_fd_status.  Host-side checks (null
 *    pointers, sizes above the plan's maxima, offsets) are reported before
 *    anything is launched.  Value checks (non-increasing knots or
 *    frequencies, non-finite values, bad mode numbers) run on the device:
 *    they latch a status word in the plan, the output kernel of the call
 *    then writes nothing (outputs are unspecified), and the status is
 *    returned by emri_fd_sync() (which also clears it).  Every kernel keeps
 *    its indices in bounds whatever the values.  No C++ exception crosses
 *    this interface.
 *  - Calls are asynchronous on the plan's stream; two calls on one plan must
 *    not overlap in time on different streams.
 */
#ifndef EMRI_FD_H
#define EMRI_FD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct emri_fd_plan_s* emri_fd_plan_t;

typedef enum {
  EMRI_FD_OK = 0,
  EMRI_FD_ERR_ARG = 1,        /* null pointer, negative size, bad descriptor or offsets */
  EMRI_FD_ERR_KNOTS = 2,      /* fewer than 4 knots, or knot times not strictly increasing */
  EMRI_FD_ERR_FREQ = 3,       /* frequencies not strictly increasing, or f <= 0 */
  EMRI_FD_ERR_MODE = 4,       /* l < 2, l > EMRI_FD_MAX_L, |m| > l, or m < 0 with conj_partners */
  EMRI_FD_ERR_NONFINITE = 5,  /* NaN or Inf in a knot, amplitude, angle or prefactor */
  EMRI_FD_ERR_CAPACITY = 6,   /* a size above the plan's maxima, or branch storage exhausted */
  EMRI_FD_ERR_CUDA = 7,       /* a CUDA runtime call failed */
  EMRI_FD_ERR_OOM = 8,        /* device allocation failed */
  EMRI_FD_ERR_TIMEOUT = 9,    /* reserved for a bounded device wait that runs out.  No kernel of
                                 this version waits on a flag, a peer or another CTA's progress
                                 (work is claimed with atomics, and thread-block cluster barriers
                                 are reached by every member the same number of times), so no
                                 call returns it. */
  EMRI_FD_ERR_INTERNAL = 10   /* a device-side index check failed: only libraries built with
                                 -DEMRI_FD_CHECKS=1 (see the package's build script) test the
                                 indices their kernels derive from the device-built run lists,
                                 latch this status and skip the access instead of reading or
                                 writing out of bounds */
} emri_fd_status;

enum { EMRI_FD_FP64 = 0, EMRI_FD_MIXED = 1, EMRI_FD_FP64X = 2 };

/* Per-root time integral of the SPA sum (Sec. 2.2).
 * EMRI_FD_SPA_STANDARD: the phase expanded to second order about each root
 *   (Eq. 4) and the Fresnel integral done exactly:
 *   exp(-i sgn(Fdot) pi/4) / sqrt|Fdot|; a root with Fdot == 0 contributes 0.
 * EMRI_FD_SPA_EXTENDED: the phase expanded to third order (Eq. 7-9) and the
 *   integral taken in closed form (Eq. 10):
 *   -(2/sqrt 3) (i Fdot/|Fddot|) e^z K_{1/3}(z),  z = -2 pi i Fdot^3/(3 Fddot^2),
 *   principal branch.  The leading minus sign is a reading of Eq. 10: with it
 *   the factor tends to the standard one as Fddot -> 0, and the two roots of
 *   a cubic phase add up to its exact (Airy) Fourier transform.  It is finite
 *   at turnovers (Fdot -> 0); a root with Fdot == 0 exactly (a double root)
 *   contributes the limit of the two-root sum,
 *   2 pi^{2/3} / (3^{2/3} Gamma(2/3)) |Fddot|^{-1/3} with no pi/4 phase.
 *   K_{1/3} is evaluated to about 3e-12 relative (FP64 and FP64X plans) or
 *   FP32 precision (mixed plans).  Not available with likelihood = 1. */
enum { EMRI_FD_SPA_STANDARD = 0, EMRI_FD_SPA_EXTENDED = 1 };

/* Window of the time-domain signal, applied in the frequency domain (Sec. 2.3:
 * the FD waveform is convolved with the transform of the window).
 * EMRI_FD_WINDOW_HANN: w(t) = sin^2(pi t df) on [0, 1/df], df the spacing of
 *   the waveform's grid, t the knots' time coordinate (the observation starts
 *   at t = 0).  Its transform on that grid has three terms:
 *   h_w(f_i) = h(f_i)/2 - h(f_{i-1})/4 - h(f_{i+1})/4, with h = 0 outside the
 *   grid (exact when the grid holds every frequency with content, plus one bin
 *   on each side, e.g. f_i = i df from i = 1).  Each waveform's grid must be
 *   uniform: a spacing further than 1e-6 relative from the mean spacing
 *   returns EMRI_FD_ERR_FREQ at the next call or emri_fd_sync.  The plan holds
 *   an extra output-sized buffer per channel. */
enum { EMRI_FD_WINDOW_NONE = 0, EMRI_FD_WINDOW_HANN = 1 };

#define EMRI_FD_MAX_L 20

typedef struct {
  int precision;            /* EMRI_FD_FP64: FP64 throughout, complex128 outputs.
                               EMRI_FD_MIXED: FP64 root and phase, FP32 amplitude,
                               weight, sincos and compensated accumulation;
                               complex64 outputs.
                               EMRI_FD_FP64X: the FP64 form's accuracy from FP32-pair
                               ("double-float", ~48-bit) and integer arithmetic, no
                               FP64 instruction per evaluation; complex128 outputs. */
  int conj_partners;        /* 0 or 1, see above */
  int max_waveforms;        /* 1 .. 65535 */
  int max_knots;            /* per waveform, >= 4 */
  long long max_knots_total;/* sum of K over a call (0: max_waveforms * max_knots) */
  long long max_modes_total;/* sum of N_m over a call, >= 1 */
  long long max_bins_total; /* sum of N_f over a call, >= 1 */
  int tile_bins;            /* output bins per work tile: 32, 64 or 128; 0 = default (128) */
  int likelihood;           /* 1: also allocate the scratch of emri_fd_loglike_and_grad
                               (FP64 standard-form plans only); 0: that call returns
                               EMRI_FD_ERR_ARG */
  int spa_form;             /* EMRI_FD_SPA_STANDARD (0) or EMRI_FD_SPA_EXTENDED (1), below */
  int window;               /* EMRI_FD_WINDOW_NONE (0) or EMRI_FD_WINDOW_HANN (1), below;
                               not available with likelihood = 1 */
  int time_domain;          /* 1: also allocate the scratch of the time-domain comparator
                               (emri_fd_td_sum, emri_fd_td_spectrum); 0: those return
                               EMRI_FD_ERR_ARG */
  int tile_split;           /* CTAs sharing each output tile: 0 or 1 = one CTA per tile;
                               2 or 4 = the tile's branch list split over a thread-block
                               cluster of that many CTAs, whose partial sums are combined
                               in rank order through distributed shared memory.  For grids
                               with few tiles (sparse grids); tile_bins must be 32 or 64.
                               The summation grouping, hence the last bits, depend on it. */
  int reserved[2];          /* must be zero */
} emri_fd_desc;

/*
 * Create a plan.  out: receives the handle.  desc: sizes and precision.
 * stream: a cudaStream_t (NULL = legacy default stream) on the current device;
 * every call of the plan is ordered on it.  Allocates all scratch up front.
 * Errors: EMRI_FD_ERR_ARG (bad desc), EMRI_FD_ERR_OOM, EMRI_FD_ERR_CUDA.
 */
emri_fd_status emri_fd_plan(emri_fd_plan_t* out, const emri_fd_desc* desc, void* stream);

/*
 * The SPA sum (Sec. 2.2; Eq. 2, 3, 6, 10 in its standard-SPA limit) of
 * n_waveforms waveforms.
 *   knot_off, mode_off, freq_off: HOST int64 [n_waveforms + 1] slice offsets.
 *   t:                 [sum K] knot times (s), strictly increasing per waveform.
 *   phi_phi, phi_r:    [sum K] azimuthal and radial orbital phases (rad).
 *   omega_phi, omega_r:[sum K] azimuthal and radial frequencies (rad/s).
 *   l, m, n:           [sum N_m] int32 mode numbers.
 *   amp:               [sum over waveforms of N_m * K] complex128 amplitude
 *                      knots (re, im interleaved), mode-major then knot.
 *   theta, phi:        [n_waveforms] source-frame viewing angles (rad).
 *   prefactor:         [n_waveforms] real amplitude prefactor (mu / d_L).
 *   freqs:             [sum N_f] output frequencies (Hz), strictly increasing
 *                      and > 0 per waveform.
 *   h_plus, h_cross:   [sum N_f] outputs, complex128 (FP64 plan) or complex64
 *                      (mixed plan), every bin written.
 * Returns EMRI_FD_OK once the work is enqueued (device-side value errors are
 * reported by emri_fd_sync).
 */
emri_fd_status emri_fd_sum_modes(emri_fd_plan_t plan, int n_waveforms,
                                 const long long* knot_off, const long long* mode_off,
                                 const long long* freq_off,
                                 const double* t, const double* phi_phi, const double* phi_r,
                                 const double* omega_phi, const double* omega_r,
                                 const int* l, const int* m, const int* n, const double* amp,
                                 const double* theta, const double* phi, const double* prefactor,
                                 const double* freqs, void* h_plus, void* h_cross);

/*
 * Whittle log-likelihood (Eq. 14 with the inner product of Eq. 13) of
 * n_waveforms waveforms against data, and its gradient with respect to every
 * knot value.  Inputs as emri_fd_sum_modes, plus:
 *   data_plus, data_cross: [sum N_f] complex128 data d+ and dx on the same bins;
 *   psd:    [sum N_f] one-sided noise PSD S(f) > 0;
 *   df:     [n_waveforms] frequency spacing of each waveform's grid;
 * outputs:
 *   loglike: [n_waveforms] L_w = -1/2 sum_alpha <d - h|d - h>_alpha
 *            = -2 df sum_i |d_i - h_i|^2 / S_i  (both channels);
 *   g_phi_phi, g_phi_r, g_omega_phi, g_omega_r: [sum K] dL/d(knot values);
 *   g_amp:  [sum over waveforms of N_m K] complex128 (dL/dRe, dL/dIm) of the
 *           amplitude knots.
 * Any gradient pointer may be NULL (not computed; all NULL = likelihood only).
 * The gradient is that of L with each bin's branch and segment assignment held
 * at the input's (L is only piecewise smooth in the frequency knots: a bin
 * changes segment when a knot frequency crosses it).  Roots t(f) are
 * recomputed in the adjoint pass, with the same arithmetic as the forward pass.
 * Every sum has a fixed order, so a call is repeatable bit for bit.  loglike is
 * summed per waveform and equals the single-waveform call bitwise; the
 * gradient's bins are spread evenly over the GPU's lanes by their position in
 * the whole call, so a waveform's gradient in a batch differs from its
 * single-waveform value in the last bits.
 * Needs an FP64 plan created with likelihood = 1 (else EMRI_FD_ERR_ARG).
 * Pointers may be device or host memory (host: staged, and the call syncs).
 */
emri_fd_status emri_fd_loglike_and_grad(emri_fd_plan_t plan, int n_waveforms,
                                        const long long* knot_off, const long long* mode_off,
                                        const long long* freq_off,
                                        const double* t, const double* phi_phi, const double* phi_r,
                                        const double* omega_phi, const double* omega_r,
                                        const int* l, const int* m, const int* n, const double* amp,
                                        const double* theta, const double* phi, const double* prefactor,
                                        const double* freqs, const double* data_plus, const double* data_cross,
                                        const double* psd, const double* df, double* loglike,
                                        double* g_phi_phi, double* g_phi_r, double* g_omega_phi,
                                        double* g_omega_r, double* g_amp);

/*
 * Time-domain comparator (Sec. 2.3, 3.2): the TD waveform of Eq. 2 sampled at
 * t_j = t_0 + j dt (t_0 = the waveform's first knot), j = 0 .. N_w - 1:
 *   h(t) = prefactor sum_modes [A Y_lm e^{-i Phi} + (partners) (-1)^l conj(A) Y_{l,-m} e^{+i Phi}],
 *   Phi = m Phi_phi + n Phi_r, h = h+ - i hx; samples after the last knot are 0.
 * Inputs as emri_fd_sum_modes (the frequency series are splined but unused),
 * plus:
 *   sample_off: host int64 [n_waveforms + 1], N_w = sample_off[w+1] - sample_off[w];
 *   dt:       [n_waveforms] sampling intervals (> 0);
 * outputs h_plus, h_cross: [sum N_w] float (real TD samples).
 * Arithmetic: FP32 amplitudes and trigonometry, the phase in 32-bit fixed-point
 * turns from per-sample Q0.64 values of Phi_phi/2pi and Phi_r/2pi, sums over
 * modes in FP32 chunks of 32 carried in FP32 pairs (about 1e-6 relative).
 * Needs a plan with time_domain = 1.  Pointers may be device or host memory.
 */
emri_fd_status emri_fd_td_sum(emri_fd_plan_t plan, int n_waveforms, const long long* knot_off,
                              const long long* mode_off, const long long* sample_off, const double* t,
                              const double* phi_phi, const double* phi_r, const double* omega_phi,
                              const double* omega_r, const int* l, const int* m, const int* n,
                              const double* amp, const double* theta, const double* phi,
                              const double* prefactor, const double* dt, float* h_plus, float* h_cross);

/*
 * DFT of TD samples with the Fourier sign of Eq. 3 (cuFFT, one complex
 * transform of h+ + i hx per waveform):
 *   H(f_k) = dt sum_j h(t_j) e^{2 pi i f_k t_j},  f_k = k/(N_w dt),  k = 1 .. N_w/2 - 1,
 * for both channels.  window = EMRI_FD_WINDOW_HANN multiplies sample j by
 * sin^2(pi j/N_w) first.
 *   sample_off: host int64 [n_waveforms + 1]; t0, dt: HOST double [n_waveforms]
 *     (t0: time of sample 0);
 *   h_plus, h_cross: DEVICE float [sum N_w] (e.g. from emri_fd_td_sum);
 *   H_plus, H_cross: DEVICE complex64 [sum (N_w/2 - 1)] (waveforms with
 *     N_w < 4 contribute no bins).
 * The FFT plan for each length and an N_w-sized complex buffer are made on
 * first use and kept by the plan (these calls allocate device memory).
 */
emri_fd_status emri_fd_td_spectrum(emri_fd_plan_t plan, int n_waveforms, const long long* sample_off,
                                   const double* t0, const double* dt, int window, const float* h_plus,
                                   const float* h_cross, void* H_plus, void* H_cross);

/*
 * Power-based mode selection (Sec. 2.1).  For each waveform and each knot t_k,
 * the powers |A_j(t_k)|^2 of its modes are ordered by decreasing power (equal
 * powers: increasing mode index) and summed in that order, one FP64 addition
 * at a time; the mode at position i is kept when the sum before it is below
 * (1 - eps) times the total.  The selection is the union over the knots.
 *   knot_off, mode_off: host int64 [n_waveforms + 1], as emri_fd_sum_modes
 *     (only the knot counts are used from knot_off; K >= 1 here);
 *   amp:  [sum N_m K] complex128 knot amplitudes, mode-major, knot-minor;
 *   eps:  finite (eps <= 0 keeps every mode, eps >= 1 keeps none);
 *   keep: [sum N_m] int, written 1 (selected) or 0.
 * Per waveform N_m <= EMRI_FD_SELECT_MAX_MODES (the per-knot sort runs in one
 * CTA's shared memory), else EMRI_FD_ERR_CAPACITY; sizes are also bounded by
 * the plan's maxima.  Non-finite powers latch EMRI_FD_ERR_NONFINITE.  The
 * result is bit-exact: every power, sum and comparison is one IEEE FP64
 * operation in the stated order.  Pointers may be device or host memory.
 */
#define EMRI_FD_SELECT_MAX_MODES 8192
emri_fd_status emri_fd_select_modes(emri_fd_plan_t plan, int n_waveforms, const long long* knot_off,
                                    const long long* mode_off, const double* amp, double eps, int* keep);

/*
 * Wait for the plan's stream and return (and clear) the status latched by the
 * device-side checks of the calls since the last sync.
 */
emri_fd_status emri_fd_sync(emri_fd_plan_t plan);

/*
 * Counters (synchronises the stream).  out[0..n), n <= 8:
 *   0: mode-bin evaluations of the last call (one per (mode, root, bin); a
 *      conjugate-partner pair counts once), 1: monotone branches ("runs")
 *      of the last call, 2: work tiles of the last call, 3: reserved (0),
 *   4: calls timed since emri_fd_profile(plan, 1) (at most 1024),
 *   5: total duration of their output (SPA) kernels in ns, 6: total duration
 *      of their preparation kernels in ns (both from CUDA events recorded on
 *      the plan's stream), 7: kernels launched since that emri_fd_profile.
 */
emri_fd_status emri_fd_stats(emri_fd_plan_t plan, long long* out, int n);

/*
 * Start (enable = 1) or stop (0) event timing of the following calls and
 * reset the timing counters of emri_fd_stats.  Synchronises the stream.
 * Timing adds three event records per call on the plan's stream.
 */
emri_fd_status emri_fd_profile(emri_fd_plan_t plan, int enable);

/*
 * No-allocation variant of emri_fd_sum_modes for one waveform (FP64 form,
 * complex128 outputs).  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- code running while another
 * component (e.g. a framework's caching allocator) holds the device's memory,
 * latency-critical code that cannot afford cudaMalloc/cudaFree (which may
 * synchronise the device), and plug-ins or callbacks that must not call the
 * allocator.  It calls no cudaMalloc, cudaFree or other allocating routine:
 * all scratch lives in one file-scope __device__ array of 7,555,328 bytes
 * (7.2 MiB), which every GPU that loads the library holds until the process
 * exits.
 *   Limits: n_knots in [4, EMRI_FD_NOALLOC_MAX_KNOTS], n_modes in
 *   [1, EMRI_FD_NOALLOC_MAX_MODES], n_freqs in [1, EMRI_FD_NOALLOC_MAX_BINS];
 *   larger sizes return EMRI_FD_ERR_CAPACITY before anything is launched.
 *   Arguments: as emri_fd_sum_modes for a single waveform (K = n_knots,
 *   N_m = n_modes, N_f = n_freqs), with the viewing angles and prefactor
 *   passed by value.  Every array must be DEVICE memory (host pointers give
 *   EMRI_FD_ERR_ARG).  stream: a cudaStream_t on the current device.
 *   Set-up: the first call on a device (with that device current) looks up the
 *   array's device address and fills a sin/cos table in it, synchronising the
 *   stream.  The set-up is kept per device ordinal for
 *   the life of the process: it does not survive cudaDeviceReset (or any other
 *   teardown of the device's primary context), after which this entry point
 *   must not be called again in that process.
 *   The call waits for its stream and returns the status of the device-side
 *   checks.  Every call uses the same array and overwrites the previous
 *   call's contents; calls whose GPU work overlaps in time (e.g. from two host
 *   threads on two streams) race on it and must be serialised by the caller.
 */
#define EMRI_FD_NOALLOC_MAX_KNOTS 200
#define EMRI_FD_NOALLOC_MAX_MODES 128
#define EMRI_FD_NOALLOC_MAX_BINS (1LL << 30)
emri_fd_status emri_fd_sum_modes_noalloc(int conj_partners, long long n_knots, long long n_modes,
                                         long long n_freqs, const double* t, const double* phi_phi,
                                         const double* phi_r, const double* omega_phi, const double* omega_r,
                                         const int* l, const int* m, const int* n, const double* amp,
                                         double theta, double phi, double prefactor, const double* freqs,
                                         void* h_plus, void* h_cross, void* stream);

/*
 * Change the output-tile width of a plan (32, 64 or 128 bins) for later calls.
 * Results may change in the last bits (the in-tile summation grouping changes).
 * EMRI_FD_ERR_ARG for 128 while the plan's tile split is above 1.
 */
emri_fd_status emri_fd_set_tile(emri_fd_plan_t plan, int tile_bins);

/*
 * Change the tile split (see emri_fd_desc.tile_split: 0, 1, 2 or 4) for later calls.
 * EMRI_FD_ERR_ARG for other values, or for a split above 1 with 128-bin tiles.
 */
emri_fd_status emri_fd_set_tile_split(emri_fd_plan_t plan, int tile_split);

/*
 * CUDA-graph capture of one emri_fd_sum_modes call (batches included): the
 * whole launch sequence (checks, preparation and output kernels) is recorded
 * once on the plan's stream and replayed with emri_fd_replay.  All data
 * pointers must be device memory; the graph reads them at every replay (the
 * caller may change their contents, not their sizes or addresses).  The graph
 * owns a copy of the batch's slice table; the plan's scratch is shared, so
 * replays and other calls of the plan must stay ordered on its stream.
 * Errors: as emri_fd_sum_modes, EMRI_FD_ERR_ARG for host pointers.
 */
typedef struct emri_fd_graph_s* emri_fd_graph_t;
emri_fd_status emri_fd_capture(emri_fd_plan_t plan, int n_waveforms,
                               const long long* knot_off, const long long* mode_off, const long long* freq_off,
                               const double* t, const double* phi_phi, const double* phi_r,
                               const double* omega_phi, const double* omega_r,
                               const int* l, const int* m, const int* n, const double* amp,
                               const double* theta, const double* phi, const double* prefactor,
                               const double* freqs, void* h_plus, void* h_cross, emri_fd_graph_t* graph);
/* Launch a captured call on its plan's stream (asynchronous). */
emri_fd_status emri_fd_replay(emri_fd_graph_t graph);
/* Release a captured call (synchronises its plan's stream first). */
void emri_fd_graph_destroy(emri_fd_graph_t graph);

/* Release the plan and its device memory (synchronises its stream first). */
void emri_fd_plan_destroy(emri_fd_plan_t plan);

/* Static, human-readable name of a status code. */
const char* emri_fd_strerror(emri_fd_status status);

/*
 * Peak-rate probe of the fused multiply-add pipes (a measurement utility; the
 * paper has no counterpart).  It gives the denominator against which the SPA
 * kernels' FP64 and FP32 roofline fractions are quoted.  Launches one kernel
 * on `stream` (a cudaStream_t on the current device; NULL = legacy default
 * stream) in which every thread of blocks_per_sm x SMs blocks of 256 threads
 * runs 8 independent FMA chains of iters x 16 steps each; the caller times the
 * launch (e.g. with CUDA events on that stream).
 *   precision: 0 = FP64 (DFMA), 1 = FP32 (FFMA);
 *   iters >= 1; blocks_per_sm in [1, 64];
 *   fma_per_launch: if not NULL, receives the FMAs one launch executes
 *     (blocks x 256 x iters x 128), each 2 flops.
 * Allocates nothing.  EMRI_FD_ERR_ARG for bad arguments, EMRI_FD_ERR_CUDA if
 * the launch fails.
 */
emri_fd_status emri_fd_fma_probe(int precision, int iters, int blocks_per_sm, void* stream,
                                 long long* fma_per_launch);

#ifdef __cplusplus
}
#endif
#endif /* EMRI_FD_H */
