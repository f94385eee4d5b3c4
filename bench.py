"""Benchmark of the frequency-domain SPA mode sum on GB300.

One step = one emri_fd_sum_modes call (the whole hot path: input checks,
not-a-knot spline solves, per-segment records, turnovers and monotone
branches, and the SPA output kernel) over one paper-shaped waveform: T = 2 yr,
200 knots, 2000 (l, m, n) modes (l <= 10, |n| <= 30), 3,155,760 bins at
df = 1/T (dt-equivalent 10 s), FP64, complex128 h+ and hx.  Eight such
waveforms (seeds 1-8) are resident in HBM and rotated, so every step's
working set (~200 MB) exceeds the 129 MB L2.

Metric: waveforms/s (whole job; with N ranks each rank sums its own
waveforms, weak scaling), plus mode-bin evaluations/s.
`--impl reference` times the CPU oracle instead (bounded samples of the
same workload, extrapolated).  Roofline: the headline kernel's algorithmic FP64
work (FP64_FLOPS_PER_MODE_BIN per mode-bin) over its event-timed duration, against
the FP64 FMA rate measured in the same run by the library's FMA probe (independent
DFMA chains on every SM, CUDA events), 2 flops per FMA; the nominal
2 FP64 FMA/clk/SM x SMs x the median sampled SM clock is reported beside it.

The default run also measures, each with its own CUDA-event timing, clocks and
roofline: the 256-waveform batch in one graph-replayed call (autotuned tiles),
the Whittle likelihood with its knot gradient (1 yr, 500 modes, 150 knots), and
the 64-waveform mixed-precision batch with its speed-up over the FP64 single
form.  The line ends with a compact "summary" of every result.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LIKE_WORKLOAD = "Whittle likelihood + knot gradient: T=1 yr, 500 modes, K=150, 1,577,880 bins, SNR 78"
WORKLOAD = ("paper-shaped FP64 single waveform: T=2 yr, K=200 knots, 2000 modes (l=2..10, m=1..l, "
            "|n|<=30, top mean power of 3294), 3,155,760 bins f=i/T, conjugate partners implied")
FP64_OPS_PER_MODE_BIN = 30      # 25 DFMA + 5 DMUL/DADD per mode-bin in k_spa<*, 0, 0> (counted from the source)
FP64_FLOPS_PER_MODE_BIN = 55    # 25 x 2 + 5
FP64_PER_CLK_PER_SM = 2          # GB300 FP64 issue rate (1.25 TFLOP/s nominal at 2.07 GHz, 152 SMs)
MIXED_FP64_OPS_PER_MODE_BIN = 6  # the mixed form's FP64 per mode-bin: g - A 1, in-segment phase 5 (the FP64
                                 # root polish runs only next to turnovers)
ADJ_FP64_OPS_PER_MODE_BIN = 75   # k_adjoint per mode-bin: the forward's 29 (with dA/du) + 46 for the derivatives
ORACLE_STRIDE = 16               # both CPU-oracle legs evaluate every 16th bin of the workload per step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp64x", "mixed"])
    ap.add_argument("--spa", default="standard", choices=["standard", "extended"])
    ap.add_argument("--window", default=None, choices=["hann"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--waveforms", type=int, default=8)
    ap.add_argument("--tile-bins", type=int, default=128)
    ap.add_argument("--config", default="paper",
                    choices=["paper", "batch", "mixed-batch", "likelihood", "td", "select", "probe"])
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batches", action="store_true")
    ap.add_argument("--check-waveforms", type=int, default=8)
    return ap.parse_args()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_setup_s(w, threads):
    """time of the oracle's per-waveform set-up (splines, voices, monotone pieces):
    one call on a single bin"""
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.sum_modes(w, freqs=w.freqs[len(w.freqs) // 2:len(w.freqs) // 2 + 1], nthreads=threads)
    return time.perf_counter() - t0


def oracle_sample_rate(w, threads, reps, warmup=0):
    """Waveforms/s of the CPU oracle on one waveform, from `reps` evaluations of every
    ORACLE_STRIDE-th bin (after `warmup` untimed ones).  Bins are independent, so the
    per-bin part extrapolates to the whole grid; the per-waveform set-up (splines,
    voices, monotone pieces: one single-bin call) is timed on its own and counted once.
    Returns (waveforms/s, seconds per sampled step, sample description)."""
    from oracle import oracle as O
    O.build()
    sel = w.freqs[::ORACLE_STRIDE]
    setup = oracle_setup_s(w, threads)
    for _ in range(warmup):
        O.sum_modes(w, freqs=sel, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(reps):
        O.sum_modes(w, freqs=sel, nthreads=threads)
    dt = (time.perf_counter() - t0) / reps
    per_wave = setup + max(dt - setup, 0.0) * (w.n_freqs / sel.shape[0])
    text = ("every %d-th bin (%d of %d bins) per step, %d step(s) of %.2f s; per-waveform set-up %.2f s counted "
            "once, per-bin part extrapolated" % (ORACLE_STRIDE, sel.shape[0], w.n_freqs, reps, dt, setup))
    return 1.0 / per_wave, dt, text


def cpu_oracle_baseline(w, pool=None):
    """The cpu_baseline leg: the oracle on all host cores (about 10 s of sampled steps)
    and on one core (one sampled step), with the reference arm's sampling; and, given
    the 3294-mode pool, the oracle's mode selection (eps = 1e-5) on one core."""
    from oracle import oracle as O
    O.build()
    threads = O.default_threads()
    v1, step, _ = oracle_sample_rate(w, threads, 1)
    reps = int(min(30, max(1, round(10.0 / max(step, 1e-3)))))
    v, _, sample = oracle_sample_rate(w, threads, reps)
    one, _, sample1 = oracle_sample_rate(w, 1, 1)
    out = {"value": v, "unit": "waveforms/s", "cores": threads, "kind": "oracle", "sample": sample,
           "one_core": {"value": one, "cores": 1, "sample": sample1}}
    if pool is not None:
        t0 = time.perf_counter()
        O.select_modes(pool.amp, 1e-5)
        out["mode_selection_1core_ms"] = (time.perf_counter() - t0) * 1e3
    return out


def reference_arm(args, rank, world):
    """CPU oracle timed as the reference implementation (rank 0 only): each step
    evaluates every ORACLE_STRIDE-th bin of the workload; the per-waveform set-up is
    timed separately and counted once per extrapolated waveform."""
    if rank != 0:
        return
    from paper_2307_12585_gb300 import synth
    from oracle import oracle as O
    O.build()
    w = synth.paper_config(1)
    threads = O.default_threads()
    val, dt, sample = oracle_sample_rate(w, threads, args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": "waveforms/s", "value": val, "unit": "waveforms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "CPU FP64 oracle (oracle/oracle.c)"},
            "cpu_baseline": {"value": val, "unit": "waveforms/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "waveforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def event_time(stream, fn, steps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        fn(i)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def max_over_ranks(ms, world):
    """The slowest rank's time (the whole job's time); one all-reduce of a scalar, on the
    process group's own device (CUDA for NCCL, the host for gloo)."""
    import torch
    import torch.distributed as dist
    if world > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms


def rank_seeds(rank, nw, base=1):
    """Seeds of the waveforms rank `rank` holds: independent problems, disjoint across
    ranks (weak scaling: every rank does the same amount of work)."""
    return [base + rank * nw + i for i in range(nw)]


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


# tile sizes of the other forms on this workload (the fastest of 32/64/128 bins when measured)
FORM_TILE = {"fp64x": 32, "mixed": 64}
DTYPES = {"fp64": "f64", "fp64x": "f32x2+i64 (double-float, FP64-accurate)", "mixed": "f64+f32"}
# DRAM bytes (read + write) of one k_spa<4,0,0> launch (FP64, standard SPA, 128-bin tiles) on
# this workload, from one ncu capture of the kernel as it stands
TRAFFIC_FP64_SPA = 102.028288e6 + 66.534400e6


def base_line(args, world, metric, value, unit, ms, workload, extra=None):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": workload, "precision": args.precision, "spa": args.spa, "window": args.window,
                       "parallelism": "independent waveforms per GPU (replicas)"}}
    if extra:
        line.update(extra)
    return line


def measured_peaks():
    """The machine's measured peaks (HBM copy GB/s, bf16 TFLOP/s), if the file is present."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def paper_aux(args, w, fd_ms_per_wf):
    """The other rows of the method on the same 2-yr, 2000-mode waveform: the time-domain
    comparator (TD sum at dt = 10 s + its FFT), the Hann window, and mode selection on the
    3294-mode pool it was drawn from."""
    import torch
    from paper_2307_12585_gb300 import api, synth
    reps = max(3, min(args.steps, 10))

    def timed(stream, fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    out = {}
    # time-domain comparator
    dt = 10.0
    N = int(np.floor((w.t[-1] - w.t[0]) / dt))
    plan = api.Plan("fp64", max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes, max_bins_total=16,
                    time_domain=True)
    b = plan.upload(synth.concat([w]))
    hp, hc, so = plan.td_sum(b, dt, N)
    plan.td_spectrum(hp, hc, so, w.t[0], dt)
    plan.profile(True)
    td_ms = timed(plan.stream, lambda: plan.td_sum(b, dt, N, check=False), reps)
    st = plan.stats()
    fft_ms = timed(plan.stream, lambda: plan.td_spectrum(hp, hc, so, w.t[0], dt), reps)
    kern_ms = st["spa_ns"] * 1e-6 / max(1, st["timed_calls"])
    out["td_comparator"] = {
        "samples": N, "dt_s": dt, "td_sum_ms": td_ms, "td_kernel_ms": kern_ms, "fft_ms": fft_ms,
        "total_ms": td_ms + fft_ms, "mode_sample_evals_per_s": N * w.n_modes / (kern_ms * 1e-3),
        "fd_fp64_speedup_vs_td": (td_ms + fft_ms) / fd_ms_per_wf,
        "arithmetic": "FP32 amplitudes/trig, 32-bit fixed-point phase, FP32 chunk sums carried in FP32 pairs; cuFFT C2C"}
    plan.close()
    # Hann window (three-term convolution after the SPA sum)
    res = {}
    for window in (None, "hann"):
        plan = api.Plan("fp64", max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes,
                        max_bins_total=w.n_freqs, tile_bins=args.tile_bins, window=window)
        b = plan.upload(synth.concat([w]))
        o = plan.sum_modes(b)
        res[window] = timed(plan.stream, lambda: plan.sum_modes(b, out=o, check=False), reps)
        plan.close()
    extra = max(res["hann"] - res[None], 1e-6)
    gbs = 72 * w.n_freqs / (extra * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs")
    out["hann_window"] = {"extra_ms": extra, "bytes_per_bin": 72, "achieved_GBs": gbs,
                          "peak_GBs": peak, "frac": (gbs / peak) if peak else None,
                          "note": "read h+/hx (32 B) and f (8 B), write h+/hx (32 B) per bin; bound by GB300's "
                                  "FP64 rate (12 FP64 operations per bin), not HBM; peak = measured copy bandwidth"}
    # the same waveform on a sparse grid of 1e4 log-spaced bins (the paper's downsampled FD, Sec. 3.3)
    ws = synth.paper_config(1, grid="sparse")
    best, unsplit = None, None
    # few bins: the tile size, and how many CTAs (a cluster) share a tile, set how many SMs take part
    for tb, split in ((32, 1), (64, 1), (128, 1), (32, 2), (32, 4), (64, 2), (64, 4)):
        plan = api.Plan("fp64", max_waveforms=1, max_knots=ws.K, max_modes_total=ws.n_modes,
                        max_bins_total=ws.n_freqs, tile_bins=tb, tile_split=split)
        b = plan.upload(synth.concat([ws]))
        o = plan.sum_modes(b)
        t = timed(plan.stream, lambda: plan.sum_modes(b, out=o, check=False), reps)
        plan.close()
        if best is None or t < best[0]:
            best = (t, tb, split)
        if split == 1 and (unsplit is None or t < unsplit):
            unsplit = t
    out["sparse_grid"] = {"bins": ws.n_freqs, "fp64_ms": best[0], "tile_bins": best[1], "tile_split": best[2],
                          "fp64_ms_unsplit": unsplit}
    # mode selection on the full pool
    pool = synth.paper_config(1, n_modes=3294, grid="sparse", n_sparse=16)
    plan = api.Plan("fp64", max_waveforms=1, max_knots=pool.K, max_modes_total=pool.n_modes, max_bins_total=16)
    b = plan.upload(synth.concat([pool]))
    kept = int(plan.select_modes(b, 1e-5).sum())
    sel_ms = timed(plan.stream, lambda: plan.select_modes(b, 1e-5, check=False), reps)
    plan.close()
    out["mode_selection"] = {"modes_pool": pool.n_modes, "knots": pool.K, "eps": 1e-5, "kept": kept, "gpu_ms": sel_ms}
    return out


def run_paper(args, rank, world, local):
    """Default: the paper-shaped single FP64 waveform (2 yr, 2000 modes, 3,155,760 bins),
    its other forms and rows, and the batched, likelihood and mixed-batch workloads."""
    import torch
    import torch.distributed as dist
    from paper_2307_12585_gb300 import api, synth

    nw = args.waveforms
    seeds = rank_seeds(rank, nw)
    wfs = synth.paper_configs(seeds)
    plan = api.Plan(args.precision, conj_partners=True, max_waveforms=1, max_knots=200,
                    max_modes_total=2000, max_bins_total=wfs[0].n_freqs, tile_bins=args.tile_bins, spa=args.spa,
                    window=args.window)
    dev = [plan.upload(synth.concat([w])) for w in wfs]
    nf = wfs[0].n_freqs
    outs = [(torch.empty(nf, dtype=plan.out_dtype, device="cuda"), torch.empty(nf, dtype=plan.out_dtype, device="cuda"))
            for _ in range(2)]
    mode_bins = []
    for b in dev:
        plan.sum_modes(b, out=outs[0])
        mode_bins.append(plan.stats()["mode_bins"])
    for i in range(args.warmup):
        plan.sum_modes(dev[i % nw], out=outs[i % 2], check=False)
    plan.sync()
    clk = ClockSampler(local)
    plan.profile(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    ms = event_time(plan.stream, lambda i: plan.sum_modes(dev[i % nw], out=outs[i % 2], check=False), args.steps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    plan.sync()
    st = plan.stats()
    ms = max_over_ranks(ms, world)
    mb = sum(mode_bins[i % nw] for i in range(args.steps))
    sec = ms * 1e-3
    value = job_rate(args.steps, world, ms)
    spa_s = st["spa_ns"] * 1e-9 / max(1, st["timed_calls"])
    mb_per_launch = mb / args.steps
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    headline = args.precision == "fp64" and args.spa == "standard" and args.window is None
    full = headline and not args.no_mixed
    # the FP64 (and FP32) FMA rates of this GPU, the roofline's denominators
    peaks = measure_fma_peaks(local)

    def other_form(prec, spa="standard"):
        # another form on the same waveforms and bins: its rate, its speed-up over this
        # FP64 run and its relative L2 difference from this run's FP64 output
        oplan = api.Plan(prec, conj_partners=True, max_waveforms=1, max_knots=200, max_modes_total=2000,
                         max_bins_total=nf, tile_bins=FORM_TILE.get(prec, args.tile_bins), spa=spa)
        oout = (torch.empty(nf, dtype=oplan.out_dtype, device="cuda"), torch.empty(nf, dtype=oplan.out_dtype, device="cuda"))
        for i in range(args.warmup):
            oplan.sum_modes(dev[i % nw], out=oout, check=False)
        oplan.sync()
        oplan.profile(True)
        oclk = ClockSampler(local)
        oclk.start()
        oms = event_time(oplan.stream, lambda i: oplan.sum_modes(dev[i % nw], out=oout, check=False), args.steps)
        oclocks = oclk.stop()
        oplan.sync()
        ost = oplan.stats()
        plan.sum_modes(dev[0], out=outs[0])
        oplan.sum_modes(dev[0], out=oout)
        num = (torch.linalg.vector_norm(oout[0].to(torch.complex128) - outs[0][0]) ** 2 +
               torch.linalg.vector_norm(oout[1].to(torch.complex128) - outs[0][1]) ** 2)
        den = torch.linalg.vector_norm(outs[0][0]) ** 2 + torch.linalg.vector_norm(outs[0][1]) ** 2
        oplan.close()
        ospa_s = ost["spa_ns"] * 1e-9 / max(1, ost["timed_calls"])
        if prec == "mixed" and spa == "standard":
            # its FP64 (g - A and the in-segment phase) against the FP64 pipe's measured rate;
            # the kernel is bound by instruction issue (integer phase and keys, FP32 work)
            roof = fp64_roof(MIXED_FP64_OPS_PER_MODE_BIN, mb_per_launch / ospa_s, peaks, oclocks, n_sms, None,
                             "output kernel alone; g - A and the in-segment phase in FP64, the rest FP32 and "
                             "integer work; instruction issue is the limit")
            roof["pipe"] = "issue (int + fp32); fp64 fraction shown"
        elif prec == "fp64x" and spa == "standard":
            # no FP64 per mode-bin: the FP64 form's flops of FP64-accurate arithmetic per
            # mode-bin, done in FP32 pairs, against the FP64 pipe's measured peak
            roof = fp64_roof(FP64_OPS_PER_MODE_BIN, mb_per_launch / ospa_s, peaks, oclocks, n_sms,
                             FP64_FLOPS_PER_MODE_BIN, "FP64-accurate work (the FP64 form's count) done in FP32 "
                             "pairs and integers; instruction issue is the limit")
            roof["pipe"] = "issue (fp32 + int)"
        else:
            roof = None
        return {"value": world * args.steps / (oms * 1e-3), "unit": "waveforms/s", "ms_per_step": oms / args.steps,
                "steps": args.steps, "roofline": roof, "clocks": oclocks,
                "spa_kernel_ms": ost["spa_ns"] * 1e-6 / max(1, ost["timed_calls"]),
                "prep_ms": ost["prep_ns"] * 1e-6 / max(1, ost["timed_calls"]),
                "mode_bin_evals_per_s": world * mb / (oms * 1e-3),
                "speedup_vs_fp64": ms / oms, "rel_l2_vs_fp64": float(torch.sqrt(num / den)),
                "tile_bins": FORM_TILE.get(prec, args.tile_bins)}

    mixed = fp64x = ext = None
    if full:
        fp64x = other_form("fp64x")
        fp64x["arithmetic"] = "FP32 pairs (double-float) and integers; FP64 only per tile and in preparation"
        mixed = other_form("mixed")
        # the extended SPA (Eq. 10): its cost over the standard form, per precision
        ext = {}
        for prec in ("fp64", "fp64x", "mixed"):
            e = other_form(prec, spa="extended")
            e["rel_l2_vs_standard_fp64"] = e.pop("rel_l2_vs_fp64")   # the size of the correction
            ext[prec] = e

    aux = {}
    if full and rank == 0:
        aux = paper_aux(args, wfs[0], ms / args.steps)

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI with pinned HOST buffers: H2D of the inputs and
        # D2H of h+ and hx happen inside every timed step
        hb = []
        for w in wfs[:2]:
            b = api.host_batch(synth.concat([w]))
            for k in list(b):
                if isinstance(b[k], np.ndarray) and k not in ("knot_off", "mode_off", "freq_off"):
                    b[k] = torch.from_numpy(b[k]).pin_memory()
            hb.append(b)
        cdt = plan.out_dtype
        hout = [(torch.empty(nf, dtype=cdt).pin_memory(), torch.empty(nf, dtype=cdt).pin_memory()) for _ in range(2)]
        h2d = sum(int(v.numel() * v.element_size()) for k, v in hb[0].items() if hasattr(v, "numel"))
        d2h = 2 * nf * (8 if args.precision == "mixed" else 16)
        for i in range(3):
            plan.sum_modes_host(hb[i % 2], out=hout[i % 2])
        torch.cuda.synchronize()
        esteps = max(20, args.steps)
        t0 = time.perf_counter()
        for i in range(esteps):
            plan.sum_modes_host(hb[i % 2], out=hout[i % 2])
        torch.cuda.synchronize()
        edt = time.perf_counter() - t0
        e2e = {"value": world * esteps / edt, "unit": "waveforms/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": esteps}
    plan.close()

    # the batched (256 waveforms, one graph), likelihood + gradient and mixed-batch
    # (64 waveforms) workloads, each timed on its own
    subs = {}
    if full and not args.no_batches:
        wl, v, bms, ex, _ = batched_measure(args, rank, world, local, False, 256, 3, 1, peaks, tune_reps=1)
        subs["batch256_fp64"] = dict(workload=wl, value=v, unit="waveforms/s", **ex)
        v, lms_, ex = likelihood_measure(args, rank, world, local, args.steps, args.warmup, peaks)
        subs["likelihood"] = dict(workload=LIKE_WORKLOAD, value=v, unit="evaluations/s", **ex)
        wl, v, bms, ex, _ = batched_measure(args, rank, world, local, True, 64, 10, 2, peaks, tune_reps=1,
                                            check_all=True)
        subs["batch64_mixed"] = dict(workload=wl, value=v, unit="waveforms/s", **ex)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_baseline(wfs[0], synth.paper_config(1, n_modes=3294, grid="sparse", n_sparse=16)
                                  if full else None)

    hbm_peak = measured_peaks().get("hbm_gbs")
    if rank == 0:
        roof = None
        if headline:
            roof = fp64_roof(FP64_OPS_PER_MODE_BIN, mb_per_launch / spa_s, peaks, clocks, n_sms,
                             FP64_FLOPS_PER_MODE_BIN, "output kernel k_spa<4,0,0,1> alone (event-timed per call); "
                             "traffic = DRAM bytes per launch from one ncu capture")
            roof["traffic"] = TRAFFIC_FP64_SPA if args.tile_bins == 128 else None
            # the same launch against HBM: far from that roof (compute-bound)
            roof["hbm"] = ({"achieved_GBs": TRAFFIC_FP64_SPA / spa_s / 1e9, "peak_GBs": hbm_peak,
                            "frac": TRAFFIC_FP64_SPA / spa_s / 1e9 / hbm_peak}
                           if args.tile_bins == 128 and hbm_peak and TRAFFIC_FP64_SPA else None)
        line = base_line(args, world, "waveforms/s", value, "waveforms/s", ms, WORKLOAD, {
            "mode_bin_evals_per_s": world * mb / sec,
            "mode_bins_per_waveform": mb_per_launch,
            "spa_kernel_ms": spa_s * 1e3, "prep_ms": st["prep_ns"] * 1e-6 / max(1, st["timed_calls"]),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": st["launches"], "clocks": clocks,
            "fma_peaks": peaks, "fp64x_form": fp64x, "mixed_form": mixed, "extended_spa": ext})
        line.update(aux)
        line.update(subs)
        line["config"].update({"waveforms_resident": nw, "tile_bins": args.tile_bins,
                               "l2": "inputs larger than L2: %d resident waveforms rotated, ~200 MB touched per step" % nw})
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)


def summary(line):
    """One short string per result, so that every number is readable at the end of the line."""
    def f(x, fmt="%.4g"):
        return "-" if x is None else fmt % x

    def roof(r):
        return "" if not r else " frac %s (nominal %s)" % (f(r.get("frac"), "%.3f"), f(r.get("frac_of_nominal"), "%.3f"))

    def clk(c):
        return "" if not c else " @%s MHz%s" % (f(c.get("sm_mhz"), "%.0f"), (" " + ",".join(c["reasons"])) if c.get("reasons") else "")

    out = {"fp64": "%s wf/s, kernel %s ms%s%s" % (f(line["value"]), f(line.get("spa_kernel_ms")),
                                                 roof(line.get("roofline")), clk(line.get("clocks")))}
    pk = line.get("fma_peaks")
    if pk:
        out["fma_peak"] = "fp64 %s TFLOP/s (%s of nominal), fp32 %s TFLOP/s" % (
            f(pk["fp64"]["tflops"]), f(pk["fp64"]["frac_of_nominal"], "%.3f"), f(pk["fp32"]["tflops"]))
    for k, name in (("fp64x_form", "fp64x"), ("mixed_form", "mixed")):
        o = line.get(k)
        if o:
            out[name] = "%s wf/s, kernel %s ms, x%s vs fp64%s" % (f(o["value"]), f(o["spa_kernel_ms"]),
                                                               f(o["speedup_vs_fp64"], "%.2f"), roof(o.get("roofline")))
    ext = line.get("extended_spa")
    if ext:
        out["extended"] = " / ".join("%s %s ms" % (p, f(ext[p]["spa_kernel_ms"])) for p in ext)
    b = line.get("batch256_fp64")
    if b:
        out["batch256_fp64"] = "%s wf/s, %s ms/step x%d, %s mode-bins/s%s%s" % (
            f(b["value"]), f(b["ms_per_step"]), b["steps"], f(b["mode_bin_evals_per_s"], "%.3g"),
            roof(b.get("roofline")), clk(b.get("clocks")))
    lk = line.get("likelihood")
    if lk:
        out["likelihood"] = "%s evals/s (loglike only %s/s), gradient path %s ms%s%s" % (
            f(lk["value"]), f(lk["loglike_only_per_s"]), f(lk["gradient_path_ms"]), roof(lk.get("roofline")),
            clk(lk.get("clocks")))
    mb = line.get("batch64_mixed")
    if mb:
        out["batch64_mixed"] = "%s wf/s, x%s vs fp64 single, rel L2 max %s, mismatch max %s (%d wf)%s%s" % (
            f(mb["value"]), f(mb["speedup_vs_fp64_single"], "%.2f"), f(mb["rel_l2_vs_fp64"]["max"], "%.2g"),
            f(mb["mismatch_vs_fp64"]["max"], "%.2g"), mb["rel_l2_vs_fp64"]["waveforms_checked"],
            roof(mb.get("roofline")), clk(mb.get("clocks")))
    e = line.get("e2e")
    if e:
        out["e2e"] = "%s wf/s over %d host-buffer calls" % (f(e["value"]), e["steps"])
    c = line.get("cpu_baseline")
    if c:
        out["cpu_oracle"] = "%s wf/s on %d cores, %s on 1" % (f(c["value"]), c["cores"], f(c["one_core"]["value"]))
    return out


def run_td(args, rank, world, local):
    """The time-domain comparator alone on the 2-yr, 2000-mode waveform: TD sum at
    dt = 10 s (6,311,520 samples) and its FFT, per waveform."""
    import torch
    from paper_2307_12585_gb300 import api, synth
    w = synth.paper_config(1 + rank)
    dt = 10.0
    N = int(np.floor((w.t[-1] - w.t[0]) / dt))
    plan = api.Plan("fp64", max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes, max_bins_total=16,
                    time_domain=True)
    b = plan.upload(synth.concat([w]))
    for _ in range(args.warmup):
        hp, hc, so = plan.td_sum(b, dt, N, check=False)
        plan.td_spectrum(hp, hc, so, w.t[0], dt, window=args.window)
    plan.sync()
    clk = ClockSampler(local)
    clk.start()
    ms = event_time(plan.stream, lambda i: plan.td_spectrum(*plan.td_sum(b, dt, N, check=False), w.t[0], dt,
                                                            window=args.window), args.steps)
    clocks = clk.stop()
    plan.sync()
    ms = max_over_ranks(ms, world)
    if rank == 0:
        line = base_line(args, world, "TD comparator waveforms/s", world * args.steps / (ms * 1e-3), "waveforms/s", ms,
                         "TD sum of the 2 yr, 2000-mode waveform at dt = 10 s (%d samples) + cuFFT spectrum" % N,
                         {"mode_sample_evals_per_s": world * N * w.n_modes * args.steps / (ms * 1e-3),
                          "dtype": "f32 + i32 phase", "clocks": clocks})
        print(json.dumps(line), flush=True)
    plan.close()


def run_select(args, rank, world, local):
    """Mode selection alone on the 3294-mode, 200-knot pool (eps = 1e-5)."""
    from paper_2307_12585_gb300 import api, synth
    pool = synth.paper_config(1 + rank, n_modes=3294, grid="sparse", n_sparse=16)
    plan = api.Plan("fp64", max_waveforms=1, max_knots=pool.K, max_modes_total=pool.n_modes, max_bins_total=16)
    b = plan.upload(synth.concat([pool]))
    for _ in range(args.warmup):
        plan.select_modes(b, 1e-5, check=False)
    plan.sync()
    ms = event_time(plan.stream, lambda i: plan.select_modes(b, 1e-5, check=False), args.steps)
    plan.sync()
    ms = max_over_ranks(ms, world)
    if rank == 0:
        line = base_line(args, world, "mode selections/s", world * args.steps / (ms * 1e-3), "selections/s", ms,
                         "power-based mode selection of 3294 modes over 200 knots, eps = 1e-5", {})
        print(json.dumps(line), flush=True)
    plan.close()


def measure_fma_peaks(local, target_ms=400.0):
    """FP64 and FP32 FMA rates of this GPU, measured by the library's probe
    (emri_fd_fma_probe: 8 independent FMA chains per thread, 8 CTAs of 256 threads
    per SM), timed with CUDA events on the current stream after a warm-up launch, with
    the SM clock sampled meanwhile.  No clock or other GPU setting is changed."""
    import torch
    from paper_2307_12585_gb300 import api
    stream = torch.cuda.current_stream()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    out = {}
    for name, prec, iters, per_clk in (("fp64", 0, 320, FP64_PER_CLK_PER_SM), ("fp32", 1, 16000, 128)):
        h = stream.cuda_stream
        n = api.emri_fd_fma_probe(prec, iters, 8, h)
        torch.cuda.synchronize()
        one = event_time(stream, lambda i: api.emri_fd_fma_probe(prec, iters, 8, h), 1)
        reps = int(min(200, max(5, target_ms / max(one, 1e-3))))
        clk = ClockSampler(local)
        clk.start()
        ms = event_time(stream, lambda i: api.emri_fd_fma_probe(prec, iters, 8, h), reps) / reps
        clocks = clk.stop()
        rate = n / (ms * 1e-3)
        nominal = per_clk * n_sms * (clocks.get("sm_mhz") or 2070.0) * 1e6
        out[name] = {"fma_per_s": rate, "tflops": 2 * rate / 1e12, "ms_per_launch": ms, "launches": reps,
                     "fma_per_launch": n, "nominal_tflops": 2 * nominal / 1e12, "frac_of_nominal": rate / nominal,
                     "clocks": clocks}
    return out


def fp64_roof(ops_per_mode_bin, mode_bins_per_s, peaks, clocks, n_sms, flops_per_mode_bin=None, note=""):
    """Roofline of FP64-pipe-bound work: FP64 instructions (and, if given, flops) per
    mode-bin times the mode-bin rate, against the FP64 FMA rate measured by the probe
    (instructions/s; x 2 for flops).  The nominal 2 FP64 FMA/clk/SM x SMs x the median
    SM clock of the timed region is reported beside it."""
    meas = peaks["fp64"]["fma_per_s"]
    nominal = FP64_PER_CLK_PER_SM * n_sms * ((clocks or {}).get("sm_mhz") or 2070.0) * 1e6
    inst = ops_per_mode_bin * mode_bins_per_s
    r = {"bound": "alu", "pipe": "fp64"}
    if flops_per_mode_bin:
        ach = flops_per_mode_bin * mode_bins_per_s
        r.update({"achieved": ach / 1e12, "peak": 2 * meas / 1e12, "unit": "TFLOP/s", "frac": ach / (2 * meas),
                  "peak_nominal": 2 * nominal / 1e12, "frac_of_nominal": ach / (2 * nominal)})
    else:
        r.update({"achieved": inst / 1e12, "peak": meas / 1e12, "unit": "T FP64 inst/s", "frac": inst / meas,
                  "peak_nominal": nominal / 1e12, "frac_of_nominal": inst / nominal})
    r["issue_frac"] = inst / meas
    r["peak_source"] = "measured: emri_fd_fma_probe in this run (DFMA chains, CUDA events)"
    r["note"] = ("%d FP64 instructions per mode-bin%s; " % (ops_per_mode_bin, "" if not flops_per_mode_bin else
                 " (%d flops)" % flops_per_mode_bin)) + note
    return r


def batched_measure(args, rank, world, local, mixed, nb, steps, warmup, peaks, tune_reps=3, check_all=False):
    """Batched workloads in one graph-captured call: nb waveforms (N_m ~ U{50..3000},
    T ~ U(0.5, 4) yr, N_f log-uniform in [1e4, 6e6], uniform or log grids) in FP64 or
    the precision of args, or nb paper-shaped 2 yr waveforms in the mixed form.
    Returns (workload, value, ms over `steps` replays, extra keys)."""
    import torch
    from paper_2307_12585_gb300 import api, autotune, synth

    if mixed:
        wfs = synth.paper_configs([1 + rank * nb + i for i in range(nb)])
        prec = "mixed"
        workload = "%d paper-shaped 2 yr waveforms (2000 modes, 3,155,760 bins each), mixed precision" % nb
    else:
        wfs = synth.batch_config(nb, seed0=100 + rank * nb)
        prec = args.precision
        workload = ("%d waveforms in one call: N_m ~ U{50..3000}, T ~ U(0.5,4) yr, N_f log-uniform [1e4, 6e6], "
                    "uniform or log grids, K=200" % nb)
    b = synth.concat(wfs)
    plan = api.Plan(prec, conj_partners=True, max_waveforms=nb, max_knots=200,
                    max_knots_total=int(b["knot_off"][-1]), max_modes_total=int(b["mode_off"][-1]),
                    max_bins_total=int(b["freq_off"][-1]))
    db = plan.upload(b)
    nf = int(b["freq_off"][-1])
    out = (torch.empty(nf, dtype=plan.out_dtype, device="cuda"), torch.empty(nf, dtype=plan.out_dtype, device="cuda"))
    tune = autotune.tune(plan, db, out, reps=tune_reps)
    plan.sum_modes(db, out=out)
    mb = plan.stats()["mode_bins"]
    g = plan.capture(db, out)
    for _ in range(warmup):
        g.replay()
    plan.sync()
    plan.profile(True)        # resets the launch counter
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    clk.start()
    ms = event_time(plan.stream, lambda i: g.replay(), steps)
    clocks = clk.stop()
    plan.sync()
    launches = plan.stats()["launches"]
    ms = max_over_ranks(ms, world)
    sec = ms * 1e-3
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    mbs = mb * steps / sec
    extra = {"steps": steps, "warmup": warmup, "ms_per_step": ms / steps, "mode_bin_evals_per_s": world * mbs,
             "mode_bins_per_batch": mb, "waveforms_per_step": nb, "bins_per_batch": nf,
             "output_bytes": 2 * nf * out[0].element_size(), "autotune": tune, "cuda_graph": True,
             "gpu_launches": launches, "clocks": clocks}
    # the whole replay (preparation included) against the FP64 pipe: the FP64 form's FP64
    # instructions per mode-bin, the mixed form's 9; FP64X has none per mode-bin and is
    # reported as FP64-accurate flops against the FP64 peak
    if prec == "fp64x":
        r = fp64_roof(FP64_OPS_PER_MODE_BIN, mbs, peaks, clocks, n_sms, FP64_FLOPS_PER_MODE_BIN,
                      "FP64-accurate work done in FP32 pairs and integers (issue-bound), whole replay")
        r["bound"], r["pipe"] = "alu", "issue (fp32 + int)"
        extra["roofline"] = r
    else:
        ops = MIXED_FP64_OPS_PER_MODE_BIN if prec == "mixed" else FP64_OPS_PER_MODE_BIN
        extra["roofline"] = fp64_roof(ops, mbs, peaks, clocks, n_sms, None,
                                      "whole replay (preparation included)" +
                                      ("; the rest is FP32 and integer work" if prec == "mixed" else ""))
    if mixed:
        # speed-up over the FP64 single-waveform form on the same GPU and waveform shape
        p64 = api.Plan("fp64", max_waveforms=1, max_knots=200, max_modes_total=2000, max_bins_total=wfs[0].n_freqs)
        d0 = p64.upload(synth.concat([wfs[0]]))
        o64 = p64.sum_modes(d0)
        for _ in range(3):
            p64.sum_modes(d0, out=o64, check=False)
        t64 = event_time(p64.stream, lambda i: p64.sum_modes(d0, out=o64, check=False), 20) / 20
        extra["fp64_single_ms"] = t64
        extra["speedup_vs_fp64_single"] = (t64 * 1e-3) / (sec / steps / nb)
        # accuracy of every checked waveform against the FP64 form (device), on all bins:
        # relative L2 over both channels and the mismatch averaged over the channels (Eq. 12)
        hm = (out[0].to(torch.complex128), out[1].to(torch.complex128))
        errs = []
        nchk = nb if check_all else min(nb, args.check_waveforms)
        for i, w in enumerate(wfs[:nchk]):
            lo, hi = int(b["freq_off"][i]), int(b["freq_off"][i + 1])
            di = p64.upload(synth.concat([w]))
            ref = p64.sum_modes(di, out=o64)
            num = sum(torch.linalg.vector_norm(hm[c][lo:hi] - ref[c]) ** 2 for c in range(2))
            den = sum(torch.linalg.vector_norm(ref[c]) ** 2 for c in range(2))
            ov = sum(torch.real(torch.vdot(ref[c], hm[c][lo:hi])) / torch.sqrt(
                torch.linalg.vector_norm(ref[c]) ** 2 * torch.linalg.vector_norm(hm[c][lo:hi]) ** 2) for c in range(2)) / 2
            errs.append((float(torch.sqrt(num / den)), float(1 - ov)))
        extra["rel_l2_vs_fp64"] = {"max": max(e[0] for e in errs), "median": float(np.median([e[0] for e in errs])),
                                   "waveforms_checked": len(errs)}
        extra["mismatch_vs_fp64"] = {"max": max(e[1] for e in errs), "median": float(np.median([e[1] for e in errs]))}
        p64.close()
    g.close()
    plan.close()
    del out, db
    torch.cuda.empty_cache()
    return workload, world * nb * steps / sec, ms, extra, prec


def run_probe(args, rank, world, local):
    """--config probe: the FP64 and FP32 FMA peak rates alone."""
    peaks = measure_fma_peaks(local)
    if rank == 0:
        line = base_line(args, world, "FP64 FMA rate", world * peaks["fp64"]["fma_per_s"], "FMA/s",
                         peaks["fp64"]["ms_per_launch"] * args.steps, "emri_fd_fma_probe: 8 CTAs of 256 threads per SM, "
                         "8 independent FMA chains per thread", {"fma_peaks": peaks})
        print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local, mixed):
    """--config batch | mixed-batch: one line for the batched workload."""
    peaks = measure_fma_peaks(local)
    nb = args.batch or (64 if mixed else 256)
    workload, value, ms, extra, prec = batched_measure(args, rank, world, local, mixed, nb, args.steps, args.warmup,
                                                       peaks)
    extra["fma_peaks"] = peaks
    if rank == 0:
        line = base_line(args, world, "waveforms/s", value, "waveforms/s", ms, workload, extra)
        line["dtype"] = DTYPES[prec]
        line["config"]["precision"] = prec
        print(json.dumps(line), flush=True)


def likelihood_measure(args, rank, world, local, steps, warmup, peaks):
    """Whittle log-likelihood + gradient of every knot value: T = 1 yr, 500 modes,
    150 knots, 1,577,880 bins at df = 1/T, PSD 1e-40((1e-3/f)^4 + 1 + (f/2e-2)^2),
    data = waveform at offset parameters + Gaussian noise, SNR 78.
    Returns (evaluations/s, ms over `steps` calls, extra keys)."""
    import torch
    from paper_2307_12585_gb300 import api, synth

    w = synth.likelihood_config(3 + rank)
    T = w.meta["T"]
    df = 1.0 / T
    plan = api.Plan("fp64", max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes, max_bins_total=w.n_freqs,
                    likelihood=True)
    b = plan.upload(synth.concat([w]))
    hp, hc = plan.sum_modes(b)
    S = torch.as_tensor(synth.psd(w.freqs)).cuda()
    rho = torch.sqrt(4 * df * torch.sum((hp.abs() ** 2 + hc.abs() ** 2) / S))
    scale = 78.0 / float(rho)
    b["prefactor"] = b["prefactor"] * scale
    rng = np.random.default_rng(7)
    dp = hp * scale * (1 + 0.01j) + torch.as_tensor(synth.noise(rng, w.freqs, df)).cuda()
    dc = hc * scale * (1 + 0.01j) + torch.as_tensor(synth.noise(rng, w.freqs, df)).cuda()
    dfs = torch.tensor([df], dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        plan.loglike_and_grad(b, dp, dc, S, dfs, grad=True, check=False)
    plan.sync()
    plan.profile(True)
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    clk.start()
    ms = event_time(plan.stream, lambda i: plan.loglike_and_grad(b, dp, dc, S, dfs, grad=True, check=False), steps)
    clocks = clk.stop()
    plan.sync()
    launches = plan.stats()["launches"]
    lms = event_time(plan.stream, lambda i: plan.loglike_and_grad(b, dp, dc, S, dfs, grad=False, check=False), steps)
    plan.sync()
    ms = max_over_ranks(ms, world)
    mb = plan.stats()["mode_bins"]
    # the gradient path (adjoint kernel, then the per-segment sums and the transposed spline
    # solves) is the difference of the two timings; its FP64 work is the adjoint's
    grad_s = max(ms - lms, 1e-6) * 1e-3 / steps
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = fp64_roof(ADJ_FP64_OPS_PER_MODE_BIN, mb / grad_s, peaks, clocks, n_sms, None,
                     "k_adjoint's work, timed with the rest of the gradient path (the difference of the "
                     "likelihood+gradient and likelihood-only timings)")
    roof["mode_bins"] = mb
    extra = {"steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
             "loglike_only_per_s": world * steps / (lms * 1e-3), "gradient_path_ms": grad_s * 1e3,
             "roofline": roof, "n_gradients": 4 * w.K + 2 * w.n_modes * w.K, "mode_bins": mb,
             "gpu_launches": launches, "clocks": clocks}
    plan.close()
    return world * steps / (ms * 1e-3), ms, extra


def run_likelihood(args, rank, world, local):
    """--config likelihood: one line for the likelihood + gradient workload."""
    peaks = measure_fma_peaks(local)
    value, ms, extra = likelihood_measure(args, rank, world, local, args.steps, args.warmup, peaks)
    extra["fma_peaks"] = peaks
    if rank == 0:
        line = base_line(args, world, "likelihood+gradient evaluations/s", value, "evaluations/s", ms,
                         LIKE_WORKLOAD, extra)
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_2307_12585_gb300 import build

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    if args.config == "paper":
        run_paper(args, rank, world, local)
    elif args.config == "batch":
        run_batched(args, rank, world, local, mixed=False)
    elif args.config == "mixed-batch":
        run_batched(args, rank, world, local, mixed=True)
    elif args.config == "likelihood":
        run_likelihood(args, rank, world, local)
    elif args.config == "td":
        run_td(args, rank, world, local)
    elif args.config == "select":
        run_select(args, rank, world, local)
    elif args.config == "probe":
        run_probe(args, rank, world, local)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
