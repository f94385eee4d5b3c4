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
2 FP64 FMA/clk/SM x 2 flops x SMs x the median sampled SM clock.
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

WORKLOAD = ("paper-shaped FP64 single waveform: T=2 yr, K=200 knots, 2000 modes (l=2..10, m=1..l, "
            "|n|<=30, top mean power of 3294), 3,155,760 bins f=i/T, conjugate partners implied")
FP64_OPS_PER_MODE_BIN = 30      # 25 DFMA + 5 DMUL/DADD per mode-bin in k_spa<*, 0, 0> (counted from the source)
FP64_FLOPS_PER_MODE_BIN = 55    # 25 x 2 + 5
FP64_PER_CLK_PER_SM = 2          # GB300 FP64 issue rate (1.25 TFLOP/s nominal at 2.07 GHz, 152 SMs)
MIXED_FP64_OPS_PER_MODE_BIN = 9  # the mixed form's FP64 left per mode-bin: difference 1, root polish 4, phase 4
ADJ_FP64_OPS_PER_MODE_BIN = 75   # k_adjoint per mode-bin: the forward's 29 (with dA/du) + 46 for the derivatives


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
    ap.add_argument("--config", default="paper", choices=["paper", "batch", "mixed-batch", "likelihood", "td", "select"])
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--no-mixed", action="store_true")
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


def cpu_oracle_rate(w, budget_s=15.0, threads=None):
    """The CPU oracle on a strided sample of the waveform's bins.  Bins are
    independent, so the per-bin part extrapolates; the per-waveform set-up is
    timed on its own and counted once.  Returns waveforms/s, threads, sample text."""
    from oracle import oracle as O
    O.build()
    threads = threads or O.default_threads()
    setup = oracle_setup_s(w, threads)
    # calibration sample (large enough that the set-up's timing noise does not matter),
    # then a sample sized to the budget
    stride = 256 if threads > 1 else 512
    sel = w.freqs[::stride]
    t0 = time.perf_counter()
    O.sum_modes(w, freqs=sel, nthreads=threads)
    dt = time.perf_counter() - t0
    per_bin = max(dt - setup, 1e-3) / sel.shape[0]
    target = max(1.0, (budget_s - setup) / per_bin)
    stride = int(min(1024, max(1, math.ceil(w.n_freqs / target))))
    sel = w.freqs[::stride]
    t0 = time.perf_counter()
    O.sum_modes(w, freqs=sel, nthreads=threads)
    dt = time.perf_counter() - t0
    per_wave = setup + max(dt - setup, 0.0) * (w.n_freqs / sel.shape[0])
    return 1.0 / per_wave, threads, ("every %d-th bin (%d of %d bins) in %.1f s, per-waveform set-up %.2f s counted "
                                     "once, per-bin part extrapolated" % (stride, sel.shape[0], w.n_freqs, dt, setup))


def reference_arm(args, rank, world):
    """CPU oracle timed as the reference implementation (rank 0 only): each step
    evaluates every 16th bin of the workload; the per-waveform set-up is timed
    separately and counted once per extrapolated waveform."""
    if rank != 0:
        return
    from paper_2307_12585_gb300 import synth
    from oracle import oracle as O
    O.build()
    w = synth.paper_config(1)
    threads = O.default_threads()
    stride = 16
    sel = w.freqs[::stride]
    setup = oracle_setup_s(w, threads)
    for _ in range(args.warmup):
        O.sum_modes(w, freqs=sel, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.sum_modes(w, freqs=sel, nthreads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    per_wave = setup + max(dt - setup, 0.0) * w.n_freqs / sel.shape[0]
    val = 1.0 / per_wave
    line = {"impl": "reference", "metric": "waveforms/s", "value": val, "unit": "waveforms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "CPU FP64 oracle (oracle/oracle.c)"},
            "cpu_baseline": {"value": val, "unit": "waveforms/s", "cores": threads, "kind": "oracle",
                             "sample": "every %d-th bin per step (%d of %d bins); set-up %.2f s counted once, "
                                       "per-bin part extrapolated" % (stride, sel.shape[0], w.n_freqs, setup)},
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
FORM_TILE = {"fp64x": 64, "mixed": 64}
DTYPES = {"fp64": "f64", "fp64x": "f32x2+i64 (double-float, FP64-accurate)", "mixed": "f64+f32"}
# DRAM bytes (read + write) of one k_spa<4,0,0> launch (FP64, standard SPA, 128-bin tiles) on
# this workload, from one ncu capture of the kernel as it stands
TRAFFIC_FP64_SPA = 102.095104e6 + 72.666368e6


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
    sel = {"modes_pool": pool.n_modes, "knots": pool.K, "eps": 1e-5, "kept": kept, "gpu_ms": sel_ms}
    if not args.no_cpu:
        from oracle import oracle as O
        t0 = time.perf_counter()
        O.select_modes(pool.amp, 1e-5)
        sel["oracle_ms_1core"] = (time.perf_counter() - t0) * 1e3
    out["mode_selection"] = sel
    return out


def run_paper(args, rank, world, local):
    """Default: the paper-shaped single FP64 waveform (2 yr, 2000 modes, 3,155,760 bins)."""
    import torch
    import torch.distributed as dist
    from paper_2307_12585_gb300 import api, synth

    nw = args.waveforms
    seeds = rank_seeds(rank, nw)
    wfs = [synth.paper_config(s) for s in seeds]
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
    clk_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_tflops = FP64_PER_CLK_PER_SM * 2 * n_sms * clk_hz / 1e12
    achieved = FP64_FLOPS_PER_MODE_BIN * mb_per_launch / spa_s / 1e12
    issue = FP64_OPS_PER_MODE_BIN * mb_per_launch / spa_s / (FP64_PER_CLK_PER_SM * n_sms * clk_hz)

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
        oms = event_time(oplan.stream, lambda i: oplan.sum_modes(dev[i % nw], out=oout, check=False), args.steps)
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
            # its FP64 (root polish, phase) against the FP64 pipe's peak; the ALU pipe
            # (integer phase and keys) is about as busy
            ach = MIXED_FP64_OPS_PER_MODE_BIN * mb_per_launch / ospa_s
            pk = FP64_PER_CLK_PER_SM * n_sms * clk_hz
            roof = {"bound": "fp64+alu", "achieved": ach / 1e12, "peak": pk / 1e12, "unit": "T FP64 inst/s",
                    "frac": ach / pk, "note": "%d FP64 instructions per mode-bin (root polish, in-segment phase) "
                    "against 2 FP64 instructions/clk/SM at the median SM clock; the rest is FP32 and integer work"
                    % MIXED_FP64_OPS_PER_MODE_BIN}
        elif prec == "fp64x" and spa == "standard":
            # no FP64 per mode-bin: the FP64 form's flops of FP64-accurate arithmetic per
            # mode-bin, done in FP32 pairs, against the FP64 pipe's peak
            ach = FP64_FLOPS_PER_MODE_BIN * mb_per_launch / ospa_s
            roof = {"bound": "issue", "fp64_equivalent_achieved": ach / 1e12, "peak": peak_tflops,
                    "unit": "TFLOP/s", "frac_of_fp64_peak": ach / (peak_tflops * 1e12),
                    "note": "FP64-accurate work (the FP64 form's %d flops per mode-bin) in FP32 pairs and "
                    "integers, against the FP64 pipe's nominal peak; instruction issue is the limit"
                    % FP64_FLOPS_PER_MODE_BIN}
        else:
            roof = None
        return {"value": world * args.steps / (oms * 1e-3), "unit": "waveforms/s", "ms_per_step": oms / args.steps,
                "roofline": roof,
                "spa_kernel_ms": ost["spa_ns"] * 1e-6 / max(1, ost["timed_calls"]),
                "prep_ms": ost["prep_ns"] * 1e-6 / max(1, ost["timed_calls"]),
                "mode_bin_evals_per_s": world * mb / (oms * 1e-3),
                "speedup_vs_fp64": ms / oms, "rel_l2_vs_fp64": float(torch.sqrt(num / den)),
                "tile_bins": FORM_TILE.get(prec, args.tile_bins)}

    mixed = fp64x = ext = None
    headline = args.precision == "fp64" and args.spa == "standard" and args.window is None
    if headline and not args.no_mixed:
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
    if headline and not args.no_mixed and rank == 0:
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
        for i in range(2):
            plan.sum_modes_host(hb[i % 2], out=hout[i % 2])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        esteps = max(3, args.steps // 4)
        for i in range(esteps):
            plan.sum_modes_host(hb[i % 2], out=hout[i % 2])
        torch.cuda.synchronize()
        edt = time.perf_counter() - t0
        e2e = {"value": world * esteps / edt, "unit": "waveforms/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": esteps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sample = cpu_oracle_rate(wfs[0])
        cpu = {"value": v, "unit": "waveforms/s", "cores": cores, "kind": "oracle", "sample": sample}
        v1, _, sample1 = cpu_oracle_rate(wfs[0], budget_s=6.0, threads=1)
        cpu["one_core"] = {"value": v1, "cores": 1, "sample": sample1}

    hbm_peak = measured_peaks().get("hbm_gbs")
    if rank == 0:
        line = base_line(args, world, "waveforms/s", value, "waveforms/s", ms, WORKLOAD, {
            "mode_bin_evals_per_s": world * mb / sec,
            "mode_bins_per_waveform": mb_per_launch,
            "spa_kernel_ms": spa_s * 1e3, "prep_ms": st["prep_ns"] * 1e-6 / max(1, st["timed_calls"]),
            "roofline": ({"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                          "frac": achieved / peak_tflops,
                          "traffic": TRAFFIC_FP64_SPA if args.tile_bins == 128 else None,
                          "issue_frac": issue,
                          # the same launch against HBM: far from that roof (compute-bound)
                          "hbm": ({"achieved_GBs": TRAFFIC_FP64_SPA / spa_s / 1e9, "peak_GBs": hbm_peak,
                                   "frac": TRAFFIC_FP64_SPA / spa_s / 1e9 / hbm_peak}
                                  if args.tile_bins == 128 and hbm_peak and TRAFFIC_FP64_SPA else None),
                          "note": "FP64 pipe: %d FP64 flops (%d FP64 instructions) per mode-bin; peak = %d FP64 FMA/clk/SM x 2 x SMs x median SM clock; traffic = DRAM bytes per launch from one ncu capture" % (
                              FP64_FLOPS_PER_MODE_BIN, FP64_OPS_PER_MODE_BIN, FP64_PER_CLK_PER_SM)}
                         if headline else None),
            "fp64x_form": fp64x, "mixed_form": mixed, "extended_spa": ext, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": st["launches"], "clocks": clocks})
        line.update(aux)
        line["config"].update({"waveforms_resident": nw, "tile_bins": args.tile_bins,
                               "l2": "inputs larger than L2: %d resident waveforms rotated, ~200 MB touched per step" % nw})
        print(json.dumps(line), flush=True)
    plan.close()


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


def run_batched(args, rank, world, local, mixed):
    """Batched workloads in one graph-captured call: 256 waveforms (N_m ~ U{50..3000},
    T ~ U(0.5, 4) yr, N_f log-uniform in [1e4, 6e6], uniform or log grids) in FP64, or
    64 paper-shaped 2 yr waveforms in the mixed form."""
    import torch
    from paper_2307_12585_gb300 import api, autotune, synth

    if mixed:
        nb = args.batch or 64
        wfs = [synth.paper_config(1 + rank * nb + i) for i in range(nb)]
        prec = "mixed"
        workload = "%d paper-shaped 2 yr waveforms (2000 modes, 3,155,760 bins each), mixed precision" % nb
    else:
        nb = args.batch or 256
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
    tune = autotune.tune(plan, db, out)
    plan.sum_modes(db, out=out)
    mb = plan.stats()["mode_bins"]
    g = plan.capture(db, out)
    for _ in range(args.warmup):
        g.replay()
    plan.sync()
    plan.profile(True)        # resets the launch counter
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    clk.start()
    ms = event_time(plan.stream, lambda i: g.replay(), args.steps)
    clocks = clk.stop()
    plan.sync()
    ms = max_over_ranks(ms, world)
    sec = ms * 1e-3
    extra = {"mode_bin_evals_per_s": world * mb * args.steps / sec, "mode_bins_per_batch": mb,
             "waveforms_per_step": nb, "bins_per_batch": nf, "autotune": tune, "cuda_graph": True,
             "gpu_launches": plan.stats()["launches"], "clocks": clocks}
    # the whole replay (preparation included) against the FP64 pipe: the FP64 form's 34
    # FP64 instructions per mode-bin, the mixed form's 9; FP64X has none per mode-bin and
    # is reported as FP64-accurate flops against the FP64 peak
    clk_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
    pk = FP64_PER_CLK_PER_SM * torch.cuda.get_device_properties(local).multi_processor_count * clk_hz
    mbs = mb * args.steps / sec
    if prec == "fp64x":
        extra["roofline"] = {"bound": "issue", "fp64_equivalent_achieved": FP64_FLOPS_PER_MODE_BIN * mbs / 1e12,
                             "peak": 2 * pk / 1e12, "unit": "TFLOP/s", "frac_of_fp64_peak": FP64_FLOPS_PER_MODE_BIN * mbs / (2 * pk)}
    else:
        ops = MIXED_FP64_OPS_PER_MODE_BIN if prec == "mixed" else FP64_OPS_PER_MODE_BIN
        extra["roofline"] = {"bound": "fp64+alu" if prec == "mixed" else "alu", "achieved": ops * mbs / 1e12,
                             "peak": pk / 1e12, "unit": "T FP64 inst/s", "frac": ops * mbs / pk,
                             "note": "%d FP64 instructions per mode-bin, whole replay (preparation included)" % ops}
    if mixed:
        # speed-up over the FP64 single-waveform form on the same GPU and waveform shape
        p64 = api.Plan("fp64", max_waveforms=1, max_knots=200, max_modes_total=2000, max_bins_total=wfs[0].n_freqs)
        d0 = p64.upload(synth.concat([wfs[0]]))
        o64 = p64.sum_modes(d0)
        t64 = event_time(p64.stream, lambda i: p64.sum_modes(d0, out=o64, check=False), 10) / 10
        extra["fp64_single_ms"] = t64
        extra["speedup_vs_fp64_single"] = (t64 * 1e-3) / (sec / args.steps / nb)
        # accuracy of every waveform against the FP64 form (device), on all bins
        hm = (out[0].to(torch.complex128), out[1].to(torch.complex128))
        errs = []
        for i, w in enumerate(wfs[: args.check_waveforms]):
            lo, hi = int(b["freq_off"][i]), int(b["freq_off"][i + 1])
            di = p64.upload(synth.concat([w]))
            ref = p64.sum_modes(di)
            num = sum(torch.linalg.vector_norm(hm[c][lo:hi] - ref[c]) ** 2 for c in range(2))
            den = sum(torch.linalg.vector_norm(ref[c]) ** 2 for c in range(2))
            ov = sum(torch.real(torch.vdot(ref[c], hm[c][lo:hi])) / torch.sqrt(
                torch.linalg.vector_norm(ref[c]) ** 2 * torch.linalg.vector_norm(hm[c][lo:hi]) ** 2) for c in range(2)) / 2
            errs.append((float(torch.sqrt(num / den)), float(1 - ov)))
        extra["rel_l2_vs_fp64"] = {"max": max(e[0] for e in errs), "median": float(np.median([e[0] for e in errs])),
                                   "waveforms_checked": len(errs)}
        extra["mismatch_vs_fp64"] = {"max": max(e[1] for e in errs), "median": float(np.median([e[1] for e in errs]))}
        p64.close()
    if rank == 0:
        line = base_line(args, world, "waveforms/s", world * nb * args.steps / sec, "waveforms/s", ms, workload, extra)
        line["dtype"] = DTYPES[prec]
        line["config"]["precision"] = prec
        print(json.dumps(line), flush=True)
    g.close()
    plan.close()


def run_likelihood(args, rank, world, local):
    """Whittle log-likelihood + gradient of every knot value: T = 1 yr, 500 modes,
    150 knots, 1,577,880 bins at df = 1/T, PSD 1e-40((1e-3/f)^4 + 1 + (f/2e-2)^2),
    data = waveform at offset parameters + Gaussian noise, SNR 78."""
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
    for _ in range(args.warmup):
        plan.loglike_and_grad(b, dp, dc, S, dfs, grad=True, check=False)
    plan.sync()
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    clk.start()
    ms = event_time(plan.stream, lambda i: plan.loglike_and_grad(b, dp, dc, S, dfs, grad=True, check=False),
                    args.steps)
    clocks = clk.stop()
    plan.sync()
    lms = event_time(plan.stream, lambda i: plan.loglike_and_grad(b, dp, dc, S, dfs, grad=False, check=False),
                     args.steps)
    plan.sync()
    ms = max_over_ranks(ms, world)
    mb = plan.stats()["mode_bins"]
    # the gradient path (adjoint kernel, then the per-segment sums and the transposed spline
    # solves) is the difference of the two timings; its FP64 work is the adjoint's
    grad_s = max(ms - lms, 1e-6) * 1e-3 / args.steps
    clk_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
    pk = FP64_PER_CLK_PER_SM * torch.cuda.get_device_properties(local).multi_processor_count * clk_hz
    ach = ADJ_FP64_OPS_PER_MODE_BIN * mb / grad_s
    roof = {"bound": "fp64", "kernel": "k_adjoint (timed with the rest of the gradient path)", "achieved": ach / 1e12,
            "peak": pk / 1e12, "unit": "T FP64 inst/s", "frac": ach / pk, "mode_bins": mb,
            "note": "%d FP64 instructions per mode-bin against 2 FP64 instructions/clk/SM at the median SM clock"
            % ADJ_FP64_OPS_PER_MODE_BIN}
    if rank == 0:
        line = base_line(args, world, "likelihood+gradient evaluations/s", world * args.steps / (ms * 1e-3),
                         "evaluations/s", ms,
                         "Whittle likelihood + knot gradient: T=1 yr, 500 modes, K=150, 1,577,880 bins, SNR 78",
                         {"loglike_only_per_s": world * args.steps / (lms * 1e-3), "gradient_path_ms": grad_s * 1e3,
                          "roofline": roof, "n_gradients": 4 * w.K + 2 * w.n_modes * w.K, "clocks": clocks})
        print(json.dumps(line), flush=True)
    plan.close()


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
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
