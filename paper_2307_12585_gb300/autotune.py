"""Tile-shape autotuner for the SPA output kernel.

For a batch already resident on the device, times emri_fd_sum_modes with each
output-tile width (32, 64, 128 bins) -- and, for batches with few tiles, with
each tile shared by a cluster of 2 or 4 CTAs -- using CUDA events on the plan's
stream, keeps the fastest, and caches the choice in a JSON file keyed by the
device name, precision and a coarse signature of the batch (waveform count and
the powers of two of the total modes and bins).  Cache file:
$EMRI_FD_AUTOTUNE_CACHE, else ~/.cache/emri_fd/autotune.json.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

CANDIDATES = (32, 64, 128)
SPLITS = ((32, 2), (32, 4), (64, 2), (64, 4))   # (tile_bins, CTAs per tile) for batches with few tiles
FEW_TILES_PER_SM = 4                             # "few": fewer 128-bin tiles than this per SM


def cache_path() -> str:
    p = os.environ.get("EMRI_FD_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "emri_fd", "autotune.json")


def signature(plan, b) -> str:
    import torch
    n_wf = len(b["knot_off"]) - 1
    nm = int(b["mode_off"][-1])
    nf = int(b["freq_off"][-1])
    name = torch.cuda.get_device_name(plan.device)
    return "%s|p%d|w%d|m2^%d|f2^%d" % (name, plan.precision, n_wf, int(math.log2(max(nm, 1))),
                                       int(math.log2(max(nf, 1))))


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _apply(plan, tb, split):
    plan.set_tile_split(1)      # a split needs 32- or 64-bin tiles: clear it before changing the width
    plan.set_tile(tb)
    plan.set_tile_split(split)


def tune(plan, b, out, reps: int = 3, use_cache: bool = True, candidates=CANDIDATES) -> dict:
    """Set the plan's tile width (and tile split) to the fastest candidate for batch b;
    returns {"tile_bins": T, "tile_split": S, "ms": {"T" or "TxS": ms...}, "cached": bool}."""
    import torch
    path = cache_path()
    key = signature(plan, b)
    data = _load(path) if use_cache else {}
    if key in data:
        tb, split = int(data[key]["tile_bins"]), int(data[key].get("tile_split", 1))
        _apply(plan, tb, split)
        return {"tile_bins": tb, "tile_split": split, "ms": data[key].get("ms", {}), "cached": True}
    cands = [(tb, 1) for tb in candidates]
    nf = int(b["freq_off"][-1])
    n_sms = torch.cuda.get_device_properties(plan.device).multi_processor_count
    if nf / 128 < FEW_TILES_PER_SM * n_sms:
        cands += [c for c in SPLITS if c[0] in candidates]
    times = {}
    stream = plan.stream
    for tb, split in cands:
        _apply(plan, tb, split)
        plan.sum_modes(b, out=out, check=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.sum_modes(b, out=out, check=False)
        e1.record(stream)
        e1.synchronize()
        times[(tb, split)] = e0.elapsed_time(e1) / reps
    plan.sync()
    best = min(times, key=times.get)
    _apply(plan, *best)
    label = lambda c: str(c[0]) if c[1] == 1 else "%dx%d" % c
    ms = {label(c): v for c, v in times.items()}
    if use_cache:
        data[key] = {"tile_bins": int(best[0]), "tile_split": int(best[1]), "ms": ms}
        _save(path, data)
    return {"tile_bins": int(best[0]), "tile_split": int(best[1]), "ms": ms, "cached": False}
