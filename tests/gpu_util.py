"""Helpers of the GPU tests: run the CUDA path through the C ABI."""
import numpy as np

from paper_2307_12585_gb300 import api, synth


def plan_for(wfs, precision="fp64", conj=True, tile_bins=0, spa="standard", tile_split=0):
    return api.Plan(precision, conj_partners=conj, max_waveforms=len(wfs),
                    max_knots=max(w.K for w in wfs), max_knots_total=sum(w.K for w in wfs),
                    max_modes_total=max(1, sum(w.n_modes for w in wfs)),
                    max_bins_total=max(1, sum(w.n_freqs for w in wfs)), tile_bins=tile_bins, spa=spa,
                    tile_split=tile_split)


def run(wfs, precision="fp64", conj=True, tile_bins=0, stats=False, spa="standard", tile_split=0):
    if not isinstance(wfs, (list, tuple)):
        wfs = [wfs]
    plan = plan_for(wfs, precision, conj, tile_bins, spa, tile_split)
    hp, hc = plan.sum_modes(plan.upload(synth.concat(wfs)))
    out = (hp.cpu().numpy(), hc.cpu().numpy())
    st = plan.stats() if stats else None
    plan.close()
    return (out + (st,)) if stats else out


def rel_l2(x, ref):
    den = np.sqrt(np.sum(np.abs(ref) ** 2))
    return float(np.sqrt(np.sum(np.abs(np.asarray(x) - ref) ** 2)) / (den if den > 0 else 1.0))
