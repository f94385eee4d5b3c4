"""Calls shared by the checked-build test: each result of a set of representative calls
(every form, a batch, split tiles, the likelihood and its gradient, the no-allocation
entry point), computed with whichever library this process loads.  Run as
`python -m tests.checked_cases OUT.npz` it writes them to OUT.npz."""
import sys

import numpy as np

from paper_2307_12585_gb300 import api, synth


def run_cases():
    import torch
    out = {}
    w = synth.small_config(0, n_bins=2 ** 15 - 7)
    cases = (("fp64", "standard", 0, 0), ("fp64x", "standard", 0, 0), ("mixed", "standard", 0, 0),
             ("fp64", "extended", 0, 0), ("fp64", "standard", 32, 2))
    for prec, spa, tb, split in cases:
        p = api.Plan(prec, max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes, max_bins_total=w.n_freqs,
                     spa=spa, tile_bins=tb, tile_split=split)
        hp, hc = p.sum_modes(p.upload(synth.concat([w])))
        out["%s_%s_%d_%d" % (prec, spa, tb, split)] = np.stack([hp.cpu().numpy(), hc.cpu().numpy()]).astype(np.complex128)
        p.close()
    wfs = [synth.small_config(1, n_bins=3001), synth.paper_config(3, n_modes=300, T_years=0.5, grid="sparse",
                                                                   n_sparse=4000)]
    b = synth.concat(wfs)
    p = api.Plan("fp64", max_waveforms=2, max_knots=200, max_knots_total=int(b["knot_off"][-1]),
                 max_modes_total=int(b["mode_off"][-1]), max_bins_total=int(b["freq_off"][-1]))
    hp, hc = p.sum_modes(p.upload(b))
    out["batch"] = np.stack([hp.cpu().numpy(), hc.cpu().numpy()])
    p.close()
    # likelihood and gradient (data: the waveform itself at another phase offset)
    wl = synth.small_config(2, n_bins=4096)
    p = api.Plan("fp64", max_waveforms=1, max_knots=wl.K, max_modes_total=wl.n_modes, max_bins_total=wl.n_freqs,
                 likelihood=True)
    bl = p.upload(synth.concat([wl]))
    hp, hc = p.sum_modes(bl)
    S = torch.as_tensor(synth.psd(wl.freqs)).cuda()
    df = torch.tensor([1.0 / (wl.t[-1] - wl.t[0])], dtype=torch.float64, device="cuda")
    L, g = p.loglike_and_grad(bl, hp * (1 + 0.01j), hc * (1 - 0.01j), S, df)
    out["loglike"] = L.cpu().numpy()
    for k, v in g.items():
        out["grad_" + k] = v.cpu().numpy()
    p.close()
    # the no-allocation entry point
    dev = torch.device("cuda")
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dt)).to(dev)
    arrs = [d(getattr(w, k), np.float64) for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r")]
    arrs += [d(getattr(w, k), np.int32) for k in ("l", "m", "n")]
    amp = d(np.ascontiguousarray(w.amp, np.complex128).view(np.float64), np.float64)
    f = d(w.freqs, np.float64)
    hp = torch.empty(w.n_freqs, dtype=torch.complex128, device=dev)
    hc = torch.empty(w.n_freqs, dtype=torch.complex128, device=dev)
    code = api.emri_fd_sum_modes_noalloc(1, w.K, w.n_modes, w.n_freqs, *[a.data_ptr() for a in arrs],
                                         amp.data_ptr(), w.theta, w.phi, w.prefactor, f.data_ptr(), hp.data_ptr(),
                                         hc.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert code == 0, api.emri_fd_strerror(code)
    out["noalloc"] = np.stack([hp.cpu().numpy(), hc.cpu().numpy()])
    return out


if __name__ == "__main__":
    res = run_cases()
    res["library"] = np.array(api.library_path())
    np.savez(sys.argv[1], **res)
