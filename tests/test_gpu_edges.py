"""Edge cases of the entry points added beside the SPA sum: empty mode lists,
zero-length outputs, one- and two-bin windowed grids, single-knot selection."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import api, synth
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_12585_gb300 import build
    build.build()


def _plan(w, **kw):
    return api.Plan("fp64", max_waveforms=2, max_knots=w.K, max_knots_total=2 * w.K,
                    max_modes_total=max(1, 2 * w.n_modes), max_bins_total=max(16, 2 * w.n_freqs), **kw)


def test_td_edges(oracle):
    w = synth.small_config(0, n_bins=16)
    plan = _plan(w, time_domain=True)
    b = plan.upload(synth.concat([w]))
    hp, hc, so = plan.td_sum(b, 10.0, 0)                 # no samples
    assert hp.numel() == 0
    hp, hc, so = plan.td_sum(b, 10.0, 3)                 # a few samples, spectrum has no bins
    tj, rp, rc = oracle.td_samples(w, 10.0, 3)
    assert rel_l2(hp.cpu().numpy(), rp) < 1e-5
    Hp, Hc = plan.td_spectrum(hp, hc, so, w.t[0], 10.0)
    assert Hp.numel() == 0
    none = w.with_modes(np.zeros(0, np.int64))          # no modes: zeros
    b0 = plan.upload(synth.concat([none]))
    hp, hc, so = plan.td_sum(b0, 10.0, 1000)
    assert torch.count_nonzero(hp) == 0 and torch.count_nonzero(hc) == 0
    plan.close()


def test_window_tiny_grids(oracle):
    w = synth.small_config(0, n_bins=16)
    for nf in (1, 2, 3):
        f = (np.arange(nf) + 40) / (w.t[-1] - w.t[0])
        wf = w.with_freqs(f)
        plan = _plan(wf, window="hann")
        hp, hc = plan.sum_modes(plan.upload(synth.concat([wf])))
        rp, rc = oracle.sum_modes(wf)
        assert np.allclose(hp.cpu().numpy(), oracle.hann_fd(rp), rtol=1e-10, atol=1e-10 * np.abs(rp).max())
        plan.close()


def test_select_edges(oracle):
    w = synth.small_config(0, n_bins=16)
    one = w.with_modes([5])
    plan = _plan(w)
    b = plan.upload(synth.concat([one]))
    assert plan.select_modes(b, 0.5).cpu().numpy().tolist() == [True]
    none = w.with_modes(np.zeros(0, np.int64))
    b0 = plan.upload(synth.concat([none]))
    assert plan.select_modes(b0, 0.5).numel() == 0
    plan.close()
