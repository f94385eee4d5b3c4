"""Parity of the extended stationary-phase form (Sec. 2.2, Eq. 7-10) on the GPU
with the CPU oracle, through the C ABI.

FP64 and FP64X plans: relative L2 <= 1e-10 per channel (the FP64 bar; the
K_{1/3} evaluation is good to ~3e-12).  Mixed plans: <= 1e-5.  Also: the
cubic-phase voice whose extended sum is an Airy function, the bins beside a
turnover (where the standard form diverges), determinism of batches, and the
plan options that are refused."""
import math

import numpy as np
import pytest

from paper_2307_12585_gb300 import api, synth
from tests import _analytic as AN
from tests.gpu_util import plan_for, rel_l2, run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL64 = 1e-10
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_12585_gb300 import build
    build.build()


def _cmp(got, ref, tol):
    for g, r in zip(got, ref):
        e = rel_l2(g, r)
        assert e <= tol, e
        assert np.array_equal(np.abs(g) > 0, np.abs(r) > 0)


@pytest.mark.parametrize("prec", ["fp64", "fp64x"])
@pytest.mark.parametrize("n_bins", [2 ** 15, 2 ** 15 - 13, 77])
def test_small_config(oracle, prec, n_bins):
    w = synth.small_config(0, n_bins=n_bins)
    _cmp(run(w, precision=prec, spa="extended"), oracle.sum_modes(w, spa="extended"), TOL64)


def test_small_config_mixed(oracle):
    w = synth.small_config(0, n_bins=2 ** 15)
    _cmp(run(w, precision="mixed", spa="extended"), oracle.sum_modes(w, spa="extended"), TOL32)


@pytest.mark.parametrize("prec", ["fp64", "fp64x", "mixed"])
def test_paper_sparse(oracle, prec):
    """2-yr, 2000-mode waveform on 1e4 log-spaced bins (many turnover voices)."""
    w = synth.paper_config(2, grid="sparse")
    _cmp(run(w, precision=prec, spa="extended"), oracle.sum_modes(w, spa="extended"),
         TOL32 if prec == "mixed" else TOL64)


@pytest.mark.parametrize("prec", ["fp64", "fp64x"])
def test_paper_dense_sampled(oracle, prec):
    """Full 3,155,760-bin grid on the GPU; 3000 sampled bins (2000 of them where
    some voice contributes) through the oracle."""
    w = synth.paper_config(3)
    hp, hc = run(w, precision=prec, spa="extended", tile_bins={"fp64": 128, "fp64x": 64}[prec])   # the bench's tiles
    rng = np.random.default_rng(7)
    occ = np.nonzero(np.abs(hp) > 0)[0]
    sel = np.unique(np.concatenate([rng.choice(w.n_freqs, 1000, replace=False), rng.choice(occ, 2000, replace=False)]))
    ref = oracle.sum_modes(w, freqs=w.freqs[sel], spa="extended")
    _cmp((hp[sel], hc[sel]), ref, TOL64)


@pytest.mark.parametrize("prec", ["fp64", "fp64x"])
def test_cubic_phase_voice_is_airy(prec):
    """The two roots of a cubic-phase voice add up to its exact Airy-function
    transform, including the bins within 1e-6 of the turnover frequency."""
    pytest.importorskip("scipy")
    from scipy.special import airy
    w, p = AN.quadratic_voice(nb=6000)
    f = np.unique(np.concatenate([np.linspace(1.3e-3, 2.1e-3, 6000), p["Fs"] - np.logspace(-13, -6, 40)]))
    w = w.with_freqs(f)
    hp, hc = run(w, precision=prec, conj=False, spa="extended")
    from oracle import oracle as O
    Y = O.swsh_closed(int(w.l[0]), int(w.m[0]), w.theta, w.phi)
    got = (hp - 1j * hc) / (Y * w.prefactor) / w.amp[0, 0]
    a = (math.pi * p["kappa"]) ** (-1.0 / 3.0)
    exp = np.exp(1j * (2 * math.pi * f * p["ts"] - p["Ps"])) * 2 * math.pi * a * airy(-2 * math.pi * (p["Fs"] - f) * a)[0]
    lo = p["Fs"] - 0.5 * p["kappa"] * (p["T"] - p["ts"]) ** 2
    both = (f < p["Fs"]) & (f > lo * 1.0001)
    err = np.abs(got[both] - exp[both]) / np.abs(exp[both]).max()
    assert err.max() < 1e-10
    assert np.all(got[f > p["Fs"]] == 0)


def test_batch_equals_singles():
    ws = [synth.small_config(0, n_bins=3000), synth.paper_config(4, grid="sparse"), synth.small_config(5, n_bins=777)]
    for prec in ("fp64", "fp64x"):
        hb = run(ws, precision=prec, spa="extended")
        off = 0
        for w in ws:
            hs = run(w, precision=prec, spa="extended")
            n = w.n_freqs
            assert np.array_equal(hb[0][off:off + n], hs[0]) and np.array_equal(hb[1][off:off + n], hs[1])
            off += n


def test_graph_replay_extended():
    w = synth.small_config(0, n_bins=4096)
    plan = plan_for([w], "fp64", spa="extended")
    b = plan.upload(synth.concat([w]))
    ref = plan.sum_modes(b)
    ref = (ref[0].clone(), ref[1].clone())
    out = (torch.zeros_like(ref[0]), torch.zeros_like(ref[1]))
    g = plan.capture(b, out)
    g.replay()
    plan.sync()
    assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
    g.close()
    plan.close()


def test_refused_options():
    with pytest.raises(api.EmriFdError):
        api.Plan("fp64", max_modes_total=10, max_bins_total=100, likelihood=True, spa="extended")
    d = api.emri_fd_desc()
    d.precision = 0; d.conj_partners = 1; d.max_waveforms = 1; d.max_knots = 10
    d.max_modes_total = 1; d.max_bins_total = 10; d.spa_form = 2
    with pytest.raises(api.EmriFdError):
        api.emri_fd_plan(d, 0)
