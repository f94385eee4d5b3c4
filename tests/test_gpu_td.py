"""Time-domain comparator on the GPU (Sec. 2.3, 3.2), through the C ABI.

TD samples (FP32 arithmetic, integer phase) against the oracle's FP64 TD sum
(relative L2 <= 1e-5); batches equal singles bitwise; the cuFFT spectrum
against numpy's FFT of the same samples and against the oracle's DFT, with
and without the Hann window; and the FD/TD comparison the paper makes: the
GPU's SPA sum against the GPU's TD spectrum on the DFT grid, whose mismatch
the window reduces."""
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


def _plan(wfs, nbins=1, **kw):
    return api.Plan("fp64", max_waveforms=len(wfs), max_knots=max(w.K for w in wfs),
                    max_knots_total=sum(w.K for w in wfs), max_modes_total=sum(w.n_modes for w in wfs),
                    max_bins_total=max(nbins, sum(w.n_freqs for w in wfs)), time_domain=True, **kw)


def _nsamp(w, dt):
    return int(np.floor((w.t[-1] - w.t[0]) / dt))


def test_samples_match_oracle(oracle):
    w = synth.small_config(0, n_bins=16)
    dt = 10.0
    N = _nsamp(w, dt) + 100                       # past the last knot: zeros
    plan = _plan([w])
    hp, hc, so = plan.td_sum(plan.upload(synth.concat([w])), dt, N)
    tj, rp, rc = oracle.td_samples(w, dt, N)
    assert rel_l2(hp.cpu().numpy(), rp) < 1e-5 and rel_l2(hc.cpu().numpy(), rc) < 1e-5
    assert np.all(hp.cpu().numpy()[tj > w.t[-1]] == 0)
    plan.close()


def test_batch_equals_singles():
    ws = [synth.small_config(0, n_bins=16), synth.small_config(4, n_bins=16)]
    dts, Ns = [10.0, 25.0], [_nsamp(ws[0], 10.0), _nsamp(ws[1], 25.0) - 333]
    plan = _plan(ws)
    hb = plan.td_sum(plan.upload(synth.concat(ws)), dts, Ns)
    plan.close()
    off = 0
    for w, d, n in zip(ws, dts, Ns):
        p1 = _plan([w])
        hs = p1.td_sum(p1.upload(synth.concat([w])), d, n)
        assert torch.equal(hb[0][off:off + n], hs[0]) and torch.equal(hb[1][off:off + n], hs[1])
        p1.close()
        off += n


@pytest.mark.parametrize("window", [None, "hann"])
def test_spectrum(oracle, window):
    w = synth.small_config(0, n_bins=16).with_modes([3, 10, 17, 30, 44])
    dt = 10.0
    N = _nsamp(w, dt)
    plan = _plan([w])
    hp, hc, so = plan.td_sum(plan.upload(synth.concat([w])), dt, N)
    Hp, Hc = plan.td_spectrum(hp, hc, so, w.t[0], dt, window=window)
    f = plan.td_freqs(so, dt)
    Hp, Hc = Hp.cpu().numpy(), Hc.cpu().numpy()
    # the FFT step alone: numpy (FP64) DFT of the same FP32 samples
    win = oracle.hann_td(N) if window == "hann" else 1.0
    k = np.arange(1, N // 2)
    for H, x in ((Hp, hp), (Hc, hc)):
        ref = dt * N * np.fft.ifft(x.cpu().numpy().astype(np.float64) * win)[k]
        assert rel_l2(H, ref) < 3e-6
    # against the oracle's FP64 TD sum and DFT
    fk, Rp, Rc = oracle.td_dft(w, dt, window=window, N=N)
    assert np.allclose(f, fk, rtol=1e-15, atol=0)
    assert rel_l2(Hp, Rp) < 1e-5 and rel_l2(Hc, Rc) < 1e-5
    plan.close()


def _match(a, b):
    return float(np.real(np.vdot(a, b)) / np.sqrt(np.real(np.vdot(a, a)) * np.real(np.vdot(b, b))))


def test_fd_vs_td_on_gpu():
    """The paper's comparison (flat PSD): FD SPA sum vs the DFT of the TD sum on
    the same grid; the Hann window (applied to both) lowers the mismatch."""
    w = synth.small_config(0, n_bins=16)
    dt = 10.0
    N = _nsamp(w, dt)
    plan = _plan([w])
    hp, hc, so = plan.td_sum(plan.upload(synth.concat([w])), dt, N)
    res = {}
    for window in (None, "hann"):
        Hp, Hc = plan.td_spectrum(hp, hc, so, w.t[0], dt, window=window)
        f = plan.td_freqs(so, dt)
        fd = _plan([w.with_freqs(f)], nbins=f.size, window=window)
        Fp, Fc = fd.sum_modes(fd.upload(synth.concat([w.with_freqs(f)])))
        band = (f > 1e-5) & (f < 4.9e-2)
        res[window] = [1 - _match(a.cpu().numpy()[band], b.cpu().numpy()[band].astype(np.complex128))
                       for a, b in ((Fp, Hp), (Fc, Hc))]
        fd.close()
    plan.close()
    for c in range(2):
        assert res[None][c] < 2e-2
        assert res["hann"][c] < 0.2 * res[None][c]


def test_requires_time_domain_plan():
    w = synth.small_config(0, n_bins=16)
    plan = api.Plan("fp64", max_modes_total=w.n_modes, max_bins_total=16, max_knots=w.K)
    with pytest.raises(api.EmriFdError):
        plan.td_sum(plan.upload(synth.concat([w])), 10.0, 1000)
    plan.close()


def test_paper_size_sampled(oracle):
    """The full 2-yr, 2000-mode waveform at dt = 10 s (6,311,520 samples) on the GPU;
    2000 sampled samples through the oracle, and the whole spectrum against numpy's
    FFT of the same samples."""
    w = synth.paper_config(2, grid="sparse", n_sparse=16)
    dt = 10.0
    N = _nsamp(w, dt)
    plan = _plan([w])
    hp, hc, so = plan.td_sum(plan.upload(synth.concat([w])), dt, N)
    idx = np.unique(np.random.default_rng(3).integers(0, N, 2000))
    tj, rp, rc = oracle.td_samples(w, dt, N, idx=idx)
    gp, gc = hp.cpu().numpy(), hc.cpu().numpy()
    assert rel_l2(gp[idx], rp) < 1e-5 and rel_l2(gc[idx], rc) < 1e-5
    Hp, Hc = plan.td_spectrum(hp, hc, so, w.t[0], dt)
    k = np.arange(1, N // 2)
    for H, x in ((Hp, gp), (Hc, gc)):
        ref = dt * N * np.fft.ifft(x.astype(np.float64))[k]
        assert rel_l2(H.cpu().numpy(), ref) < 3e-6
    plan.close()
