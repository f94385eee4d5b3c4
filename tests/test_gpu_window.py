"""The Hann window on the GPU (Sec. 2.3), through the C ABI: a plan with
window = "hann" returns the three-term convolution of its SPA sum.

Checks: parity with the oracle's SPA sum windowed by oracle.hann_fd (FP64 and
FP64X <= 1e-10, mixed <= 1e-5); bitwise equality with the same three-term
formula applied to the plan's own unwindowed output; batches; a non-uniform
grid is refused with EMRI_FD_ERR_FREQ; likelihood plans refuse a window."""
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


def _plan(wfs, prec, window, spa="standard"):
    return api.Plan(prec, conj_partners=True, max_waveforms=len(wfs), max_knots=max(w.K for w in wfs),
                    max_knots_total=sum(w.K for w in wfs), max_modes_total=sum(w.n_modes for w in wfs),
                    max_bins_total=sum(w.n_freqs for w in wfs), window=window, spa=spa)


def _run(wfs, prec, window, spa="standard"):
    plan = _plan(wfs, prec, window, spa)
    hp, hc = plan.sum_modes(plan.upload(synth.concat(wfs)))
    out = (hp.cpu().numpy(), hc.cpu().numpy())
    plan.close()
    return out


def _grid(T, n):
    return np.arange(1, n + 1) / T


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp64x", 1e-10), ("mixed", 1e-5)])
def test_parity_with_oracle(oracle, prec, tol):
    w = synth.small_config(0)
    T = w.t[-1] - w.t[0]
    w = w.with_freqs(_grid(T, 60000))
    hp, hc = oracle.sum_modes(w)
    ref = (oracle.hann_fd(hp), oracle.hann_fd(hc))
    got = _run([w], prec, "hann")
    for g, r in zip(got, ref):
        assert rel_l2(g, r) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_equals_formula_on_own_output(prec):
    w = synth.small_config(1)
    w = w.with_freqs(_grid(w.t[-1] - w.t[0], 20000))
    raw = _run([w], prec, None)
    win = _run([w], prec, "hann")
    for a, b in zip(raw, win):
        lo = np.concatenate([np.zeros(1, a.dtype), a[:-1]])
        hi = np.concatenate([a[1:], np.zeros(1, a.dtype)])
        ref = (0.5 * a - 0.25 * (lo + hi)).astype(a.dtype)
        assert np.array_equal(b, ref)


def test_batch_and_extended():
    ws = [synth.small_config(0), synth.small_config(2)]
    ws = [w.with_freqs(_grid(w.t[-1] - w.t[0], n)) for w, n in zip(ws, (5000, 7777))]
    hb = _run(ws, "fp64", "hann", spa="extended")
    off = 0
    for w in ws:
        hs = _run([w], "fp64", "hann", spa="extended")
        assert np.array_equal(hb[0][off:off + w.n_freqs], hs[0])
        off += w.n_freqs


def test_nonuniform_grid_refused():
    w = synth.small_config(0, n_bins=4096)
    f = w.freqs.copy()
    f[2000:] += 0.3 * (f[1] - f[0])
    w = w.with_freqs(f)
    plan = _plan([w], "fp64", "hann")
    with pytest.raises(api.EmriFdError) as e:
        plan.sum_modes(plan.upload(synth.concat([w])))
        plan.sync()
    assert e.value.code == 3   # EMRI_FD_ERR_FREQ
    plan.close()


def test_likelihood_plan_refuses_window():
    with pytest.raises(api.EmriFdError):
        api.Plan("fp64", max_modes_total=10, max_bins_total=100, likelihood=True, window="hann")


def test_paper_size_sampled(oracle):
    """The full 3,155,760-bin grid windowed on the GPU; the oracle evaluates the SPA sum
    at 1500 sampled bins and their two neighbours and applies the three-term form."""
    w = synth.paper_config(3)
    got = _run([w], "fp64", "hann")
    rng = np.random.default_rng(5)
    occ = np.nonzero(np.abs(got[0]) > 0)[0]
    sel = np.unique(np.concatenate([rng.choice(occ, 1000, replace=False),
                                    rng.integers(1, w.n_freqs - 1, 500), [0, w.n_freqs - 1]]))
    trip = np.unique(np.clip(np.concatenate([sel - 1, sel, sel + 1]), 0, w.n_freqs - 1))
    rp, rc = oracle.sum_modes(w, freqs=w.freqs[trip])
    pos = {b: i for i, b in enumerate(trip)}
    def win(h):
        out = []
        for b in sel:
            v = 0.5 * h[pos[b]]
            v -= 0.25 * (h[pos[b - 1]] if b - 1 >= 0 else 0.0)
            v -= 0.25 * (h[pos[b + 1]] if b + 1 < w.n_freqs else 0.0)
            out.append(v)
        return np.array(out)
    assert rel_l2(got[0][sel], win(rp)) <= 1e-10 and rel_l2(got[1][sel], win(rc)) <= 1e-10
