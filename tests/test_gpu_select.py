"""Mode selection on the GPU (Sec. 2.1) through the C ABI: bit-exact against
the oracle (every power, cumulative sum and comparison is one FP64 operation
in the defined order), on the paper's 3294-mode pool at several thresholds,
on batches with different mode and knot counts, on ties, and at the limits."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import api, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_12585_gb300 import build
    build.build()


def _plan(wfs):
    return api.Plan("fp64", max_waveforms=len(wfs), max_knots=max(w.K for w in wfs),
                    max_knots_total=sum(w.K for w in wfs), max_modes_total=sum(w.n_modes for w in wfs),
                    max_bins_total=max(1, sum(w.n_freqs for w in wfs)))


def _select(wfs, eps):
    plan = _plan(wfs)
    b = plan.upload(synth.concat(wfs))
    out = plan.select_modes(b, eps).cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-5, 1e-8, 0.0, 1.0, -1.0])
def test_paper_pool_bit_exact(oracle, eps):
    w = synth.paper_config(1, n_modes=3294, grid="sparse", n_sparse=16)
    got = _select([w], eps)
    assert np.array_equal(got, oracle.select_modes(w.amp, eps))


def test_batch(oracle):
    ws = [synth.paper_config(5, n_modes=n, grid="sparse", n_sparse=16) for n in (3294, 700)]
    ws.append(synth.small_config(3, n_bins=64))
    got = _select(ws, 1e-4)
    off = 0
    for w in ws:
        assert np.array_equal(got[off:off + w.n_modes], oracle.select_modes(w.amp, 1e-4))
        off += w.n_modes


def test_ties_and_small(oracle):
    w = synth.small_config(0, n_bins=64)
    w.amp[:] = 3 + 4j                         # all powers equal: the index decides
    for eps in (0.5, 0.1, 1 / 55):
        assert np.array_equal(_select([w], eps), oracle.select_modes(w.amp, eps))
    one = w.with_modes([7])
    assert _select([one], 0.5).tolist() == [True]


def test_capacity_and_arguments():
    w = synth.small_config(0, n_bins=64)
    big = w.with_modes(np.zeros(8193, np.int64))
    plan = _plan([big])
    b = plan.upload(synth.concat([big]))
    with pytest.raises(api.EmriFdError) as e:
        plan.select_modes(b, 1e-3)
    assert e.value.code == 6   # EMRI_FD_ERR_CAPACITY
    with pytest.raises(api.EmriFdError) as e:
        plan.select_modes(b, float("nan"))
    assert e.value.code == 1   # EMRI_FD_ERR_ARG
    plan.close()
