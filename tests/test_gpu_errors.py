"""Error behaviour of the C ABI on a device: host-side shape checks return at
once; value checks run on the device and are reported by emri_fd_sync (or by the
call itself when its outputs are host memory, since it then synchronises).  The
invalid inputs here are all rejected by those checks (nothing out of bounds
is ever read or written)."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import api, synth
from tests.gpu_util import plan_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _status(w, mutate=None, conj=True):
    plan = plan_for([w], conj=conj)
    b = synth.concat([w])
    if mutate:
        mutate(b)
    db = plan.upload(b)
    try:
        plan.sum_modes(db, check=True)
        code = 0
    except api.EmriFdError as e:
        code = e.code
    # the same plan stays usable after an error (the status was cleared by the sync)
    hp, _ = plan.sum_modes(plan.upload(synth.concat([w])))
    assert torch.isfinite(hp.real).all() and torch.isfinite(hp.imag).all()
    plan.close()
    return code


def test_valid_is_ok():
    assert _status(synth.small_config(0, n_bins=500)) == 0


def test_non_increasing_knots():
    def m(b):
        b["t"] = b["t"].copy()
        b["t"][10] = b["t"][9]
    assert _status(synth.small_config(0, n_bins=500), m) == 2


def test_bad_frequencies():
    def m(b):
        b["freqs"] = b["freqs"].copy()
        b["freqs"][7] = b["freqs"][3]
    assert _status(synth.small_config(0, n_bins=500), m) == 3


def test_bad_mode_numbers():
    def m(b):
        b["l"] = b["l"].copy()
        b["l"][0] = 1
    assert _status(synth.small_config(0, n_bins=500), m) == 4


def test_negative_m_with_partners():
    def m(b):
        b["m"] = b["m"].copy()
        b["m"][0] = -1
    assert _status(synth.small_config(0, n_bins=500), m) == 4


def test_nonfinite_amplitude():
    def m(b):
        b["amp"] = b["amp"].copy()
        b["amp"][5] = np.nan
    assert _status(synth.small_config(0, n_bins=500), m) == 5


def test_host_side_shape_errors():
    w = synth.small_config(0, n_bins=500)
    plan = plan_for([w])
    b = plan.upload(synth.concat([w]))
    bad = dict(b)
    bad["knot_off"] = np.array([0, 3], np.int64)        # K = 3 < 4
    with pytest.raises(api.EmriFdError) as e:
        plan.sum_modes(bad)
    assert e.value.code == 2
    big = dict(b)
    big["freq_off"] = np.array([0, 10 ** 6], np.int64)  # above max_bins_total
    with pytest.raises(api.EmriFdError) as e:
        plan.sum_modes(big)
    assert e.value.code == 6
    plan.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_host_outputs_report_device_errors(pinned):
    """With host outputs the call synchronises, so it returns its own device-detected
    error (here: frequencies out of order, staged on the side stream), and the plan
    stays usable."""
    w = synth.small_config(0, n_bins=800)
    plan = plan_for([w])
    hb = api.host_batch(synth.concat([w]))
    hb["freqs"] = hb["freqs"].copy()
    hb["freqs"][100] = hb["freqs"][50]
    out = None
    if pinned:
        out = (torch.empty(800, dtype=torch.complex128).pin_memory(), torch.empty(800, dtype=torch.complex128).pin_memory())
    with pytest.raises(api.EmriFdError) as e:
        plan.sum_modes_host(hb, out=out)
    assert e.value.code == 3
    good = api.host_batch(synth.concat([w]))
    hp, hc = plan.sum_modes_host(good, out=out)
    assert np.all(np.isfinite(np.asarray(hp))) and np.any(np.asarray(hp) != 0)
    plan.close()
