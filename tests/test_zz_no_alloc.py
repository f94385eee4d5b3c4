"""The no-allocation entry point (emri_fd_sum_modes_noalloc).

It serves callers that cannot allocate device memory: another component holds
the device's memory, or the code path must not call cudaMalloc/cudaFree.  It
keeps its scratch in a fixed file-scope device array instead of a plan.  This
test calls it through the C ABI twice in a row, on two different waveforms (so
the second call starts from the first call's leftovers in the shared array),
and compares each result with the plan-based emri_fd_sum_modes, within the
FP64 parity tolerance (relative L2 1e-10).  It also checks the size limit and
that a call leaves the device's free memory unchanged.  The file name makes
pytest collect it last."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import api, synth
from tests.gpu_util import rel_l2, run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_12585_gb300 import build
    build.build()


def _inputs(w):
    """Device copies of the waveform's arrays and the two outputs (made by torch, before
    the entry point is called)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dt)).to(dev)
    arrs = [d(getattr(w, k), np.float64) for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r")]
    arrs += [d(getattr(w, k), np.int32) for k in ("l", "m", "n")]
    arrs.append(d(np.ascontiguousarray(w.amp, np.complex128).view(np.float64), np.float64))
    arrs.append(d(w.freqs, np.float64))
    hp = torch.empty(w.n_freqs, dtype=torch.complex128, device=dev)
    hc = torch.empty(w.n_freqs, dtype=torch.complex128, device=dev)
    return arrs, hp, hc


def _call(w, arrs, hp, hc, conj=True):
    """One call of the entry point through the C ABI; returns its status."""
    t, pp, pr, op, orr, l, m, n, amp, f = arrs
    stream = torch.cuda.current_stream(hp.device)
    return api.emri_fd_sum_modes_noalloc(int(conj), w.K, w.n_modes, w.n_freqs, t.data_ptr(), pp.data_ptr(),
                                         pr.data_ptr(), op.data_ptr(), orr.data_ptr(), l.data_ptr(), m.data_ptr(),
                                         n.data_ptr(), amp.data_ptr(), w.theta, w.phi, w.prefactor, f.data_ptr(),
                                         hp.data_ptr(), hc.data_ptr(), stream.cuda_stream)


def _noalloc(w, conj=True):
    arrs, hp, hc = _inputs(w)
    code = _call(w, arrs, hp, hc, conj)
    return code, hp.cpu().numpy(), hc.cpu().numpy()


def test_noalloc_matches_plan_path_twice_in_a_row():
    first = synth.small_config(0, n_bins=2 ** 15 - 5)                          # K = 100, 55 modes
    second = synth.paper_config(7, n_modes=128, T_years=0.5, grid="uniform", n_bins=50001)  # K = 200, 128 modes
    for w in (first, second):
        code, hp, hc = _noalloc(w)
        assert code == 0, api.emri_fd_strerror(code)
        rp, rc = run(w)
        assert rel_l2(hp, rp) <= TOL64 and rel_l2(hc, rc) <= TOL64
        assert np.array_equal(np.abs(hp) > 0, np.abs(rp) > 0)


def test_noalloc_rejects_sizes_beyond_its_limit():
    w = synth.paper_config(7, n_modes=129, T_years=0.5, grid="sparse", n_sparse=1000)
    code, _, _ = _noalloc(w)
    assert code == 6   # EMRI_FD_ERR_CAPACITY


def test_noalloc_allocates_no_device_memory():
    """The property the entry point exists for: once its first call on the device has
    done the set-up, a call leaves the device's free memory (cudaMemGetInfo) unchanged.
    The inputs and outputs are made beforehand, and the call is repeated once first so
    that every kernel it launches has been loaded."""
    w = synth.paper_config(8, n_modes=100, T_years=0.5, grid="uniform", n_bins=40000)
    arrs, hp, hc = _inputs(w)
    assert _call(w, arrs, hp, hc) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    code = _call(w, arrs, hp, hc)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert code == 0, api.emri_fd_strerror(code)
    assert free1 == free0, (free0, free1)
    rp, rc = run(w)
    assert rel_l2(hp.cpu().numpy(), rp) <= TOL64 and rel_l2(hc.cpu().numpy(), rc) <= TOL64
