"""Whittle log-likelihood and its adjoint on the GPU (Eq. 13-14), through the
C ABI, against the CPU oracle and against finite differences."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import api, synth
from tests import likelihood_case as LC
from tests.gpu_util import plan_for, rel_l2
from tests.test_oracle_grad import safe_grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_12585_gb300 import build
    build.build()


def _gpu_like(wfs, data, grad=True):
    if not isinstance(wfs, (list, tuple)):
        wfs, data = [wfs], [data]
    plan = api.Plan("fp64", conj_partners=True, max_waveforms=len(wfs), max_knots=max(w.K for w in wfs),
                    max_knots_total=sum(w.K for w in wfs), max_modes_total=sum(w.n_modes for w in wfs),
                    max_bins_total=sum(w.n_freqs for w in wfs), likelihood=True)
    b = plan.upload(synth.concat(wfs))
    dev = plan.device
    cat = lambda i: torch.as_tensor(np.concatenate([d[i] for d in data])).to(dev)
    dp, dc = cat(0), cat(1)
    S = torch.as_tensor(np.concatenate([d[2] for d in data])).to(dev)
    df = torch.as_tensor(np.array([d[3] for d in data], np.float64)).to(dev)
    L, g = plan.loglike_and_grad(b, dp, dc, S, df, grad=grad)
    out = L.cpu().numpy(), ({k: v.cpu().numpy() for k, v in g.items()} if g else None)
    plan.close()
    return out


def _case(oracle, w, seed=3):
    w, dp, dc, S, df = LC.make(oracle, w, seed=seed)
    return w, (dp, dc, S, df)


def test_loglike_and_gradient_match_oracle_small(oracle):
    w, d = _case(oracle, synth.small_config(0, n_bins=8192))
    L, g = _gpu_like(w, d)
    Lo, go = oracle.loglike_grad(w, *d)
    assert abs(L[0] - Lo) <= 1e-10 * abs(Lo)
    for k in ("phi_phi", "phi_r", "omega_phi", "omega_r"):
        assert rel_l2(g[k], go[k]) <= 1e-8, k
    assert rel_l2(g["amp"], go["amp"].reshape(-1)) <= 1e-8


def test_loglike_and_gradient_match_oracle_full_likelihood_workload(oracle):
    """1 yr, 500 modes, 150 knots, 1,577,880 bins at df = 1/T, SNR 78"""
    w, d = _case(oracle, synth.likelihood_config(3))
    L, g = _gpu_like(w, d)
    Lo, go = oracle.loglike_grad(w, *d)
    assert abs(L[0] - Lo) <= 1e-10 * abs(Lo)
    for k in ("phi_phi", "phi_r", "omega_phi", "omega_r"):
        assert rel_l2(g[k], go[k]) <= 1e-8, k
    assert rel_l2(g["amp"], go["amp"].reshape(-1)) <= 1e-8


def test_gradient_central_differences():
    """Richardson central differences of the GPU likelihood along random knot
    directions, on a grid kept away from knot / end / turnover frequencies
    (the assignment of bins to branches is then fixed): <= 1e-6"""
    from oracle import oracle as O
    base = synth.small_config(0, n_bins=8192).with_modes(np.arange(20))
    base = base.with_freqs(safe_grid(base, margin=5e-6))
    w, d = _case(O, base)
    L0, g = _gpu_like(w, d)
    rng = np.random.default_rng(5)
    for which, step in (("phi_phi", 3e-5), ("phi_r", 3e-5), ("omega_phi", 1e-8), ("omega_r", 1e-8), ("amp", 1e-4)):
        if which == "amp":
            v = rng.normal(size=w.amp.shape) + 1j * rng.normal(size=w.amp.shape)
            h = step * np.abs(w.amp).max()
            gv = np.sum(g["amp"].reshape(w.amp.shape).real * v.real + g["amp"].reshape(w.amp.shape).imag * v.imag)
        else:
            v = rng.normal(size=w.K)
            h = step if which.startswith("phi") else step * np.abs(getattr(w, which)).max()
            gv = np.dot(g[which], v)
        fd = []
        for hh in (h, h / 2):
            Ls = []
            for sg in (1, -1):
                wp = w.with_freqs(w.freqs)
                if which == "amp":
                    wp.amp = w.amp + sg * hh * v
                else:
                    setattr(wp, which, getattr(w, which) + sg * hh * v)
                Ls.append(_gpu_like(wp, d, grad=False)[0][0])
            fd.append((Ls[0] - Ls[1]) / (2 * hh))
        rich = (4 * fd[1] - fd[0]) / 3
        assert abs(rich - gv) <= 1e-6 * abs(gv), (which, fd, gv)


def test_euler_identity(oracle):
    w, d = _case(oracle, synth.small_config(0, n_bins=8192))
    L, g = _gpu_like(w, d)
    lhs = np.sum(w.amp.reshape(-1).real * g["amp"].real + w.amp.reshape(-1).imag * g["amp"].imag)
    hp, hc = oracle.sum_modes(w)
    rhs = oracle.inner(d[0] - hp, hp, d[2], d[3]) + oracle.inner(d[1] - hc, hc, d[2], d[3])
    assert abs(lhs - rhs) <= 1e-9 * abs(rhs)


def test_batch_equals_singles(oracle):
    """The likelihood of a batch equals its singles bitwise (per-waveform fixed-order
    sums).  The gradient's bin stream is split over the grid's lanes by position, so the
    grouping of its sums depends on the batch: members agree with their singles to
    rounding (1e-12 relative per series), and a repeated call is bitwise identical."""
    w1, d1 = _case(oracle, synth.small_config(0, n_bins=4096))
    w2, d2 = _case(oracle, synth.paper_config(5, n_modes=200, T_years=0.5, grid="sparse", n_sparse=3000), seed=4)
    L, g = _gpu_like([w1, w2], [d1, d2])
    L1, g1 = _gpu_like(w1, d1)
    L2, g2 = _gpu_like(w2, d2)
    assert L[0] == L1[0] and L[1] == L2[0]
    na = w1.n_modes * w1.K
    pairs = [(g[k][: w1.K], g1[k]) for k in ("phi_phi", "phi_r", "omega_phi", "omega_r")]
    pairs += [(g[k][w1.K:], g2[k]) for k in ("phi_phi", "phi_r", "omega_phi", "omega_r")]
    pairs += [(g["amp"][:na], g1["amp"]), (g["amp"][na:], g2["amp"])]
    for x, y in pairs:
        assert rel_l2(x, y) <= 1e-12, rel_l2(x, y)
    La, ga = _gpu_like([w1, w2], [d1, d2])
    assert np.array_equal(La, L)
    for k in g:
        assert np.array_equal(ga[k], g[k])


def test_autograd_function(oracle):
    w, d = _case(oracle, synth.small_config(0, n_bins=4096))
    plan = plan_for([w])
    plan.close()
    plan = api.Plan("fp64", max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes, max_bins_total=w.n_freqs,
                    likelihood=True)
    b = plan.upload(synth.concat([w]))
    for k in ("phi_phi", "phi_r", "omega_phi", "omega_r", "amp"):
        b[k].requires_grad_(True)
    dev = plan.device
    dp, dc = (torch.as_tensor(x).to(dev) for x in d[:2])
    S = torch.as_tensor(d[2]).to(dev)
    df = torch.tensor([d[3]], dtype=torch.float64, device=dev)
    L = api.whittle_loglike(plan, b, dp, dc, S, df)
    (2.5 * L).backward()
    Lr, g = plan.loglike_and_grad({k: (v.detach() if hasattr(v, "detach") else v) for k, v in b.items()},
                                  dp, dc, S, df)
    assert float(L.detach()) == float(Lr[0])
    for k in ("phi_phi", "phi_r", "omega_phi", "omega_r"):
        assert torch.equal(b[k].grad, 2.5 * g[k])
    assert torch.equal(b["amp"].grad, 2.5 * torch.view_as_real(g["amp"]).reshape(-1))
    plan.close()


def test_autograd_rejects_knots_changed_in_place(oracle):
    """The knot tensors are saved for backward: changing one in place between the forward
    and backward passes makes autograd raise instead of returning a stale gradient."""
    w, d = _case(oracle, synth.small_config(0, n_bins=2048))
    plan = api.Plan("fp64", max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes, max_bins_total=w.n_freqs,
                    likelihood=True)
    b = plan.upload(synth.concat([w]))
    for k in ("phi_phi", "phi_r", "omega_phi", "omega_r", "amp"):
        b[k].requires_grad_(True)
    dev = plan.device
    dp, dc = (torch.as_tensor(x).to(dev) for x in d[:2])
    S = torch.as_tensor(d[2]).to(dev)
    df = torch.tensor([d[3]], dtype=torch.float64, device=dev)
    L = api.whittle_loglike(plan, b, dp, dc, S, df)
    with torch.no_grad():
        b["omega_r"].mul_(1.0 + 1e-9)
    with pytest.raises(RuntimeError):
        L.backward()
    plan.close()


@pytest.mark.parametrize("n_bins,n_modes", [(1 << 18, 1), (1 << 18, 2), (600, 2)])
def test_gradient_stream_extremes(oracle, n_bins, n_modes):
    """The adjoint's bin stream at its extremes, against the oracle's gradient: one or two
    voices on five knots over a dense grid, so that each (run, segment) item holds tens of
    thousands of bins and runs through hundreds of warps' ranges (the cross-warp chains);
    and 600 bins, fewer positions than the grid has lanes (warps with empty ranges)."""
    base = synth.small_config(0, n_bins=16)
    idx = np.array([0, 25, 50, 75, 99])
    w = base.with_modes([3, 14][:n_modes])   # (2, 1, -2) and (2, 2, -2)
    for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r"):
        setattr(w, k, getattr(w, k)[idx].copy())
    w.amp = np.ascontiguousarray(w.amp[:, idx])
    F = [(m * w.omega_phi + n * w.omega_r) / (2 * np.pi) for m, n in zip(w.m, w.n)]
    lo = min(np.abs(x).min() for x in F)
    hi = max(np.abs(x).max() for x in F)
    w = w.with_freqs(np.linspace(lo * 1.001, hi * 0.999, n_bins))
    w.meta["T"] = w.t[-1] - w.t[0]
    w, d = _case(oracle, w)
    L, g = _gpu_like(w, d)
    Lo, go = oracle.loglike_grad(w, *d)
    assert abs(L[0] - Lo) <= 1e-10 * abs(Lo)
    for k in ("phi_phi", "phi_r", "omega_phi", "omega_r"):
        assert rel_l2(g[k], go[k]) <= 1e-8, k
    assert rel_l2(g["amp"], go["amp"].reshape(-1)) <= 1e-8
