"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 form: relative L2 <= 1e-10 per channel (h+ and hx), the FP64 parity bar of
this path; integer work (which bins a branch covers, mode-bin counts) is compared
exactly.  Mixed form: <= 1e-5."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import synth
from tests import _analytic as AN
from tests.gpu_util import rel_l2, run

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
        # the same bins are covered (no branch assignment differences)
        assert np.array_equal(np.abs(g) > 0, np.abs(r) > 0)


PRECS = ["fp64", "fp64x"]   # both must meet the FP64 tolerance
BENCH_TILE = {"fp64": 128, "fp64x": 64, "mixed": 64}   # the tile sizes bench.py times each form at


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n_bins", [2 ** 15, 2 ** 15 - 13, 1000, 77])
def test_small_config(oracle, n_bins, prec):
    w = synth.small_config(0, n_bins=n_bins)
    _cmp(run(w, precision=prec), oracle.sum_modes(w), TOL64)


@pytest.mark.parametrize("tb", [32, 64, 128])
def test_tile_shapes(oracle, tb):
    w = synth.small_config(0, n_bins=5000)
    _cmp(run(w, tile_bins=tb), oracle.sum_modes(w), TOL64)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp64x", TOL64), ("mixed", TOL32)])
@pytest.mark.parametrize("tb,split", [(32, 2), (32, 4), (64, 4)])
def test_tile_split_clusters(oracle, prec, tol, tb, split):
    """Tiles shared by a thread-block cluster of 2 or 4 CTAs (partials combined through
    distributed shared memory): the small config and the sparse paper grid against the
    oracle, and close to the unsplit call (only the grouping of the sums differs: 1e-14
    for FP64, 1e-13 for the FP32-pair form, whose unit roundoff is 2^-48)."""
    regroup = {"fp64": 1e-14, "fp64x": 1e-13}
    for w in (synth.small_config(0, n_bins=3001), synth.paper_config(1, grid="sparse")):
        got = run(w, precision=prec, tile_bins=tb, tile_split=split)
        _cmp(got, oracle.sum_modes(w), tol)
        if prec != "mixed":
            ref = run(w, precision=prec, tile_bins=tb)
            for x, y in zip(got, ref):
                assert rel_l2(x, y) < regroup[prec]


@pytest.mark.parametrize("split", [2, 4])
def test_tile_split_batch_extended_graph(oracle, split):
    """With a split: batch = singles bitwise, the extended form against its oracle, and
    graph replay = direct call; a split with 128-bin tiles is refused."""
    from paper_2307_12585_gb300 import api
    from tests.gpu_util import plan_for
    wfs = [synth.small_config(0, n_bins=3001), synth.paper_config(3, n_modes=300, T_years=0.5, grid="sparse", n_sparse=4000)]
    bh, bc = run(wfs, tile_bins=64, tile_split=split)
    off = 0
    for w in wfs:
        sh, sc = run(w, tile_bins=64, tile_split=split)
        assert np.array_equal(bh[off:off + w.n_freqs], sh) and np.array_equal(bc[off:off + w.n_freqs], sc)
        off += w.n_freqs
    w = synth.paper_config(2, grid="sparse")
    _cmp(run(w, spa="extended", tile_bins=32, tile_split=split), oracle.sum_modes(w, spa="extended"), TOL64)
    plan = plan_for(wfs, tile_bins=32, tile_split=split)
    b = plan.upload(synth.concat(wfs))
    direct = [x.clone() for x in plan.sum_modes(b)]
    out = (torch.zeros_like(direct[0]), torch.zeros_like(direct[1]))
    g = plan.capture(b, out)
    g.replay()
    plan.sync()
    assert torch.equal(out[0], direct[0]) and torch.equal(out[1], direct[1])
    g.close()
    with pytest.raises(api.EmriFdError):
        plan.set_tile(128)
    plan.close()
    with pytest.raises(api.EmriFdError):
        api.Plan("fp64", max_waveforms=1, max_knots=100, max_modes_total=10, max_bins_total=10, tile_split=2)


def test_tile_shapes_agree():
    w = synth.small_config(0, n_bins=3001)
    a = run(w, tile_bins=32)
    for tb in (64, 128):
        b = run(w, tile_bins=tb)
        for x, y in zip(a, b):
            assert rel_l2(x, y) < 1e-14


def test_mode_bin_count_matches_oracle(oracle):
    w = synth.small_config(0)
    _, _, st = run(w, stats=True)
    _, _, ost = oracle.sum_modes(w, return_stats=True)
    # the oracle expands conjugate partners into separate voices
    assert 2 * st["mode_bins"] == ost["contributions"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K", [50, 100, 400])
def test_power_law_chirp(oracle, K, prec):
    w, p = synth.chirp_config(K=K, n_bins=2 ** 13)
    _cmp(run(w, conj=False, precision=prec), oracle.sum_modes(w, conj_partners=False), TOL64)


@pytest.mark.parametrize("prec", PRECS)
def test_linear_chirp_closed_form(oracle, prec):
    w, p = AN.linear_chirp()
    hp, hc = run(w, conj=False, precision=prec)
    ref = oracle.sum_modes(w, conj_partners=False)
    _cmp((hp, hc), ref, TOL64)
    Y = oracle.swsh_closed(2, 1, w.theta, w.phi)
    got = (hp - 1j * hc) / (Y * w.amp[0, 0])
    exp = AN.linear_chirp_expected(w, p, w.freqs)
    assert np.max(np.abs(got - exp)) / np.max(np.abs(exp)) < (1e-11 if prec == "fp64" else 5e-11)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("uniform", [False, True])
def test_quadratic_turnover(oracle, prec, uniform):
    # uniform knots put the maximum mid-segment; the dense cluster below F* has both of its
    # roots in that segment
    w, p = AN.quadratic_voice(K=40, uniform=True) if uniform else AN.quadratic_voice()
    w = w.with_freqs(np.unique(np.concatenate([w.freqs, p["Fs"] * (1 - np.logspace(-5.9, -3.3, 160))])))
    got = run(w, conj=False, precision=prec)
    ref = oracle.sum_modes(w, conj_partners=False)
    dist = (p["Fs"] - w.freqs) / p["Fs"]
    # Near the maximum the root is ill-conditioned: a residual rounded to eps F* moves it by
    # eps F*/|F'|, and with F'^2 = 2|F''|(F* - f) the weight 1/sqrt|F'| takes a relative error
    # eps/(4 dist).  Each bin of the cluster is held to eps/dist, eps the unit of the form's
    # arithmetic (2^-53 in FP64; 2^-47 for FP32 pairs); bins away from F* to the usual bound.
    eps = 2.0 ** -53 if prec == "fp64" else 2.0 ** -47
    near = (dist > 0) & (dist < 1e-3)
    away = np.abs(dist) >= 1e-3
    for g, r in zip(got, ref):
        assert rel_l2(g[away], r[away]) <= TOL64
        rel = np.abs(g[near] - r[near]) / np.abs(r[near])
        assert np.all(rel <= np.maximum(eps / dist[near], 1e-12)), np.max(rel * dist[near])
    assert np.array_equal(np.abs(got[0]) > 0, np.abs(ref[0]) > 0)


@pytest.mark.parametrize("prec", PRECS)
def test_sparse_paper_grid(oracle, prec):
    w = synth.paper_config(1, grid="sparse")
    _cmp(run(w, precision=prec), oracle.sum_modes(w), TOL64)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [1, 2])
def test_paper_config_sampled(oracle, seed, prec):
    """Full-size 2 yr waveform (2000 modes, 3,155,760 bins) in the bench's launch
    configuration; the oracle evaluates ~4000 sampled bins (bins are independent)."""
    w = synth.paper_config(seed)
    hp, hc = run(w, precision=prec, tile_bins=BENCH_TILE[prec])
    rng = np.random.default_rng(seed)
    occupied = np.nonzero(np.abs(hp) > 0)[0]
    sel = np.unique(np.concatenate([rng.choice(w.n_freqs, 1000, replace=False),
                                    rng.choice(occupied, 3000, replace=False)]))
    rp, rc = oracle.sum_modes(w, freqs=w.freqs[sel])
    _cmp((hp[sel], hc[sel]), (rp, rc), TOL64)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_equals_singles_bitwise(prec):
    wfs = [synth.small_config(0, n_bins=3001), synth.paper_config(3, n_modes=300, T_years=0.5, grid="sparse", n_sparse=4000),
           synth.chirp_config(K=60, n_bins=999)[0]]
    bh, bc = run(wfs, precision=prec)
    off = 0
    for w in wfs:
        sh, sc = run(w, precision=prec)
        assert np.array_equal(bh[off:off + w.n_freqs], sh) and np.array_equal(bc[off:off + w.n_freqs], sc)
        off += w.n_freqs


def test_host_pointer_path_equals_device_path():
    from paper_2307_12585_gb300 import api
    from tests.gpu_util import plan_for
    w = synth.small_config(0, n_bins=4000)
    plan = plan_for([w])
    b = synth.concat([w])
    dh, dc = plan.sum_modes(plan.upload(b))
    hh, hc = plan.sum_modes_host(api.host_batch(b))
    assert np.array_equal(dh.cpu().numpy(), hh) and np.array_equal(dc.cpu().numpy(), hc)
    plan.close()


@pytest.mark.parametrize("prec,window", [("fp64", None), ("mixed", None), ("fp64", "hann")])
def test_pinned_host_outputs_written_in_place(prec, window):
    """Page-locked host outputs are written by the kernels directly; the result is
    bitwise the device-pointer result (also with no modes at all)."""
    from paper_2307_12585_gb300 import api
    w = synth.small_config(0, n_bins=5000)
    for wf in (w, w.with_modes(np.zeros(0, np.int64))):
        plan = api.Plan(prec, conj_partners=True, max_waveforms=1, max_knots=w.K, max_modes_total=w.n_modes,
                        max_bins_total=w.n_freqs, window=window)
        b = synth.concat([wf])
        dh, dc = plan.sum_modes(plan.upload(b))
        cdt = torch.complex64 if prec == "mixed" else torch.complex128
        out = (torch.full((w.n_freqs,), 7.0, dtype=cdt).pin_memory(), torch.full((w.n_freqs,), 7.0, dtype=cdt).pin_memory())
        plan.sum_modes_host(api.host_batch(b), out=out)
        assert torch.equal(dh.cpu(), out[0]) and torch.equal(dc.cpu(), out[1])
        plan.close()


def test_pinned_host_outputs_batch():
    """A batch of three waveforms (different grids) with page-locked outputs and pageable
    inputs equals the device-pointer call bitwise."""
    from paper_2307_12585_gb300 import api
    from tests.gpu_util import plan_for
    wfs = [synth.small_config(0, n_bins=3001), synth.small_config(1, n_bins=777), synth.small_config(2, n_bins=4096)]
    plan = plan_for(wfs)
    b = synth.concat(wfs)
    dh, dc = plan.sum_modes(plan.upload(b))
    nf = sum(w.n_freqs for w in wfs)
    out = (torch.empty(nf, dtype=torch.complex128).pin_memory(), torch.empty(nf, dtype=torch.complex128).pin_memory())
    plan.sum_modes_host(api.host_batch(b), out=out)
    assert torch.equal(dh.cpu(), out[0]) and torch.equal(dc.cpu(), out[1])
    plan.close()


def test_host_inputs_device_outputs_back_to_back():
    """Page-locked host inputs (the frequency grid staged on the side stream) with device
    outputs, two calls in a row without a sync in between and with different grids:
    each equals its device-input result bitwise (the second staging waits for the
    first call's readers)."""
    from paper_2307_12585_gb300 import api
    from tests.gpu_util import plan_for
    w1 = synth.small_config(0, n_bins=6000)
    w2 = synth.small_config(1, n_bins=6000).with_freqs(np.linspace(2e-4, 1.5e-2, 6000))
    plan = plan_for([w1])
    refs = []
    for w in (w1, w2):
        hp, hc = plan.sum_modes(plan.upload(synth.concat([w])))
        refs.append((hp.cpu(), hc.cpu()))
    hbs = []
    for w in (w1, w2):
        hb = api.host_batch(synth.concat([w]))
        for k in list(hb):
            if isinstance(hb[k], np.ndarray) and k not in ("knot_off", "mode_off", "freq_off"):
                hb[k] = torch.from_numpy(hb[k]).pin_memory()
        hbs.append(hb)
    outs = [(torch.empty(6000, dtype=torch.complex128, device="cuda"), torch.empty(6000, dtype=torch.complex128, device="cuda"))
            for _ in range(2)]
    for i in range(2):
        plan.sum_modes(hbs[i], out=outs[i], check=False)
    plan.sync()
    for i in range(2):
        assert torch.equal(outs[i][0].cpu(), refs[i][0]) and torch.equal(outs[i][1].cpu(), refs[i][1])
    plan.close()


def test_degenerate_inputs(oracle):
    w = synth.small_config(0, n_bins=2000)
    # bins where no voice is present
    far = w.with_freqs(np.linspace(0.5, 0.6, 100))
    hp, hc = run(far)
    assert np.all(hp == 0) and np.all(hc == 0)
    # a single bin
    one = w.with_freqs(w.freqs[500:501])
    _cmp(run(one), oracle.sum_modes(one), TOL64)
    # minimum knot count
    t4 = synth.small_config(0, n_bins=2000)
    idx = np.array([0, 33, 66, 99])
    for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r"):
        setattr(t4, k, getattr(t4, k)[idx].copy())
    t4.amp = np.ascontiguousarray(t4.amp[:, idx])
    _cmp(run(t4), oracle.sum_modes(t4), TOL64)


@pytest.mark.parametrize("prec", PRECS)
def test_batched_workload_sampled(oracle, prec):
    """The batched workload's recipe (N_m ~ U{50..3000}, T ~ U(0.5, 4) yr, N_f log-uniform in
    [1e4, 6e6], uniform or log grids) for 24 waveforms (17.6e6 bins) in one call at the
    tile size the autotuner picks: 8 of the waveforms against the oracle on 300 sampled
    bins each (bins are independent)."""
    from paper_2307_12585_gb300 import autotune
    from tests.gpu_util import plan_for
    wfs = synth.batch_config(24)
    plan = plan_for(wfs, precision=prec)
    b = plan.upload(synth.concat(wfs))
    out = plan.sum_modes(b)
    autotune.tune(plan, b, out, use_cache=False)
    hp, hc = (x.cpu().numpy() for x in plan.sum_modes(b, out=out))
    plan.close()
    off = np.concatenate([[0], np.cumsum([w.n_freqs for w in wfs])])
    rng = np.random.default_rng(24)
    for i in rng.choice(len(wfs), 8, replace=False):
        w = wfs[i]
        idx = np.sort(rng.choice(w.n_freqs, min(300, w.n_freqs), replace=False))
        rp, rc = oracle.sum_modes(w, freqs=w.freqs[idx])
        _cmp((hp[off[i]:off[i + 1]][idx], hc[off[i]:off[i + 1]][idx]), (rp, rc), TOL64)


@pytest.mark.parametrize("prec", ["fp64", "fp64x", "mixed"])
def test_batch_with_empty_members(prec):
    """A batch whose members include a waveform with no bins and one with no modes, between
    ordinary ones: every member equals its single-waveform call bitwise, the no-mode member
    is zero, and the zero-bin member takes no output."""
    a = synth.small_config(0, n_bins=3001)
    nob = synth.small_config(1, n_bins=5).with_freqs(np.zeros(0))
    nom = synth.small_config(2, n_bins=777).with_modes(np.zeros(0, np.int64))
    b = synth.small_config(3, n_bins=4096)
    wfs = [a, nob, nom, b]
    hp, hc = run(wfs, precision=prec)
    off = np.concatenate([[0], np.cumsum([w.n_freqs for w in wfs])])
    assert hp.shape[0] == off[-1]
    for i, w in enumerate(wfs):
        if w.n_freqs == 0:
            continue
        sp, sc = run(w, precision=prec)
        assert np.array_equal(hp[off[i]:off[i + 1]], sp) and np.array_equal(hc[off[i]:off[i + 1]], sc)
    assert np.all(hp[off[2]:off[3]] == 0) and np.all(hc[off[2]:off[3]] == 0)


def test_mixed_precision_small(oracle):
    w = synth.small_config(0)
    _cmp(run(w, precision="mixed"), oracle.sum_modes(w), TOL32)


def test_mixed_precision_paper_sampled(oracle):
    w = synth.paper_config(4)
    hp, hc = run(w, precision="mixed", tile_bins=BENCH_TILE["mixed"])
    rng = np.random.default_rng(4)
    occupied = np.nonzero(np.abs(hp) > 0)[0]
    sel = np.unique(rng.choice(occupied, 3000, replace=False))
    rp, rc = oracle.sum_modes(w, freqs=w.freqs[sel])
    for g, r in zip((hp[sel], hc[sel]), (rp, rc)):
        assert rel_l2(g, r) <= TOL32


def test_graph_replay_equals_direct_call():
    from tests.gpu_util import plan_for
    wfs = [synth.small_config(0, n_bins=3001), synth.paper_config(3, n_modes=150, T_years=0.5, grid="sparse", n_sparse=2000)]
    plan = plan_for(wfs)
    b = plan.upload(synth.concat(wfs))
    direct = [x.clone() for x in plan.sum_modes(b)]
    out = (torch.zeros_like(direct[0]), torch.zeros_like(direct[1]))
    g = plan.capture(b, out)
    for _ in range(2):
        out[0].zero_()
        out[1].zero_()
        g.replay()
        plan.sync()
        assert torch.equal(out[0], direct[0]) and torch.equal(out[1], direct[1])
    # the graph reads the input buffers at every replay
    b["amp"].mul_(2.0)
    g.replay()
    plan.sync()
    assert torch.allclose(out[0], 2 * direct[0], rtol=1e-13, atol=0)
    g.close()
    plan.close()


def test_autotuner(tmp_path, monkeypatch):
    from paper_2307_12585_gb300 import autotune
    from tests.gpu_util import plan_for
    monkeypatch.setenv("EMRI_FD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    w = synth.small_config(0, n_bins=20000)
    plan = plan_for([w])
    b = plan.upload(synth.concat([w]))
    out = plan.sum_modes(b)
    r1 = autotune.tune(plan, b, out)
    assert r1["tile_bins"] in (32, 64, 128) and not r1["cached"]
    # 20000 bins are few tiles: the split candidates were timed too
    assert "32x4" in r1["ms"] and r1["tile_split"] in (1, 2, 4)
    r2 = autotune.tune(plan, b, out)
    assert r2["cached"] and r2["tile_bins"] == r1["tile_bins"] and r2["tile_split"] == r1["tile_split"]
    # the tuned plan still matches the oracle's result within the FP64 bar
    got = tuple(x.cpu().numpy() for x in plan.sum_modes(b))
    ref = run(w)
    for x, y in zip(got, ref):
        assert rel_l2(x, y) < 1e-14
    plan.close()



@pytest.mark.parametrize("prec", PRECS)
def test_long_trajectory_and_high_l(oracle, prec):
    """1000 knots (every lane of the spline scans carries about 31 rows) and modes up
    to l = 20, the largest the library accepts, with partners, on a ragged grid."""
    T = 1.0 * synth.YEAR_S
    t, pp, pr, op, orr = synth.trajectory(T, 1000)
    l = np.array([2, 5, 9, 14, 20, 20, 17, 20], np.int32)
    m = np.array([2, 3, 9, 1, 20, 7, 0, 13], np.int32)
    n = np.array([0, -2, 4, 1, 0, -3, 2, 5], np.int32)
    A = synth.amplitudes(np.random.default_rng(11), t, l, m, n, 1.0)
    f = np.sort(np.random.default_rng(12).uniform(1e-4, 1.2e-2, 7777))
    w = synth.Waveform(t, pp, pr, op, orr, l, m, n, A, 0.9, 0.3, 1.0, f)
    _cmp(run(w, precision=prec), oracle.sum_modes(w), TOL64)


@pytest.mark.parametrize("prec", PRECS)
def test_many_nonuniform_knots(oracle, prec):
    """Linear chirp and quadratic voice on 1000 and 700 random knots (no partners)."""
    for w, p in (AN.linear_chirp(K=1000, seed=5), AN.quadratic_voice(K=700, seed=6)):
        got = run(w, conj=False, precision=prec)
        ref = oracle.sum_modes(w, conj_partners=False)
        # bins within 1e-6 of a turnover frequency are ill-conditioned (|H| ~ |f - F*|^(-1/4))
        far = np.abs(w.freqs - p.get("Fs", -1.0)) > 1e-6 * p.get("Fs", 0.0)
        for g, r in zip(got, ref):
            assert rel_l2(g[far], r[far]) <= TOL64
        assert np.array_equal(np.abs(got[0]) > 0, np.abs(ref[0]) > 0)
