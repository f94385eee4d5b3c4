"""Parity at the benchmark workloads' full sizes, through the C ABI.

- The 2 yr, 2000-mode waveform of seed 1: every one of its 3,155,760 bins
  against the oracle (FP64 and FP64X at 1e-10, mixed at 1e-5, per channel),
  in the launch configuration the benchmark times.
- Seeds 3-16 of the same recipe: about 1.2e4 sampled bins each (1e4 of them
  occupied), FP64 and FP64X.
- The 64-waveform mixed-precision batch (seeds 1-64, one call): every member
  against the oracle on sampled bins, relative L2 <= 1e-5 per channel and the
  mismatch of Eq. 12 over those bins.
- The 256-waveform batch (N_m ~ U{50..3000}, T ~ U(0.5, 4) yr, N_f log-uniform
  in [1e4, 6e6]) in one graph-replayed FP64 call with autotuned tiles: 32
  members against the oracle on sampled bins.
Bins are independent, so a sampled bin is checked exactly as in a full run."""
import numpy as np
import pytest

from paper_2307_12585_gb300 import synth
from tests.gpu_util import plan_for, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL64 = 1e-10
TOL32 = 1e-5
BENCH_TILE = {"fp64": 128, "fp64x": 64, "mixed": 64}   # the tile sizes bench.py times each form at


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
        assert np.array_equal(np.abs(g) > 0, np.abs(r) > 0)   # the same bins are covered


def _run_device(wfs, prec, tile_bins=0):
    plan = plan_for(wfs, precision=prec, tile_bins=tile_bins)
    b = plan.upload(synth.concat(wfs))
    out = plan.sum_modes(b)
    plan.close()
    return out


@pytest.fixture(scope="module")
def seed1(oracle):
    w = synth.paper_config(1)
    return w, oracle.sum_modes(w)          # the whole grid, on every host core


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp64x", TOL64), ("mixed", TOL32)])
def test_paper_seed1_every_bin(seed1, prec, tol):
    w, ref = seed1
    hp, hc = _run_device([w], prec, BENCH_TILE[prec])
    got = tuple(x.cpu().numpy().astype(np.complex128) for x in (hp, hc))
    _cmp(got, ref, tol)


@pytest.mark.parametrize("seed", list(range(3, 17)))
def test_paper_seeds_sampled(oracle, seed):
    w = synth.paper_config(seed)
    outs = {p: _run_device([w], p, BENCH_TILE[p]) for p in ("fp64", "fp64x")}
    rng = np.random.default_rng(1000 + seed)
    occupied = torch.nonzero(outs["fp64"][0].abs() > 0).flatten().cpu().numpy()
    sel = np.unique(np.concatenate([rng.choice(w.n_freqs, 2000, replace=False),
                                    rng.choice(occupied, min(10000, occupied.size), replace=False)]))
    ref = oracle.sum_modes(w, freqs=w.freqs[sel])
    idx = torch.as_tensor(sel, device="cuda")
    for p, (hp, hc) in outs.items():
        _cmp((hp[idx].cpu().numpy(), hc[idx].cpu().numpy()), ref, TOL64)


def test_mixed_batch_64_members_against_oracle(oracle):
    """64 paper-shaped waveforms in one mixed-precision call (the benchmark's batch):
    each member against the FP64 oracle on 1800 sampled bins (1500 occupied)."""
    wfs = synth.paper_configs(range(1, 65))
    hp, hc = _run_device(wfs, "mixed", 64)
    off = np.concatenate([[0], np.cumsum([w.n_freqs for w in wfs])])
    rng = np.random.default_rng(64)
    errs, mms = [], []
    for i, w in enumerate(wfs):
        lo = int(off[i])
        occ = torch.nonzero(hp[lo:lo + w.n_freqs].abs() > 0).flatten().cpu().numpy()
        sel = np.unique(np.concatenate([rng.choice(w.n_freqs, 300, replace=False),
                                        rng.choice(occ, min(1500, occ.size), replace=False)]))
        idx = torch.as_tensor(sel + lo, device="cuda")
        got = tuple(x[idx].cpu().numpy().astype(np.complex128) for x in (hp, hc))
        ref = oracle.sum_modes(w, freqs=w.freqs[sel])
        _cmp(got, ref, TOL32)
        errs.append(max(rel_l2(g, r) for g, r in zip(got, ref)))
        mms.append(oracle.mismatch(ref, got))
    # rel. L2 e bounds the mismatch by about e^2/2 (Eq. 12 over the sampled bins)
    assert max(mms) <= 0.5 * max(errs) ** 2 * 1.01 + 1e-15, (max(mms), max(errs))
    assert max(errs) <= TOL32


def test_batch256_graph_sampled(oracle, tmp_path, monkeypatch):
    """The 256-waveform batch in one graph-replayed FP64 call at the tiles the autotuner
    picks (as the benchmark runs it): 32 members against the oracle on sampled bins."""
    from paper_2307_12585_gb300 import autotune
    monkeypatch.setenv("EMRI_FD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    wfs = synth.batch_config(256)
    plan = plan_for(wfs)
    b = plan.upload(synth.concat(wfs))
    out = plan.sum_modes(b)
    autotune.tune(plan, b, out, reps=1)
    g = plan.capture(b, out)
    out[0].zero_()
    out[1].zero_()
    g.replay()
    plan.sync()
    off = np.concatenate([[0], np.cumsum([w.n_freqs for w in wfs])])
    rng = np.random.default_rng(256)
    for i in rng.choice(len(wfs), 32, replace=False):
        w = wfs[i]
        sel = np.sort(rng.choice(w.n_freqs, min(300, w.n_freqs), replace=False))
        idx = torch.as_tensor(sel + int(off[i]), device="cuda")
        got = tuple(x[idx].cpu().numpy() for x in out)
        _cmp(got, oracle.sum_modes(w, freqs=w.freqs[sel]), TOL64)
    g.close()
    plan.close()
