"""Host logic of the tile-shape autotuner, on the CPU: a fake plan (which refuses a
tile split with 128-bin tiles, as the library does) and fake CUDA events on a
synthetic clock stand in for the device.  Checks which candidates are timed, that
the fastest is applied, and the cache round trip."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2307_12585_gb300 import autotune


class FakePlan:
    def __init__(self, cost):
        self.device, self.precision, self.stream = 0, 0, None
        self.tile, self.split = 128, 1
        self.cost = cost          # (tile, split) -> ms per call
        self.clock = [0.0]
        self.calls = []

    def set_tile(self, tb):
        if self.split > 1 and tb == 128:
            raise ValueError("a tile split needs 32- or 64-bin tiles")
        self.tile = tb

    def set_tile_split(self, s):
        if s > 1 and self.tile == 128:
            raise ValueError("a tile split needs 32- or 64-bin tiles")
        self.split = s

    def sum_modes(self, b, out=None, check=True):
        self.calls.append((self.tile, self.split))
        self.clock[0] += self.cost[(self.tile, self.split)]

    def sync(self):
        pass


def _fake_cuda(monkeypatch, plan, n_sms=152):
    class Event:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = plan.clock[0]

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return other.t - self.t

    class Props:
        multi_processor_count = n_sms

    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda d=None: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d=None: Props())


def _batch(n_bins):
    return {"knot_off": np.array([0, 200]), "mode_off": np.array([0, 2000]), "freq_off": np.array([0, n_bins])}


COST = {(32, 1): 3.0, (64, 1): 2.0, (128, 1): 2.5, (32, 2): 1.5, (32, 4): 1.2, (64, 2): 1.8, (64, 4): 1.7}


def test_many_tiles_times_widths_only(monkeypatch, tmp_path):
    plan = FakePlan(COST)
    _fake_cuda(monkeypatch, plan)
    monkeypatch.setenv("EMRI_FD_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    r = autotune.tune(plan, _batch(3155760), None)      # 24,654 tiles of 128 bins: many per SM
    assert {c[1] for c in plan.calls} == {1}
    assert (r["tile_bins"], r["tile_split"], r["cached"]) == (64, 1, False)
    assert (plan.tile, plan.split) == (64, 1)
    assert set(r["ms"]) == {"32", "64", "128"} and r["ms"]["64"] == pytest.approx(2.0)


def test_few_tiles_also_times_splits(monkeypatch, tmp_path):
    plan = FakePlan(COST)
    _fake_cuda(monkeypatch, plan)
    monkeypatch.setenv("EMRI_FD_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    r = autotune.tune(plan, _batch(10000), None)        # 79 tiles of 128 bins: fewer than 4 per SM
    assert set(r["ms"]) == {"32", "64", "128", "32x2", "32x4", "64x2", "64x4"}
    assert (r["tile_bins"], r["tile_split"]) == (32, 4)
    assert (plan.tile, plan.split) == (32, 4)


def test_cache_round_trip(monkeypatch, tmp_path):
    plan = FakePlan(COST)
    _fake_cuda(monkeypatch, plan)
    monkeypatch.setenv("EMRI_FD_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    first = autotune.tune(plan, _batch(10000), None)
    plan2 = FakePlan(COST)
    plan2.clock = plan.clock
    _fake_cuda(monkeypatch, plan2)
    again = autotune.tune(plan2, _batch(10000), None)
    assert again["cached"] and not plan2.calls                   # nothing timed the second time
    assert (plan2.tile, plan2.split) == (first["tile_bins"], first["tile_split"]) == (32, 4)
    # another batch signature (more bins) is tuned afresh
    plan3 = FakePlan(COST)
    _fake_cuda(monkeypatch, plan3)
    assert not autotune.tune(plan3, _batch(3155760), None)["cached"] and plan3.calls


def test_no_cache(monkeypatch, tmp_path):
    plan = FakePlan(COST)
    _fake_cuda(monkeypatch, plan)
    path = tmp_path / "c.json"
    monkeypatch.setenv("EMRI_FD_AUTOTUNE_CACHE", str(path))
    autotune.tune(plan, _batch(10000), None, use_cache=False)
    assert not path.exists()
