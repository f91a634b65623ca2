"""The batched launch's autotuner, host logic on CPU: a stand-in batch whose
'launches' take a known time per (threads per CTA, photons per warp chunk)
pair, and a stand-in for the CUDA timing calls. It must pick the fastest
launchable pair, skip pairs that cannot launch, and cache the choice under a
key of the GPU and the configuration."""
import types

import pytest


class _Clock:
    now = 0.0


class _Event:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = _Clock.now

    def synchronize(self):
        pass

    def elapsed_time(self, end):
        return end.t - self.t


def _cost(block, item):
    # fastest at 512 threads and warp chunks of 128 photons
    return 1.0 + abs(block - 512) / 256.0 + abs(item.bit_length() - 8) * 0.25


class _FakeBatch:
    runs = []

    def __init__(self, n, camera, geometry, device):
        self.n, self.camera, self.geometry, self.device = n, camera, geometry, device

    def run(self, media, n_photons, seeds, offsets, item_photons=0, block_size=0):
        if block_size == 256 and item_photons == 32:
            raise RuntimeError("not launchable")
        _FakeBatch.runs.append((block_size, item_photons, tuple(n_photons)))
        _Clock.now += _cost(block_size, item_photons)


@pytest.fixture
def tuner(monkeypatch, tmp_path):
    import torch
    import paper_2507_23189_gb300.autotune as A
    import paper_2507_23189_gb300.engine as E
    monkeypatch.setenv(A.CACHE_ENV, str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "Fake GB300")
    monkeypatch.setattr(torch.cuda, "synchronize", lambda dev=None: None)
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(E, "Batch", _FakeBatch)
    _FakeBatch.runs = []
    return A


def _setup(gpu):
    table = types.SimpleNamespace(params=dict(diameter_um=5.0))
    media = [gpu.Medium(0.1, 0.0, "table", 0.0, table), gpu.Medium(0.3, 0.01, "hg", 0.7, None)]
    batch = _FakeBatch(2, gpu.Camera(128, 128), gpu.Geometry(), "cuda:0")
    return batch, media, [800_000, 2_000_000]


def test_picks_the_fastest_launchable_shape_and_caches_it(tuner):
    import paper_2507_23189_gb300 as gpu
    batch, media, n = _setup(gpu)
    r = tuner.tune_batch(batch, media, n, scale=8, reps=2)
    assert r["cached"] is False
    assert r["block_size"] == 512 and r["item_photons"] == 128
    assert r["ms"] == pytest.approx(_cost(512, 128))
    # every launchable pair ran on the scaled budgets (1 untimed + reps timed), the unlaunchable one never
    shapes = {(b, i) for b, i, _ in _FakeBatch.runs}
    assert (256, 32) not in shapes
    assert len(shapes) == len(tuner.BLOCKS) * len(tuner.ITEMS) - 1
    assert all(p == (100_000, 250_000) for _, _, p in _FakeBatch.runs)
    # the same configuration comes from the cache without running anything
    _FakeBatch.runs = []
    again = tuner.tune_batch(batch, media, n, scale=8, reps=2)
    assert again["cached"] is True and again["block_size"] == 512 and _FakeBatch.runs == []
    # another configuration is tuned afresh
    other = tuner.tune_batch(batch, media, [800_000, 2_000_001], scale=8, reps=2)
    assert other["cached"] is False and _FakeBatch.runs


def test_no_launchable_shape_raises(tuner, monkeypatch):
    import paper_2507_23189_gb300 as gpu
    batch, media, n = _setup(gpu)

    def never(self, *a, **k):
        raise RuntimeError("not launchable")
    monkeypatch.setattr(_FakeBatch, "run", never)
    with pytest.raises(RuntimeError):
        tuner.tune_batch(batch, media, n, use_cache=False)
