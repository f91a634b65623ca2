"""Checkpoint / resume and the run log, host logic on a CPU stand-in for the
engine (its run adds a fixed integer pattern per photon index, as the real
tallies are integer sums over photons), and the argument checks of the
watchdog and bounded-wait entry points (no GPU needed)."""
import ctypes as C
import json

import numpy as np
import pytest


class FakeEngine:
    def __init__(self, gpu):
        import torch
        self.camera, self.geometry = gpu.Camera(16, 8, 4), gpu.Geometry()
        self.image = torch.zeros((8, 16), dtype=torch.int64)
        self.radial = torch.zeros(4, dtype=torch.int64)
        self.totals = torch.zeros(8, dtype=torch.int64)
        self.error = torch.zeros(1, dtype=torch.int32)
        self.image_frac_bits = 32
        self.calls = []

    def run(self, medium, n, seed=1, photon_offset=0, accumulate=False, stream=None, **kw):
        import torch
        assert accumulate
        p = np.arange(photon_offset, photon_offset + n, dtype=np.int64)
        h = (p * 2654435761 + seed) % 1000003
        self.image += torch.from_numpy(np.bincount(h % 128, weights=h, minlength=128).astype(np.int64)).view(8, 16)
        self.radial += torch.from_numpy(np.bincount(h % 4, minlength=4).astype(np.int64))
        self.totals[7] += int(n) * 3
        self.totals[1] += int(h.sum())
        self.calls.append((photon_offset, n))

    def check(self, stream=None):
        pass

    def result(self):
        return dict(raw_image=self.image.numpy().copy(), raw_totals=self.totals.numpy().copy(),
                    radial=self.radial.numpy().copy(),
                    image=self.image.numpy().astype(np.float64) * 2.0 ** -self.image_frac_bits)


@pytest.fixture
def gpu_mod():
    import paper_2507_23189_gb300 as gpu
    return gpu


def test_resume_equals_one_run(gpu_mod, tmp_path):
    from paper_2507_23189_gb300.checkpoint import run_resumable
    med = gpu_mod.Medium(0.1, 0.0, "hg", 0.8, None)
    ref = FakeEngine(gpu_mod)
    ref.run(med, 10_000, seed=3, accumulate=True)
    e = FakeEngine(gpu_mod)
    path = str(tmp_path / "ck.npz")
    log = str(tmp_path / "run.jsonl")
    r = run_resumable(e, med, 10_000, path, chunk=3000, seed=3, stop_after=2, log=log)
    assert r["photons_done"] == 6000 and e.calls == [(0, 3000), (3000, 3000)]
    e2 = FakeEngine(gpu_mod)                      # a new process: state only from the file
    r2 = run_resumable(e2, med, 10_000, path, chunk=3000, seed=3, log=log)
    assert r2["photons_done"] == 10_000 and e2.calls == [(6000, 3000), (9000, 1000)]
    np.testing.assert_array_equal(r2["raw_image"], ref.image.numpy())
    np.testing.assert_array_equal(r2["raw_totals"], ref.totals.numpy())
    np.testing.assert_array_equal(r2["radial"], ref.radial.numpy())
    recs = [json.loads(line) for line in open(log)]
    assert [x["photons_done"] for x in recs] == [3000, 6000, 9000, 10_000]
    assert all(x["photon_steps"] == 3 * x["photons"] for x in recs)
    # a finished run resumes to nothing
    e3 = FakeEngine(gpu_mod)
    r3 = run_resumable(e3, med, 10_000, path, chunk=3000, seed=3)
    assert e3.calls == [] and r3["photons_done"] == 10_000


def test_checkpoint_of_another_configuration_is_refused(gpu_mod, tmp_path):
    from paper_2507_23189_gb300.checkpoint import run_resumable
    med = gpu_mod.Medium(0.1, 0.0, "hg", 0.8, None)
    path = str(tmp_path / "ck.npz")
    run_resumable(FakeEngine(gpu_mod), med, 5000, path, chunk=2000, seed=1, stop_after=1)
    for kw in (dict(seed=2), dict(seed=1, rr_threshold=1e-3)):
        with pytest.raises(ValueError):
            run_resumable(FakeEngine(gpu_mod), med, 5000, path, chunk=2000, **kw)
    with pytest.raises(ValueError):
        run_resumable(FakeEngine(gpu_mod), gpu_mod.Medium(0.2, 0.0, "hg", 0.8, None), 5000, path, chunk=2000)
    with pytest.raises(ValueError):
        run_resumable(FakeEngine(gpu_mod), med, 5000, str(tmp_path / "x.npz"), photon_offset=5)


def test_watchdog_and_selftest_reject_bad_arguments(gpu_mod):
    from paper_2507_23189_gb300 import _native as N
    L = N.lib()
    err = (C.c_uint32 * 4)()
    assert L.mc_check_within(None, None, 1.0) == -1
    assert L.mc_check_within(C.cast(err, C.c_void_p), None, -1.0) == -1
    assert L.mc_check_within(C.cast(err, C.c_void_p), None, float("nan")) == -1
    assert L.mc_wait_selftest(None, 10, None) == -1
    assert L.mc_wait_selftest(C.cast(err, C.c_void_p), 0, None) == -1
    assert L.mc_wait_selftest(C.cast(err, C.c_void_p), (1 << 22) + 1, None) == -1
    assert L.mc_status_string(1) == b"work still running"


def test_image_sigma_is_the_batch_means_error(gpu_mod, tmp_path):
    """Equal chunks: sigma(image) = n sqrt(k) * sample std of the chunks'
    per-photon images, computed here from the chunk images directly."""
    from paper_2507_23189_gb300.checkpoint import run_resumable
    med = gpu_mod.Medium(0.1, 0.0, "hg", 0.8, None)
    n, k = 2500, 4
    e = FakeEngine(gpu_mod)
    r = run_resumable(e, med, n * k, str(tmp_path / "s.npz"), chunk=n, seed=5)
    chunks = []
    for c in range(k):
        f = FakeEngine(gpu_mod)
        f.run(med, n, seed=5, photon_offset=c * n, accumulate=True)
        chunks.append(f.image.numpy().astype(np.float64) * 2.0 ** -32 / n)
    chunks = np.stack(chunks)
    want = n * np.sqrt(k) * chunks.std(axis=0, ddof=1)
    np.testing.assert_allclose(r["image_sigma"], want, rtol=1e-9, atol=1e-12 * want.max())
    # resumed after two chunks: the same errors
    p2 = str(tmp_path / "s2.npz")
    run_resumable(FakeEngine(gpu_mod), med, n * k, p2, chunk=n, seed=5, stop_after=2)
    r2 = run_resumable(FakeEngine(gpu_mod), med, n * k, p2, chunk=n, seed=5)
    np.testing.assert_allclose(r2["image_sigma"], r["image_sigma"], rtol=1e-12)
    one = run_resumable(FakeEngine(gpu_mod), med, n, str(tmp_path / "one.npz"), chunk=n, seed=5)
    assert one["image_sigma"] is None



def test_run_record_logs_the_word_the_last_check_read(gpu_mod):
    """The record's error field is the word Engine.check() read before it
    cleared it (not the cleared device word)."""
    from paper_2507_23189_gb300.checkpoint import run_record
    med = gpu_mod.Medium(0.1, 0.0, "hg", 0.8, None)
    e = FakeEngine(gpu_mod)
    e.run(med, 100, accumulate=True)
    assert run_record(e, med, 100, 1.0)["error"] == 0
    e.last_error = 0x1          # MC_EFLAG_EVENTS seen by the last check
    assert run_record(e, med, 100, 1.0)["error"] == 1
