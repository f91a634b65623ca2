"""The seeded synthetic inputs (paper_2507_23189_gb300/workloads.py) are what
the input recipe states: deterministic, in their stated ranges and shapes."""
import math

import numpy as np
import pytest

from paper_2507_23189_gb300 import workloads as W


def test_sweep_small_and_headline_cases():
    s = W.sweep()
    assert [(c.tau, c.phase) for c in s] == [(t, p) for t in (1.0, 2.0, 5.0, 10.0, 20.0) for p in ("mie", "hg")]
    assert all(c.n_photons == 100_000_000 and (c.nx, c.nz, c.n_radial) == (256, 256, 128) for c in s)
    assert [(c.tau, c.phase, c.n_photons, c.nx) for c in W.small()] == [(1.0, "mie", 1_000_000, 64),
                                                                       (1.0, "hg", 1_000_000, 64)]
    h = W.headline()
    assert (h.tau, h.phase, h.n_photons, h.nx, h.nz, h.seed) == (5.0, "mie", 100_000_000, 256, 256, 1)
    assert (W.RR_THRESHOLD, W.RR_SURVIVAL) == (1e-4, 0.1)


def test_batched_media_are_deterministic_and_in_range():
    a, b = W.batched(), W.batched()
    assert len(a) == 64 and [(c.tau, c.diameter_um, c.n_photons) for c in a] == \
        [(c.tau, c.diameter_um, c.n_photons) for c in b]
    d = np.array([c.diameter_um for c in a])
    tau = np.array([c.tau for c in a])
    n = np.array([c.n_photons for c in a])
    assert d.min() >= 1.0 and d.max() <= 10.0 and tau.min() >= 0.5 and tau.max() <= 20.0
    assert n.min() >= 1_000_000 and n.max() <= 100_000_000 and n.max() / n.min() > 10   # uneven budgets
    # log-uniform diameters: log10 d spreads over most of [0, 1]
    assert np.log10(d).min() < 0.15 and np.log10(d).max() > 0.85
    assert all((c.nx, c.nz) == (128, 128) for c in a)
    assert [c.tau for c in W.batched(seed=7)] != [c.tau for c in a]
    assert [c.tau for c in W.batched_draw()] == pytest.approx([c.tau for c in a], rel=1e-14)


def test_batched_media_are_the_record_and_a_fresh_draw_agrees():
    """The default batched media are the committed record; a fresh draw from
    the recipe gives the same names and photon budgets and the same
    diameters and optical depths up to the last bits of numpy's exp and log,
    which differ between platforms."""
    import json
    with open(W.BATCHED_RECORD) as f:
        rec = json.load(f)
    cases = W.batched()
    assert [(c.name, c.diameter_um, c.tau, c.n_photons) for c in cases] == \
        [(m["name"], m["diameter_um"], m["tau"], m["n_photons"]) for m in rec["media"]]
    assert all((c.nx, c.nz, c.seed, c.phase) == (128, 128, 1, "mie") for c in cases)
    fresh = W.batched_draw()
    assert [(c.name, c.n_photons) for c in fresh] == [(c.name, c.n_photons) for c in cases]
    for a, b in zip(fresh, cases):
        assert a.diameter_um == pytest.approx(b.diameter_um, rel=1e-14)
        assert a.tau == pytest.approx(b.tau, rel=1e-14)


def test_size_bins_are_log_normal_quantile_centres():
    from scipy.stats import norm
    d, f = W.size_bins(5.0, 0.3, 16)
    assert f.sum() == pytest.approx(1.0) and np.all(f == f[0])
    q = norm.cdf(np.log(d / 5.0) / 0.3)
    np.testing.assert_allclose(q, (np.arange(16) + 0.5) / 16, rtol=0, atol=1e-12)
    assert np.all(np.diff(d) > 0)
    assert math.sqrt(d[7] * d[8]) == pytest.approx(5.0, rel=1e-12)     # symmetric about the median


def test_plume_is_the_stated_gaussian():
    shape = (32, 32, 64)
    p = W.plume_shape(shape)
    assert p.dtype == np.float32 and p.shape == shape
    gz, gy, gx = shape
    np.testing.assert_array_equal(p, p[::-1, :, :])        # mirror symmetric in z
    np.testing.assert_array_equal(p, p[:, ::-1, :])        # and in y
    # along the beam: peak at x = 22.5 mm, value exp(-1/2) one sigma (5 mm) away
    x = (np.arange(gx) + 0.5) * 45.0 / gx
    row = p[gz // 2, gy // 2, :].astype(np.float64)
    yz = math.exp(-0.5 * ((0.5 * 10.0 / gz) / 5.0) ** 2) ** 2        # voxel centres just off the axis
    np.testing.assert_allclose(row, yz * np.exp(-0.5 * ((x - 22.5) / 5.0) ** 2), rtol=1e-6)
    P = W.plume()
    assert (P.shape, P.tau_peak, P.n_size_bins, P.n_photons, P.nx, P.nz) == ((256, 256, 256), 30.0, 16,
                                                                             1_000_000_000, 512, 512)


def test_rough_grid_is_seeded_log_normal():
    a = W.rough_grid((16, 16, 64), 4, mean=2000.0)
    np.testing.assert_array_equal(a, W.rough_grid((16, 16, 64), 4, mean=2000.0))
    assert not np.array_equal(a, W.rough_grid((16, 16, 64), 5, mean=2000.0))
    z = np.log(a.astype(np.float64) / 2000.0) / 0.6
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1.0) < 0.05 and np.all(a > 0)
