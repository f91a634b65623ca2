"""Pins for the oracle's gradient with respect to the voxel densities.

* Scaling identity: multiplying every density by (1 + e) scales mu_s and the
  particles' absorption together, so sum_v n_v dL/dn_v must equal
  mu_s dL/dmu_s + mu_a,particles dL/dmu_a of the (separately pinned)
  homogeneous adjoint on the same photons, with and without absorption.
* Single scattering: the expected order-1 image is a closed-form function of
  the voxel densities along the beam row and the columns above it; its
  gradient by finite differences in numpy against the estimate, voxel by
  voxel, and exact zeros elsewhere.
* The value equals sum(adj * image) of the walk on the same photons.
"""
import math

import numpy as np
import pytest

LX, LY, LZ = 45.0, 10.0, 10.0


def _hg_sr(g, mu):
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


@pytest.mark.parametrize("absorb,mu_a0,beam", [(False, 0.0, 0.0), (True, 0.0, 0.0), (True, 0.004, 0.0),
                                               (True, 0.004, 2.0)])
def test_scaling_identity_against_homogeneous_adjoint(oracle_mod, absorb, mu_a0, beam):
    k_ext = 2e-5
    k_sca = 0.85 * k_ext if absorb else k_ext
    rho = 3.0 / LX / k_ext
    dens = np.full((8, 8, 16), rho)
    n, nx, nz = 4000, 16, 16
    adj = np.random.default_rng(2).uniform(0, 1, (nz, nx))
    common = dict(phase="hg", hg_g=0.8, n_photons=n, nx=nx, nz=nz, seed=5, rr_threshold=1e-2, beam_radius=beam)
    g = oracle_mod.grid_adjoint(adj, mu_s=0.0, mu_a=mu_a0,
                                grid=dict(density=dens, k_ext=k_ext, k_sca=k_sca, block=(4, 2, 2)), **common)
    mu_s, mu_ap = k_sca * rho, (k_ext - k_sca) * rho
    h = oracle_mod.adjoint(adj, 0, mu_s=mu_s, mu_a=mu_ap + mu_a0, **common)
    want = mu_s * h["grad"][0] + mu_ap * h["grad"][1]
    assert g["value"] == pytest.approx(h["value"], rel=1e-10)
    assert float(np.sum(rho * g["grad"])) == pytest.approx(want, rel=1e-8, abs=1e-10 * abs(h["value"]))


def test_single_scatter_gradient_closed_form(oracle_mod):
    rng = np.random.default_rng(7)
    shape = (16, 16, 32)
    dens = 2000.0 * np.exp(0.5 * rng.standard_normal(shape))
    k_ext, k_sca, g = 4e-5, 3e-5, 0.6
    nx, nz = 32, 16
    adj = np.zeros((nz, nx))
    adj[nz // 2] = rng.uniform(0.2, 1.0, nx)
    dx, vy = LX / 32, LY / 16

    def expected(d):
        mu_row = k_ext * d[8, 8, :]
        before = np.concatenate([[0.0], np.cumsum(mu_row * dx)])[:-1]
        p_col = np.exp(-before) * (1 - np.exp(-mu_row * dx))
        od = np.sum(k_ext * d[8, 8:, :], axis=0) * vy
        return float(np.sum(adj[nz // 2] * p_col * (k_sca / k_ext) * _hg_sr(g, 0.0) * np.exp(-od)))

    # closed-form gradient (per photon) by central differences
    want = np.zeros(shape)
    for iy in range(8, 16):
        for ix in range(32):
            e = np.zeros(shape)
            h = 1e-4 * dens[8, iy, ix]
            e[8, iy, ix] = h
            want[8, iy, ix] = (expected(dens + e) - expected(dens - e)) / (2 * h)
    n_b, batches = 40_000, 16
    grads = []
    val = 0.0
    for b in range(batches):
        r = oracle_mod.grid_adjoint(adj, phase="hg", hg_g=g, mu_s=0.0, n_photons=n_b, photon_offset=b * n_b,
                                    nx=nx, nz=nz, max_scatter=1, seed=3,
                                    grid=dict(density=dens, k_ext=k_ext, k_sca=k_sca, block=(8, 4, 4)))
        grads.append(r["grad"])
        val += r["value"]
    grads = np.stack(grads)
    n = n_b * batches
    est = grads.sum(axis=0) / n
    sig = grads.std(axis=0, ddof=1) * math.sqrt(batches) / n
    assert val / n == pytest.approx(expected(dens), rel=0.02)
    mask = np.zeros(shape, bool)
    mask[8, 8:, :] = True
    assert np.all(est[~mask] == 0.0)
    z = (est[mask] - want[mask]) / np.maximum(sig[mask], 1e-30)
    print("max |z| %.2f chi2/dof %.1f/%d" % (np.max(np.abs(z)), np.sum(z ** 2), z.size))
    assert np.max(np.abs(z)) < 5.0
    assert np.sum(z ** 2) < z.size + 6 * math.sqrt(2 * z.size)


@pytest.mark.parametrize("beam_radius", [0.0, 2.0])
def test_value_is_the_walk_functional(oracle_mod, beam_radius):
    rng = np.random.default_rng(9)
    dens = 1500.0 * np.exp(0.5 * rng.standard_normal((8, 8, 16)))
    adj = rng.uniform(0, 1, (16, 16))
    kw = dict(phase="hg", hg_g=0.7, mu_s=0.0, mu_a=0.001, n_photons=3000, nx=16, nz=16, seed=4,
              beam_radius=beam_radius, grid=dict(density=dens, k_ext=5e-5, k_sca=4e-5, block=(4, 2, 2)))
    r = oracle_mod.grid_adjoint(adj, **kw)
    w = oracle_mod.walk(**kw)
    assert r["value"] == pytest.approx(float(np.sum(adj * w["image"])), rel=1e-12)
    assert np.all(np.isfinite(r["grad"]))


# ---------------------------------------------------------------- null scores


def test_null_scores_single_scatter_closed_form(oracle_mod):
    """The null-collision estimator is unbiased: its single-scatter gradient
    agrees voxel by voxel, within its batch error, with finite differences of
    the closed-form expected image (the same expectation as above), on paths
    of the walk with majorants 1.3 times the cell maxima."""
    rng = np.random.default_rng(7)
    shape = (16, 16, 32)
    dens = 2000.0 * np.exp(0.5 * rng.standard_normal(shape))
    k_ext, k_sca, g = 4e-5, 3e-5, 0.6
    nx, nz = 32, 16
    adj = np.zeros((nz, nx))
    adj[nz // 2] = rng.uniform(0.2, 1.0, nx)
    dx, vy = LX / 32, LY / 16

    def expected(d):
        mu_row = k_ext * d[8, 8, :]
        before = np.concatenate([[0.0], np.cumsum(mu_row * dx)])[:-1]
        p_col = np.exp(-before) * (1 - np.exp(-mu_row * dx))
        od = np.sum(k_ext * d[8, 8:, :], axis=0) * vy
        return float(np.sum(adj[nz // 2] * p_col * (k_sca / k_ext) * _hg_sr(g, 0.0) * np.exp(-od)))

    want = np.zeros(shape)
    for iy in range(8, 16):
        for ix in range(32):
            e = np.zeros(shape)
            h = 1e-4 * dens[8, iy, ix]
            e[8, iy, ix] = h
            want[8, iy, ix] = (expected(dens + e) - expected(dens - e)) / (2 * h)
    n_b, batches = 40_000, 16
    grads, val = [], 0.0
    grid = dict(density=dens, k_ext=k_ext, k_sca=k_sca, block=(8, 4, 4), majorant_scale=1.3)
    for b in range(batches):
        r = oracle_mod.grid_adjoint(adj, nulls=True, max_events=256, phase="hg", hg_g=g, mu_s=0.0, n_photons=n_b,
                                    photon_offset=b * n_b, nx=nx, nz=nz, max_scatter=1, seed=3, grid=grid)
        grads.append(r["grad"])
        val += r["value"]
    grads = np.stack(grads)
    n = n_b * batches
    est = grads.sum(axis=0) / n
    sig = grads.std(axis=0, ddof=1) * math.sqrt(batches) / n
    assert val / n == pytest.approx(expected(dens), rel=0.02)
    mask = np.zeros(shape, bool)
    mask[8, 8:, :] = True
    assert np.all(est[~mask] == 0.0)
    z = (est[mask] - want[mask]) / np.maximum(sig[mask], 1e-30)
    print("nulls: max |z| %.2f chi2/dof %.1f/%d" % (np.max(np.abs(z)), np.sum(z ** 2), z.size))
    assert np.max(np.abs(z)) < 5.0
    assert np.sum(z ** 2) < z.size + 6 * math.sqrt(2 * z.size)


def test_null_scores_agree_with_exact_lengths_in_expectation(oracle_mod):
    """Multiple scattering: block sums of the null-score and the exact-length
    gradients agree within their combined batch errors (independent paths:
    the majorants differ), and the null version's value is the walk's
    functional with the same majorants."""
    rng = np.random.default_rng(12)
    shape = (8, 8, 16)
    dens = 1500.0 * np.exp(0.5 * rng.standard_normal(shape))
    k_ext, k_sca, mu_a = 5e-5, 4.5e-5, 0.002
    nx = nz = 16
    adj = rng.uniform(0, 1, (nz, nx))
    common = dict(phase="hg", hg_g=0.8, mu_s=0.0, mu_a=mu_a, nx=nx, nz=nz, rr_threshold=1e-2)
    blk = lambda t: t.reshape(2, 4, 2, 4, 4, 4).sum(axis=(1, 3, 5))
    n_b, batches = 20_000, 12
    out = {}
    for name, nulls, scale in (("exact", False, 1.0), ("nulls", True, 1.5)):
        grid = dict(density=dens, k_ext=k_ext, k_sca=k_sca, block=(4, 2, 2), majorant_scale=scale)
        bs = []
        for b in range(batches):
            r = oracle_mod.grid_adjoint(adj, nulls=nulls, max_events=2048, n_photons=n_b, photon_offset=b * n_b,
                                        seed=21, grid=grid, **common)
            bs.append(blk(r["grad"]))
        bs = np.stack(bs)
        out[name] = (bs.mean(axis=0), bs.std(axis=0, ddof=1) / math.sqrt(batches))
    (m0, s0), (m1, s1) = out["exact"], out["nulls"]
    z = (m1 - m0) / np.sqrt(s0 ** 2 + s1 ** 2)
    print("block sums: max |z| %.2f; null/exact batch error ratio median %.2f" %
          (np.max(np.abs(z)), np.median(s1 / s0)))
    assert np.max(np.abs(z)) < 4.0
    assert np.sum(z ** 2) < z.size + 6 * math.sqrt(2 * z.size)
    kw = dict(common, n_photons=3000, seed=4,
              grid=dict(density=dens, k_ext=k_ext, k_sca=k_sca, block=(4, 2, 2), majorant_scale=1.5))
    r = oracle_mod.grid_adjoint(adj, nulls=True, max_events=2048, **kw)
    w = oracle_mod.walk(**kw)
    assert r["value"] == pytest.approx(float(np.sum(adj * w["image"])), rel=1e-12)


def test_majorant_scale_leaves_the_walk_unbiased(oracle_mod):
    """Delta tracking against larger majorants samples the same transport:
    images at majorant scale 1 and 1.5 agree within their errors, and the
    larger majorant takes more tentative collisions."""
    rng = np.random.default_rng(13)
    dens = 1500.0 * np.exp(0.5 * rng.standard_normal((8, 8, 16)))
    base = dict(phase="hg", hg_g=0.8, mu_s=0.0, n_photons=200_000, nx=8, nz=8)
    r1 = oracle_mod.walk(seed=1, grid=dict(density=dens, k_ext=5e-5, k_sca=5e-5, block=(4, 2, 2)), **base)
    r2 = oracle_mod.walk(seed=2, grid=dict(density=dens, k_ext=5e-5, k_sca=5e-5, block=(4, 2, 2),
                                           majorant_scale=1.5), **base)
    var = lambda r: np.maximum(r["image_sq"] - r["image"] ** 2 / r["n_photons"], 0)
    z = (r1["image"] - r2["image"]) / np.sqrt(var(r1) + var(r2) + 1e-300)
    assert np.max(np.abs(z)) < 4.5
    assert r2["steps"] > 1.2 * r1["steps"]
