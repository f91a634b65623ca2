"""Pins for the oracle's heterogeneous medium (delta tracking on a voxel
density grid) and its phase-function mixture table.

Independent of the oracle's own arithmetic: the homogeneous walk (a constant
grid whose majorant equals mu_ext makes the same decisions with the same
random numbers), Beer-Lambert transmission through the voxel row the beam
follows, the single-scatter camera image from voxel sums in numpy, the
invariance of the result under the choice of majorant cells, the camera
transmittance from numpy column sums, and the closed-form H-G mixture CDF.
"""
import math

import numpy as np
import pytest

LX, LY, LZ = 45.0, 10.0, 10.0
M_PS = complex(1.59 / 1.33, 0.0)
X_PS = 39.26990816987241


def _hg_sr(g, mu):
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


def _random_grid(shape, seed, mean=2000.0, spread=0.6):
    rng = np.random.default_rng(seed)
    return mean * np.exp(spread * rng.standard_normal(shape))


@pytest.mark.parametrize("block", [(1, 1, 1), (8, 4, 4)])
@pytest.mark.parametrize("absorb", [False, True])
def test_constant_grid_equals_homogeneous_walk(oracle_mod, block, absorb):
    k_ext = 2e-5
    k_sca = 0.8 * k_ext if absorb else k_ext
    rho = 4.0 / LX / k_ext
    dens = np.full((16, 16, 32), rho)
    n = 20_000
    kw = dict(phase="hg", hg_g=0.85, n_photons=n, nx=32, nz=32, seed=9, rr_threshold=1e-2, n_trace=300,
              n_trace_events=24)
    a = oracle_mod.walk(mu_s=0.0, mu_a=0.0, grid=dict(density=dens, k_ext=k_ext, k_sca=k_sca, block=block),
                        **kw)
    b = oracle_mod.walk(mu_s=k_sca * rho, mu_a=(k_ext - k_sca) * rho, **kw)
    np.testing.assert_allclose(a["image"], b["image"], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(a["totals"], b["totals"], rtol=1e-9, atol=1e-12)
    assert a["steps"] == b["steps"]
    # every recorded quantity but the decision margin (column 12)
    np.testing.assert_allclose(a["trace"][..., :12], b["trace"][..., :12], rtol=1e-9, atol=1e-10)


@pytest.fixture(scope="module")
def rough_grid():
    return _random_grid((16, 16, 64), 4)


def test_ballistic_transmission_through_the_beam_row(oracle_mod, rough_grid):
    k = 4e-5
    n = 400_000
    r = oracle_mod.walk(mu_s=0.0, phase="hg", hg_g=0.5, n_photons=n, nx=8, nz=8, max_scatter=1,
                        grid=dict(density=rough_grid, k_ext=k, k_sca=k, block=(4, 4, 4)))
    # the pencil beam runs along y = z = 0, the lower face of voxel row 8
    tau = np.sum(k * rough_grid[8, 8, :]) * LX / 64
    p = math.exp(-tau)
    got = r["totals"][6] / n
    assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / n)
    assert r["steps"] > n * (1 + 0.5 * (1 - p))     # null collisions happened


def test_single_scatter_camera_image(oracle_mod, rough_grid):
    """First collisions lie on the beam row; the camera term of a collision in
    voxel column ix is a p_sr(0) exp(-sum of mu dy over voxels 8.. of that
    column), whatever x inside the voxel."""
    k_ext, k_sca, g = 4e-5, 3e-5, 0.7
    n, nx, nz = 400_000, 64, 16
    grid = rough_grid
    r = oracle_mod.walk(mu_s=0.0, phase="hg", hg_g=g, n_photons=n, nx=nx, nz=nz, max_scatter=1,
                        grid=dict(density=grid, k_ext=k_ext, k_sca=k_sca, block=(8, 2, 2)))
    img = r["image"]
    assert np.count_nonzero(np.delete(img, nz // 2, axis=0)) == 0
    mu_row = k_ext * grid[8, 8, :]
    dx = LX / 64
    before = np.concatenate([[0.0], np.cumsum(mu_row * dx)])[:-1]
    p_col = np.exp(-before) * (1 - np.exp(-mu_row * dx))
    od_cam = np.sum(k_ext * grid[8, 8:, :], axis=0) * (LY / 16)
    c = (k_sca / k_ext) * _hg_sr(g, 0.0) * np.exp(-od_cam)
    want = n * p_col * c
    sigma = c * np.sqrt(n * p_col * (1 - p_col))
    z = (img[nz // 2] - want) / sigma
    assert np.max(np.abs(z)) < 5.0
    assert float(np.sum(z ** 2)) < nx + 6 * math.sqrt(2 * nx)


def test_majorant_cells_do_not_bias(oracle_mod, rough_grid):
    n = 300_000
    # roulette active: its survival draw must stay uniform under null collisions
    kw = dict(mu_s=0.0, phase="hg", hg_g=0.8, n_photons=n, nx=16, nz=16, rr_threshold=0.3)
    runs = []
    for block, seed in (((1, 1, 1), 1), ((16, 16, 64), 2)):
        runs.append(oracle_mod.walk(seed=seed, grid=dict(density=rough_grid, k_ext=4e-5, k_sca=2.4e-5,
                                                          block=block), **kw))
    a, b = runs
    assert b["steps"] > 1.5 * a["steps"]        # one global majorant: many more nulls
    for k in range(5):
        va = a["totals_sq"][k] - a["totals"][k] ** 2 / n
        vb = b["totals_sq"][k] - b["totals"][k] ** 2 / n
        assert abs(a["totals"][k] - b["totals"][k]) < 4.5 * math.sqrt(va + vb) + 1e-9
    va = np.maximum(a["image_sq"] - a["image"] ** 2 / n, 0)
    vb = np.maximum(b["image_sq"] - b["image"] ** 2 / n, 0)
    ok = (a["image_hits"] >= 20) & (b["image_hits"] >= 20)
    z = (a["image"] - b["image"])[ok] / np.sqrt((va + vb)[ok])
    assert np.sum(z ** 2) < z.size + 5 * math.sqrt(2 * z.size)


def test_camera_transmittance_is_the_column_depth(oracle_mod, rough_grid):
    k_ext, k_sca, g = 4e-5, 4e-5, 0.6
    n, ev = 4000, 8
    r = oracle_mod.walk(mu_s=0.0, phase="hg", hg_g=g, n_photons=n, nx=16, nz=16, n_trace=n,
                        n_trace_events=ev, seed=3, grid=dict(density=rough_grid, k_ext=k_ext, k_sca=k_sca,
                                                             block=(4, 4, 4)))
    tr = r["trace"]
    vy = LY / 16
    checked = 0
    for p in range(n):
        d = np.array([1.0, 0.0, 0.0])
        for e in range(ev):
            rec = tr[p, e]
            if rec[0] != 0:
                break
            x, y, zc = rec[1:4]
            fx, fy, fz = x / LX * 64, (y + LY / 2) / LY * 16, (zc + LZ / 2) / LZ * 16
            if min(abs(fx - round(fx)), abs(fy - round(fy)), abs(fz - round(fz))) > 1e-9:
                ix, iy, iz = int(fx), int(fy), int(fz)
                col = k_ext * rough_grid[iz, :, ix]
                od = col[iy] * ((iy + 1) * vy - LY / 2 - y) + np.sum(col[iy + 1:]) * vy
                want = rec[7] * _hg_sr(g, d[1]) * math.exp(-od)
                assert rec[8] == pytest.approx(want, rel=1e-10)
                checked += 1
            d = rec[4:7]
    assert checked > 3000


def test_weight_is_conserved_with_absorption_and_roulette(oracle_mod, rough_grid):
    n = 50_000
    r = oracle_mod.walk(mu_s=0.0, mu_a=0.01, phase="hg", hg_g=0.8, n_photons=n, nx=16, nz=16,
                        rr_threshold=1e-2, grid=dict(density=rough_grid, k_ext=5e-5, k_sca=4e-5, block=(8, 4, 4)))
    t = r["totals"]
    assert t[0] + t[1] + t[2] + t[3] + t[4] + t[5] == pytest.approx(n, rel=1e-10)
    assert t[4] != 0.0 and t[3] > 0.0


def test_grid_rejects_bad_arguments(oracle_mod, rough_grid):
    bad = rough_grid.copy()
    bad[0, 0, 0] = -1.0
    with pytest.raises(ValueError):
        oracle_mod.walk(mu_s=0.0, phase="hg", hg_g=0.5, grid=dict(density=bad, k_ext=1e-5, k_sca=1e-5))
    with pytest.raises(ValueError):
        oracle_mod.walk(mu_s=0.0, phase="hg", hg_g=0.5, grid=dict(density=rough_grid, k_ext=1e-5, k_sca=2e-5))


# ---------------------------------------------------------------- mixture


def _hg_cdf_mu(g, mu):
    return (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))


def test_hg_mixture_table_closed_form(oracle_mod):
    comps = [("hg", 0.9), ("hg", 0.3), ("hg", -0.4)]
    w = np.array([0.5, 0.3, 0.2])
    t = oracle_mod.phase_table_mixture(comps, w * 7.0)        # weights need not sum to 1
    levels = np.arange(4097) / 4096
    F = sum(wi * _hg_cdf_mu(g, t["icdf"]) for (_, g), wi in zip(comps, w))
    np.testing.assert_allclose(F, levels, rtol=0, atol=2e-9)
    assert t["mean"] == pytest.approx(float(np.dot(w, [0.9, 0.3, -0.4])), abs=1e-6)


def test_mixture_of_identical_components_is_the_component(oracle_mod):
    single = oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, X_PS, n_bins=1024, n_fine=1 << 16)
    mix = oracle_mod.phase_table_mixture([("mie", M_PS, X_PS), ("mie", M_PS, X_PS)], [2.0, 5.0],
                                         n_bins=1024, n_fine=1 << 16)
    np.testing.assert_allclose(mix["icdf"], single["icdf"], rtol=0, atol=1e-12)
    zero = oracle_mod.phase_table_mixture([("mie", M_PS, X_PS), ("hg", 0.5)], [1.0, 0.0], n_bins=1024,
                                          n_fine=1 << 16)
    np.testing.assert_allclose(zero["icdf"], single["icdf"], rtol=0, atol=1e-12)


def test_mie_mixture_is_the_weighted_sum_of_component_cdfs(oracle_mod):
    """Components with different raw normalisations (x^2 Q_sca / 2): the
    mixture's levels satisfy sum_i w_i F_i(icdf) = level with each F_i read
    from that component's own (separately pinned) table."""
    xs, w = (10.0, X_PS), np.array([0.3, 0.7])
    kw = dict(n_bins=4096, n_fine=1 << 17)
    mix = oracle_mod.phase_table_mixture([("mie", M_PS, x) for x in xs], w, **kw)
    levels = np.arange(4097) / 4096
    F = 0.0
    fine = np.arange((1 << 16) + 1) / (1 << 16)     # fine component tables: small interpolation error
    for wi, x in zip(w, xs):
        t = oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, x, n_bins=1 << 16, n_fine=1 << 18)
        F = F + wi * np.interp(mix["icdf"], t["icdf"], fine)
    np.testing.assert_allclose(F, levels, rtol=0, atol=2e-5)
