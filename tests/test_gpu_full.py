"""The optical-depth sweep at full size: tau in {1, 2, 5, 10, 20}, Mie and
H-G, 1e8 photons, 256x256 image and 128-bin radial profile, in the launch
configuration the benchmark uses.

At this size the oracle cannot run every photon, so each case checks
  * properties that hold at any size (exact energy bookkeeping, Beer-Lambert),
  * bit-exact parity on a sampled photon range: the engine re-runs photons
    [k, k + m) on their own and the oracle runs the same range,
  * the full image against the oracle's estimate from that sample (3 sigma),
and reports the per-bin single-vs-double precision error for each tau.
"""
import math

import numpy as np
import pytest

from parity import oracle_var, tally_agreement

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5
N_FULL = 100_000_000
TAUS = [1.0, 2.0, 5.0, 10.0, 20.0]


@pytest.fixture(scope="module")
def g_or(oracle_mod):
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    return oracle_mod.mie_efficiencies(complex(1.59 / 1.33, 0.0), x)[2]


@pytest.mark.parametrize("phase", ["mie", "hg"])
@pytest.mark.parametrize("tau", TAUS)
def test_sweep_point(gpu, oracle_mod, ps_table, ps_oracle_table, g_or, tau, phase):
    mu_ext = tau / LX
    med = gpu.Medium(mu_ext, 0.0, "table" if phase == "mie" else "hg", ps_table.info["g"], ps_table)
    cam = gpu.Camera(256, 256, 128, R_MAX)
    eng = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    eng.run(med, N_FULL, seed=1)
    eng.check()
    full = eng.result()
    t = full["raw_totals"]
    assert t[0] + t[1] + t[2] == N_FULL << 32
    p = math.exp(-tau)
    assert abs(full["totals"][6] / N_FULL - p) < 5 * math.sqrt(p * (1 - p) / N_FULL)

    # sampled photons: [k, k + m) alone on both sides
    m = 200_000
    k = 37_000_000 + int(tau * 1000)
    eng.run(med, m, seed=1, photon_offset=k)
    eng.check()
    part = eng.result()
    om = dict(mu_s=mu_ext, phase="mie" if phase == "mie" else "hg", hg_g=g_or)
    ores = oracle_mod.walk(table=ps_oracle_table, n_photons=m, photon_offset=k, nx=256, nz=256,
                           n_radial=128, r_max=R_MAX, seed=1, **om)
    var = oracle_var(ores)
    zmax, chi2, dof, pv = tally_agreement(part["image"], ores["image"], 2 * var)
    assert zmax < 3.0 and pv > 0.01
    pop = ores["image"] > 0
    rel = np.abs(part["image"] - ores["image"])[pop] / ores["image"][pop]
    print("tau=%g %s steps/photon %.3f  fp32-vs-fp64 per-bin rel err median %.2e p99 %.2e max %.2e"
          % (tau, phase, full["steps"] / N_FULL, np.median(rel), np.quantile(rel, 0.99), rel.max()))
    assert abs(part["steps"] - ores["steps"]) <= 1e-3 * ores["steps"]
    np.testing.assert_allclose(part["radial"], ores["radial"], rtol=0,
                               atol=3 * math.sqrt(2) * math.sqrt(max(ores["radial_sq"].max(), 1.0)))

    # the whole run against the sample's estimate (scaled to N_FULL photons)
    scale = N_FULL / m
    zf, chi2f, doff, pf = tally_agreement(full["image"] / scale, ores["image"],
                                          var * (1 + m / N_FULL), min_rel_sigma=0.2)
    assert pf > 0.001 and doff > 100
    sps = full["steps"] / N_FULL
    assert abs(sps - ores["steps"] / m) < 0.05 * sps


def test_split_ranges_bit_identical(gpu, ps_table):
    med = gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table)
    cam = gpu.Camera(256, 256, 128, R_MAX)
    a = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    a.run(med, N_FULL, seed=1)
    b = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    b.run(med, 33_333_333, seed=1)
    b.run(med, N_FULL - 33_333_333, seed=1, photon_offset=33_333_333, accumulate=True)
    a.check()
    b.check()
    ra, rb = a.result(), b.result()
    np.testing.assert_array_equal(ra["raw_image"], rb["raw_image"])
    np.testing.assert_array_equal(ra["raw_totals"], rb["raw_totals"])
