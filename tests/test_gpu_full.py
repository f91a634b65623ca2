"""The optical-depth sweep at full size: tau in {1, 2, 5, 10, 20}, Mie and
H-G, 1e8 photons, 256x256 image and 128-bin radial profile, in the launch
configuration the benchmark uses.

Each case checks
  * properties that hold at any size (exact energy bookkeeping, Beer-Lambert),
  * the one-launch result against the same photons run as 32 launches
    (bit-identical integer sums; the batches also give the engine's variance),
  * every image bin against the threaded oracle on all 1e8 photons with the
    same seed (within 3 sigma, pooled chi-square p > 0.01 over bins with at
    least 20 contributions), the radial profile and the step count,
  * a sampled photon range [k, k + m) run on its own by both sides,
and reports the per-bin single-vs-double precision error for each tau.
"""
import math

import numpy as np
import pytest

from parity import gpu_batches, oracle_var, tally_agreement

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
    geo = gpu.Geometry(LX, LY, LZ)
    eng = gpu.Engine(cam, geo)
    eng.run(med, N_FULL, seed=1)        # one launch, as the benchmark runs it
    eng.check()
    full = eng.result()
    t = full["raw_totals"]
    assert t[0] + t[1] + t[2] == N_FULL << 32
    p = math.exp(-tau)
    assert abs(full["totals"][6] / N_FULL - p) < 5 * math.sqrt(p * (1 - p) / N_FULL)

    # the same photons as 32 launches: bit-identical sums, and a batch variance
    bat = gpu_batches(gpu, med, N_FULL, 32, cam, geo, seed=1)
    np.testing.assert_array_equal(bat["raw_image"], full["raw_image"])
    np.testing.assert_array_equal(bat["raw_totals"], full["raw_totals"])

    # all photons on the oracle, same seed
    om = dict(mu_s=mu_ext, phase="mie" if phase == "mie" else "hg", hg_g=g_or)
    ores = oracle_mod.walk(table=ps_oracle_table, n_photons=N_FULL, nx=256, nz=256, n_radial=128,
                           r_max=R_MAX, seed=1, **om)
    var = oracle_var(ores) + bat["var"]
    zmax, chi2, dof, pv, z = tally_agreement(full["image"], ores["image"], var, ores["image_hits"])
    pop = ores["image_hits"] >= 20
    rel = np.abs(full["image"] - ores["image"])[pop] / ores["image"][pop]
    print("tau=%g %s steps/photon %.4f  zmax %.2f chi2/dof %.1f/%d p %.3g  fp32-vs-fp64 per-bin rel "
          "err median %.2e p99 %.2e max %.2e" % (tau, phase, full["steps"] / N_FULL, zmax, chi2, dof, pv,
                                                 np.median(rel), np.quantile(rel, 0.99), rel.max()))
    assert zmax < 3.0 and pv > 0.01 and dof > 200
    assert abs(full["steps"] - ores["steps"]) <= 1e-5 * ores["steps"]
    rsig = np.sqrt(np.maximum(ores["radial_sq"] - ores["radial"] ** 2 / N_FULL, 0))
    assert np.all(np.abs(full["radial"] - ores["radial"]) <= 3 * np.sqrt(2) * rsig + 1e-6)

    # a sampled photon range on its own, both sides
    m = 200_000
    k = 37_000_000 + int(tau * 1000)
    part = gpu_batches(gpu, med, m, 16, cam, geo, offset=k, seed=1)
    opart = oracle_mod.walk(table=ps_oracle_table, n_photons=m, photon_offset=k, nx=256, nz=256,
                            n_radial=128, r_max=R_MAX, seed=1, **om)
    zmax, chi2, dof, pv, z = tally_agreement(part["image"], opart["image"],
                                             oracle_var(opart) + part["var"], opart["image_hits"])
    assert zmax < 3.0 and pv > 0.01
    assert abs(part["steps"] - opart["steps"]) <= 1e-3 * opart["steps"]


def test_split_ranges_bit_identical(gpu, ps_table):
    med = gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table)
    cam = gpu.Camera(256, 256, 128, R_MAX)
    f = gpu.auto_frac_bits(N_FULL)       # the scale one launch of all photons uses
    a = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    a.run(med, N_FULL, seed=1)
    assert a.image_frac_bits == f == 27
    b = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    b.run(med, 33_333_333, seed=1, image_frac_bits=f)
    b.run(med, N_FULL - 33_333_333, seed=1, photon_offset=33_333_333, accumulate=True)
    a.check()
    b.check()
    ra, rb = a.result(), b.result()
    np.testing.assert_array_equal(ra["raw_image"], rb["raw_image"])
    np.testing.assert_array_equal(ra["raw_totals"], rb["raw_totals"])
