"""Closed forms the CUDA walk must reproduce on its own (no oracle needed):
Beer-Lambert ballistic transmission (Eq. 1), exact weight bookkeeping with
implicit capture (Eq. 16) and roulette, and the single-scattering image."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0


def _run(gpu, med, n, nx=64, nz=64, **kw):
    eng = gpu.Engine(gpu.Camera(nx, nz, 128, 5 * 2 ** 0.5), gpu.Geometry(LX, LY, LZ))
    eng.run(med, n, **kw)
    eng.check()
    return eng.result()


@pytest.mark.parametrize("tau", [1.0, 5.0, 20.0])
@pytest.mark.parametrize("phase", ["table", "hg"])
def test_ballistic_fraction(gpu, ps_table, tau, phase):
    n = 10_000_000
    med = gpu.Medium(tau / LX, 0.0, phase, ps_table.info["g"], ps_table)
    r = _run(gpu, med, n, seed=3)
    p = math.exp(-tau)
    got = r["totals"][6] / n
    assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / n) + 1e-12


@pytest.mark.parametrize("phase", ["table", "hg"])
def test_energy_bookkeeping(gpu, ps_table, phase):
    n = 2_000_000
    g = ps_table.info["g"]
    r = _run(gpu, gpu.Medium(5 / LX, 0.0, phase, g, ps_table), n)
    t = r["raw_totals"]
    assert t[0] + t[1] + t[2] == n << 32          # exact: every escape carries 1.0
    assert t[3] == t[4] == t[5] == 0
    r = _run(gpu, gpu.Medium(4 / LX, 1 / LX, phase, g, ps_table), n, rr_threshold=0.5, rr_survival=0.1)
    t = r["raw_totals"].astype(np.float64)
    total = t[0] + t[1] + t[2] + t[3] + t[4] + t[5]
    # each contribution is rounded once to 2^-32: at most ~1/2 unit per term
    assert abs(total - float(n << 32)) < 4.0 * r["steps"]
    assert t[3] > 0 and t[4] != 0


@pytest.mark.parametrize("mu_a", [0.0, 0.01])
def test_single_scatter_image(gpu, ps_table, mu_a):
    g, tau, n, nx, nz = 0.8667, 2.0, 20_000_000, 32, 16
    mu_ext = tau / LX
    mu_s = mu_ext - mu_a
    r = _run(gpu, gpu.Medium(mu_s, mu_a, "hg", g), n, nx, nz, max_scatter=1)
    img = r["image"]
    assert np.count_nonzero(np.delete(img, nz // 2, axis=0)) == 0
    psr0 = (1 - g * g) / (4 * math.pi * (1 + g * g) ** 1.5)
    c = (mu_s / mu_ext) * psr0 * math.exp(-mu_ext * LY / 2)
    edges = np.arange(nx + 1) * LX / nx
    prob = np.exp(-mu_ext * edges[:-1]) - np.exp(-mu_ext * edges[1:])
    want = n * c * prob
    sigma = c * np.sqrt(n * prob * (1 - prob))
    z = (img[nz // 2] - want) / sigma
    assert np.max(np.abs(z)) < 5.0
    assert float(np.sum(z ** 2)) < nx + 6 * math.sqrt(2 * nx)
