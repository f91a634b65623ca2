"""Pins for the oracle's inverse-CDF table (Sec. 2.6, Sec. 3.1.2, Eq. 10-12).

The table machinery is checked on the Henyey-Greenstein phase function, whose
inverse CDF has a closed form, and on the Mie phase function against an
adaptive quadrature (scipy) of Eq. 9 that does not use the table code.
"""
import numpy as np
import pytest

M_PS = complex(1.59 / 1.33, 0.0)
X_PS = 39.26990816987241


def _hg_inverse(g, xi):
    if g == 0.0:
        return 2 * xi - 1
    q = (1 - g * g) / (1 - g + 2 * g * xi)
    return (1 + g * g - q * q) / (2 * g)


@pytest.mark.parametrize("g", [0.8667, 0.5, 0.0, -0.3, 0.95])
def test_hg_table_matches_closed_form(oracle_mod, g):
    t = oracle_mod.phase_table(oracle_mod.PHASE_HG, hg_g=g)
    xi = np.arange(4097) / 4096.0
    np.testing.assert_allclose(t["icdf"], _hg_inverse(g, xi), rtol=0, atol=1e-10)
    np.testing.assert_allclose(t["omu"], 1.0 - t["icdf"], rtol=0, atol=1e-15)
    assert t["norm"] == pytest.approx(1.0, abs=1e-10)  # Eq. 11 is normalised already
    assert t["g_quad"] == pytest.approx(g, abs=1e-10)


def test_mie_table_levels_by_independent_quadrature(oracle_mod):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    t = oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, X_PS)
    norm = t["norm"]

    def dens(mu):
        return 0.5 * oracle_mod.mie_phase_raw(M_PS, X_PS, np.array([mu]))[0] / norm

    # integrate from the nearer end; split the forward peak finely
    for i in (1, 37, 512, 1500, 2048, 3000, 3900, 4050, 4090, 4095):
        mu_i = t["icdf"][i]
        if i < 2048:
            val, _ = scipy_integrate.quad(dens, -1.0, mu_i, limit=2000, epsabs=1e-13, epsrel=1e-12)
            target = i / 4096.0
        else:
            pts = [p for p in (0.99, 0.999, 0.9999) if p > mu_i]
            val, _ = scipy_integrate.quad(dens, mu_i, 1.0, points=pts or None, limit=4000,
                                          epsabs=1e-13, epsrel=1e-12)
            target = 1.0 - i / 4096.0
        assert val == pytest.approx(target, abs=2e-10), i


def test_mie_table_shape(oracle_mod):
    qe, qs, g = oracle_mod.mie_efficiencies(M_PS, X_PS)
    t = oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, X_PS)
    icdf, omu, pdf = t["icdf"], t["omu"], t["pdf"]
    assert icdf[0] == -1.0 and icdf[-1] == 1.0
    assert np.all(np.diff(icdf) > 0)
    assert np.all(np.diff(omu) < 0)
    np.testing.assert_allclose(omu, 1.0 - icdf, rtol=0, atol=5e-16)  # a few ulps near 2
    # the piecewise-constant density integrates to one
    assert np.sum(pdf * -np.diff(omu)) == pytest.approx(1.0, abs=1e-13)
    # its mean equals g (Eq. 12) up to the discretisation of 4096 bins
    assert t["mean"] == pytest.approx(g, abs=2e-5)
    # strongly forward peaked (Sec. 5.1): half the probability within ~10 degrees,
    # only a few percent scattered backwards
    assert np.degrees(np.arccos(icdf[2048])) < 12.0
    assert np.searchsorted(icdf, 0.0) / 4096 < 0.05


def test_table_rejects_bad_arguments(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.phase_table(oracle_mod.PHASE_HG, hg_g=1.0)
    with pytest.raises(ValueError):
        oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, X_PS, n_fine=1001)
    with pytest.raises(ValueError):
        oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, -1.0)
