"""Pins for the oracle's Mie quantities (Sec. 2.2, 2.4, 2.5).

Each test checks the oracle against something other than its own formulas:
Eq. 7-8 evaluated literally at 50 digits with mpmath's Bessel functions, the
Rayleigh closed forms, the optical theorem, the large-particle extinction
limit, exact symmetry identities, and numbers the paper prints.
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
M_PS = complex(1.59 / 1.33, 0.0)  # polystyrene in water, relative index


def _mp_ab(m, x, nmax, dps=50):
    """Eq. 7-8 as printed, with psi_n(z) = sqrt(pi z / 2) J_{n+1/2}(z) and
    xi_n(x) = sqrt(pi x / 2) H1_{n+1/2}(x); primes from psi_n' = psi_{n-1} - n psi_n / z."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    mm = mp.mpc(m.real, m.imag)
    xx = mp.mpf(x)
    z = mm * xx

    def psi(n, t):
        return mp.sqrt(mp.pi * t / 2) * mp.besselj(n + mp.mpf(1) / 2, t)

    def xi(n, t):
        return mp.sqrt(mp.pi * t / 2) * (mp.besselj(n + mp.mpf(1) / 2, t)
                                        + 1j * mp.bessely(n + mp.mpf(1) / 2, t))

    a, b = [], []
    psx_prev, psz_prev, xix_prev = psi(0, xx), psi(0, z), xi(0, xx)
    for n in range(1, nmax + 1):
        psx, psz, xix = psi(n, xx), psi(n, z), xi(n, xx)
        dpsx = psx_prev - n * psx / xx
        dpsz = psz_prev - n * psz / z
        dxix = xix_prev - n * xix / xx
        an = (mm * psz * dpsx - psx * dpsz) / (mm * psz * dxix - xix * dpsz)
        bn = (psz * dpsx - mm * psx * dpsz) / (psz * dxix - mm * xix * dpsz)
        a.append(complex(an))
        b.append(complex(bn))
        psx_prev, psz_prev, xix_prev = psx, psz, xix
    return np.array(a), np.array(b)


@pytest.mark.parametrize("x", [0.1, 1.0, 10.0, 39.26990816987241, 100.0])
@pytest.mark.parametrize("m", [M_PS, complex(1.5, 0.1), complex(1.33, 1e-3)])
def test_ab_match_50_digit_eq7_eq8(oracle_mod, m, x):
    n = oracle_mod.nmax(x)
    a, b = oracle_mod.mie_ab(m, x)
    ra, rb = _mp_ab(m, x, n)
    for got, ref in ((a, ra), (b, rb)):
        err = np.abs(got - ref)
        assert np.all(err <= 1e-9 * np.abs(ref) + 1e-13), (x, m, np.max(err / (np.abs(ref) + 1e-30)))


def test_rayleigh_limit(oracle_mod):
    m, x = complex(1.5, 0.0), 0.01
    qe, qs, g = oracle_mod.mie_efficiencies(m, x)
    alpha = (m * m - 1) / (m * m + 2)
    assert qs == pytest.approx(8.0 / 3.0 * x ** 4 * abs(alpha) ** 2, rel=1e-4)
    assert abs(g) < 1e-3
    mu = np.array([-0.9, -0.5, 0.0, 0.3, 0.8, 1.0])
    p = oracle_mod.mie_phase_raw(m, x, mu)
    # Rayleigh: P proportional to 1 + cos^2
    np.testing.assert_allclose(p / p[2], 1 + mu ** 2, rtol=1e-4)
    # and separately |S1| flat, |S2| proportional to |cos|
    s1, s2 = oracle_mod.mie_s12(m, x, mu)
    np.testing.assert_allclose(np.abs(s1) / np.abs(s1[2]), 1.0, rtol=1e-4)
    # (at 90 degrees the magnetic dipole b_1 ~ x^2 a_1 / 30 is what remains)
    np.testing.assert_allclose(np.abs(s2) / np.abs(s1), np.abs(mu), rtol=1e-4, atol=2e-5)


def test_rayleigh_absorbing_extinction(oracle_mod):
    # small-particle extinction is dominated by absorption: Q_abs ~ 4 x Im(alpha)
    m, x = complex(1.5, 0.2), 0.005
    qe, qs, _ = oracle_mod.mie_efficiencies(m, x)
    alpha = (m * m - 1) / (m * m + 2)
    assert (qe - qs) == pytest.approx(4 * x * alpha.imag, rel=1e-3)


def test_extinction_paradox_large_x(oracle_mod):
    qe, qs, g = oracle_mod.mie_efficiencies(complex(1.5, 0.0), 1000.0)
    assert abs(qe - 2.0) < 0.03
    assert qs == pytest.approx(qe, rel=1e-10)


@pytest.mark.parametrize("x", [0.5, 5.0, 39.26990816987241])
def test_nonabsorbing_qext_equals_qsca(oracle_mod, x):
    qe, qs, _ = oracle_mod.mie_efficiencies(M_PS, x)
    assert qe == pytest.approx(qs, rel=1e-11)


@pytest.mark.parametrize("m", [M_PS, complex(1.5, 0.05)])
@pytest.mark.parametrize("x", [0.7, 8.0, 39.26990816987241, 78.5])
def test_optical_theorem(oracle_mod, m, x):
    """Q_ext = (4/x^2) Re S(0) ties the amplitude sums to Eq. 13."""
    qe, qs, _ = oracle_mod.mie_efficiencies(m, x)
    s1, s2 = oracle_mod.mie_s12(m, x, np.array([1.0]))
    assert 4.0 / x ** 2 * s1[0].real == pytest.approx(qe, rel=1e-11)
    assert s1[0] == pytest.approx(s2[0], rel=1e-12)
    if m.imag > 0:
        assert qe > qs > 0


@pytest.mark.parametrize("x", [0.7, 8.0, 39.26990816987241])
def test_backscatter_identity(oracle_mod, x):
    """pi_n(-1) = -tau_n(-1) makes S1(180 deg) = -S2(180 deg) exactly."""
    s1, s2 = oracle_mod.mie_s12(M_PS, x, np.array([-1.0]))
    assert abs(s1[0] + s2[0]) <= 1e-11 * abs(s1[0])


@pytest.mark.parametrize("m", [M_PS, complex(1.5, 0.02)])
@pytest.mark.parametrize("x", [1.0, 12.0, 39.26990816987241])
def test_normalisation_and_g_two_ways(oracle_mod, m, x):
    """Eq. 10 by quadrature equals the series value x^2 Q_sca / 2, and Eq. 12
    by quadrature equals the series g."""
    qe, qs, g = oracle_mod.mie_efficiencies(m, x)
    t = oracle_mod.phase_table(oracle_mod.PHASE_MIE, m, x)
    assert t["norm"] == pytest.approx(x * x * qs / 2.0, rel=1e-10)
    assert t["g_quad"] == pytest.approx(g, abs=1e-10)


def test_anisotropy_grows_with_size(oracle_mod):
    """Sec. 2.2: forward scattering strengthens as x grows."""
    gs = [oracle_mod.mie_efficiencies(M_PS, x)[2] for x in (0.05, 0.5, 2.0, 10.0, 39.27)]
    assert gs[0] < 0.01
    assert all(b > a for a, b in zip(gs[:3], gs[1:4]))
    assert gs[-1] > 0.8


def test_paper_worked_values(oracle_mod):
    gold = json.load(open(os.path.join(HERE, "golden", "paper_worked_values.json")))
    e = gold["eq14_cross_section"]
    assert oracle_mod.cross_section_mm2(e["q_ext"], e["d_um"]) == pytest.approx(
        e["sigma_mm2"], rel=e["rel_tol"])
    t = gold["table2_size_parameter"]
    x = oracle_mod.size_parameter(t["d_um"], t["n_medium"], t["lambda0_nm"])
    assert abs(x - t["x"]) <= t["abs_tol"]


def test_size_parameter_is_the_wavelength_in_the_medium(oracle_mod):
    """A sphere in a medium of index n at vacuum wavelength lambda0 scatters
    as the same sphere (index relative to the medium) in vacuum at
    lambda0 / n: the size parameter may depend on n and lambda0 only through
    lambda0 / n, and in vacuum it is the circumference over the wavelength."""
    for d, n, lam in ((5.0, 1.33, 532.0), (1.0, 1.5, 633.0), (10.0, 1.0, 400.0)):
        x = oracle_mod.size_parameter(d, n, lam)
        assert x == pytest.approx(oracle_mod.size_parameter(d, 1.0, lam / n), rel=1e-14)
        assert oracle_mod.size_parameter(d, 1.0, lam / n) == pytest.approx(
            oracle_mod.size_parameter(2 * d, 1.0, 2 * lam / n), rel=1e-14)
    assert oracle_mod.size_parameter(1.0, 1.0, 1000.0 * np.pi) == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("m,x", [(M_PS, 10.0), (M_PS, 39.26990816987241), (complex(1.5, 0.1), 39.26990816987241)])
def test_series_is_summed_to_convergence(oracle_mod, m, x):
    """The oracle stops the Mie series after nmax terms; with 40 more terms of
    the 50-digit coefficients (Eq. 7-8) the Eq. 13 sums must not move."""
    n = oracle_mod.nmax(x) + 40
    a, b = _mp_ab(m, x, n)
    k = np.arange(1, n + 1)
    qe_ref = 2.0 / x ** 2 * np.sum((2 * k + 1) * np.real(a + b))
    qs_ref = 2.0 / x ** 2 * np.sum((2 * k + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    qe, qs, _ = oracle_mod.mie_efficiencies(m, x)
    assert qe == pytest.approx(qe_ref, rel=1e-9)
    assert qs == pytest.approx(qs_ref, rel=1e-9)


def test_eq17_optical_depth_roundtrip(oracle_mod):
    qe, _, _ = oracle_mod.mie_efficiencies(M_PS, oracle_mod.size_parameter(5.0, 1.33, 532.0))
    sig = oracle_mod.cross_section_mm2(qe, 5.0)
    n = 5.0 / (sig * 45.0)
    assert oracle_mod.optical_depth(n, sig, 45.0) == pytest.approx(5.0, rel=1e-14)
