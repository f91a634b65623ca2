"""Pins for the oracle's paper-faithful sampling (Sec. 3.1.2): the phase
function at 3000 equally spaced angles, a cumulative distribution over them,
binary search and linear interpolation in theta; and for the walk that uses
it with the paper's cuvette, beam and weight cut (Sec. 3.1.3, Sec. 4.1,
Sec. 4.3).

Independent of the oracle's own arithmetic: the H-G cumulative distribution
in closed form, the isotropic case (exact for the trapezoidal rule after
normalisation), second-order convergence, Gauss-Legendre quadrature of the
Mie density, inversion of the sampler by numpy's forward interpolation, the
single-scatter camera image and the analog count of escaping photons.
"""
import math

import numpy as np
import pytest

M_PS = complex(1.59 / 1.33, 0.0)
X_PS = 39.26990816987241
LX, LY, LZ = 45.0, 10.0, 10.0


def _hg_cdf_theta(g, th):
    """P(scattering angle <= th) for Eq. 11."""
    return 1.0 - (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * np.cos(th)) - 1 / (1 + g))


def test_isotropic_cdf_is_exact(oracle_mod):
    # trapezoid sums of sin on a uniform grid are proportional to the exact
    # integral, so normalisation makes them exact
    c = oracle_mod.paper_cdf(oracle_mod.PHASE_HG, hg_g=0.0, n_theta=3000)
    np.testing.assert_allclose(c["cdf"], 0.5 * (1 - np.cos(c["theta"])), rtol=0, atol=1e-13)
    assert c["cdf"][0] == 0.0 and c["cdf"][-1] == 1.0


@pytest.mark.parametrize("g", [0.5, 0.8667])
def test_hg_cdf_closed_form_and_second_order(oracle_mod, g):
    errs = []
    for n_theta in (1501, 3001):
        c = oracle_mod.paper_cdf(oracle_mod.PHASE_HG, hg_g=g, n_theta=n_theta)
        err = c["cdf"] - _hg_cdf_theta(g, c["theta"])
        errs.append(err)
        assert np.all(np.diff(c["cdf"]) >= 0)
    assert np.max(np.abs(errs[1])) < 1e-5
    # nested grids: the error at the shared nodes falls by 4 per halving
    ratio = np.max(np.abs(errs[0])) / np.max(np.abs(errs[1][::2]))
    assert 3.6 < ratio < 4.4


def test_mie_cdf_against_gauss_legendre(oracle_mod):
    n_theta = 3000
    c = oracle_mod.paper_cdf(oracle_mod.PHASE_MIE, M_PS, X_PS, n_theta=n_theta)
    th = c["theta"]
    # exact-to-rounding integral of (1/2) P sin over each node interval with
    # 12-point Gauss-Legendre (the density is smooth on a 1e-3 rad interval)
    xg, wg = np.polynomial.legendre.leggauss(12)
    a, b = th[:-1], th[1:]
    t = 0.5 * (a + b)[:, None] + 0.5 * (b - a)[:, None] * xg[None, :]
    p = oracle_mod.mie_phase_raw(M_PS, X_PS, np.cos(t.ravel())).reshape(t.shape)
    seg = 0.5 * (b - a) * np.sum(wg[None, :] * 0.5 * p * np.sin(t), axis=1)
    exact = np.concatenate([[0.0], np.cumsum(seg)])
    exact /= exact[-1]
    err = c["cdf"] - exact
    # trapezoid: error O(h^2 F''), the forward peak (width ~1/x) dominates
    assert np.max(np.abs(err)) < 2e-3
    # and it converges at second order
    c2 = oracle_mod.paper_cdf(oracle_mod.PHASE_MIE, M_PS, X_PS, n_theta=2 * (n_theta - 1) + 1)
    err2 = c2["cdf"][::2] - exact
    assert 3.5 < np.max(np.abs(err)) / np.max(np.abs(err2)) < 4.5


@pytest.fixture(scope="module")
def paper_table(oracle_mod):
    return oracle_mod.paper_cdf(oracle_mod.PHASE_MIE, M_PS, X_PS, n_theta=3000)


def test_sampler_inverts_the_interpolated_cdf(oracle_mod, paper_table):
    """The sampled angle theta satisfies CDF(theta) = u1 for the piecewise-
    linear interpolant of the cdf in theta: a wrong interval, a wrong
    interpolation variable or a transposed fraction all fail this."""
    n = 20_000
    big = 1e9
    r = oracle_mod.walk(mu_s=0.1, phase="paper", table=paper_table, lx=big, ly=big, lz=big,
                        n_photons=n, nx=4, nz=4, n_trace=n, n_trace_events=1, max_events=1, seed=3)
    tr = r["trace"][:, 0]
    assert np.all(tr[:, 0] == 0)
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    u = oracle_mod.philox4x32_10(ctr, 3).astype(np.float64)
    u1 = np.floor(u[:, 1] / 512.0) * 2.0 ** -23 + 2.0 ** -24
    # first collision: the photon travelled along +x, so d'_x = cos(theta)
    th = np.arccos(np.clip(tr[:, 4], -1, 1))
    ok = np.sin(th) > 1e-3      # arccos loses digits near 0 and pi
    back = np.interp(th, paper_table["theta"], paper_table["cdf"])
    np.testing.assert_allclose(back[ok], u1[ok], rtol=0, atol=2e-9)
    assert ok.mean() > 0.95


def test_sampled_angles_follow_the_table(oracle_mod, paper_table):
    n = 200_000
    big = 1e9
    r = oracle_mod.walk(mu_s=0.1, phase="paper", table=paper_table, lx=big, ly=big, lz=big,
                        n_photons=n, nx=4, nz=4, n_trace=n, n_trace_events=1, max_events=1, seed=11)
    th = np.arccos(np.clip(r["trace"][:, 0, 4], -1, 1))
    groups = np.arange(0, 3000, 100)
    edges = np.append(paper_table["theta"][groups], np.pi + 1e-12)
    cnt, _ = np.histogram(th, bins=edges)
    mass = np.diff(np.append(paper_table["cdf"][groups], 1.0))
    exp = n * mass
    keep = exp > 20
    chi2 = float(np.sum((cnt[keep] - exp[keep]) ** 2 / exp[keep]))
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_single_scatter_closed_form(oracle_mod, paper_table):
    """First collisions lie on the axis with d = +x (d_y = 0, theta_c = pi/2):
    the order-1 image is (mu_s/mu_ext) p_sr(0) exp(-mu_ext ly/2) P(column)."""
    tau, n, nx, nz, mu_a = 2.0, 400_000, 32, 16, 0.01
    mu_s = tau / LX - mu_a
    mu_ext = mu_s + mu_a
    r = oracle_mod.walk(mu_s=mu_s, mu_a=mu_a, phase="paper", table=paper_table, n_photons=n,
                        nx=nx, nz=nz, max_scatter=1)
    img = r["image"]
    assert np.count_nonzero(np.delete(img, nz // 2, axis=0)) == 0
    # density per radian of the interval holding pi/2, by a centred difference
    # of the interpolated cdf; per unit cos(theta) at theta = pi/2 it is equal
    h = 1e-7
    dens = (np.interp(np.pi / 2 + h, paper_table["theta"], paper_table["cdf"]) -
            np.interp(np.pi / 2 - h, paper_table["theta"], paper_table["cdf"])) / (2 * h)
    c = (mu_s / mu_ext) * dens / (2 * math.pi) * math.exp(-mu_ext * LY / 2)
    edges = np.arange(nx + 1) * LX / nx
    prob = np.exp(-mu_ext * edges[:-1]) - np.exp(-mu_ext * edges[1:])
    want = n * c * prob
    sigma = c * np.sqrt(n * prob * (1 - prob))
    z = (img[nz // 2] - want) / sigma
    assert np.max(np.abs(z)) < 5.0
    assert float(np.sum(z ** 2)) < nx + 6 * math.sqrt(2 * nx)


def test_camera_estimate_matches_analog_count(oracle_mod):
    """The camera density of the paper's table (interval density / sin theta)
    belongs to the distribution the walk samples: the camera image equals an
    analog count of photons leaving y = +ly/2 in a cone around +y."""
    half = 0.15
    cone = math.cos(half)
    omega = 2 * math.pi * (1 - cone)
    t = oracle_mod.paper_cdf(oracle_mod.PHASE_HG, hg_g=0.3, n_theta=3000)
    n = 6_000_000
    r = oracle_mod.walk(mu_s=1.0 / LX, phase="paper", table=t, n_photons=n, nx=8, nz=8, cone_cos=cone)
    nee = r["image"].sum()
    analog = r["totals"][7] / omega
    sig = math.sqrt(r["totals_sq"][7]) / omega
    assert abs(analog - nee) < 4 * sig + 0.02 * nee, (analog, nee, sig)


def test_paper_setup_conserves_weight(oracle_mod, paper_table):
    """30 x 10 x 45 mm cuvette (beam through the 30 mm side, camera across the
    10 mm one), 2.5 mm beam, absorption and the plain cut at w < 0.001:
    every photon's weight ends in exactly one tally."""
    n = 40_000
    r = oracle_mod.walk(mu_s=8 / 30.0, mu_a=0.3, phase="paper", table=paper_table, lx=30.0, ly=10.0,
                        lz=45.0, beam_radius=1.25, n_photons=n, nx=60, nz=90, rr_threshold=1e-3,
                        rr_survival=0.0)
    t = r["totals"]
    assert t[0] + t[1] + t[2] + t[3] + t[4] + t[5] == pytest.approx(n, rel=1e-12)
    assert t[4] > 0          # the cut removed weight, never added any
    assert r["capped"] == 0


def test_paper_walk_rejects_bad_table(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.walk(mu_s=0.1, phase="paper", table=dict(cdf=np.array([0.0, 1.0])))
    with pytest.raises(ValueError):
        oracle_mod.paper_cdf(oracle_mod.PHASE_HG, hg_g=1.0)


def test_camera_density_is_derivative_of_the_interpolated_cdf(oracle_mod, paper_table):
    """Per collision, the camera term uses dCDF/dtheta at theta_c = acos(d_y)
    (from numpy's interpolant) divided by sin(theta_c) and 2 pi."""
    n, ev = 2000, 6
    mu_s = 3 / LX
    r = oracle_mod.walk(mu_s=mu_s, phase="paper", table=paper_table, n_photons=n, nx=16, nz=16,
                        n_trace=n, n_trace_events=ev, seed=5)
    tr = r["trace"]
    th_n, cdf = paper_table["theta"], paper_table["cdf"]
    checked = 0
    for p in range(n):
        d = np.array([1.0, 0.0, 0.0])
        for e in range(ev):
            rec = tr[p, e]
            if rec[0] != 0:
                break
            thc = math.acos(max(-1.0, min(1.0, d[1])))
            j = int(rec[10])
            assert th_n[j] <= thc <= th_n[j + 1] + 1e-15
            if math.sin(thc) > 1e-3:
                # slope of the interpolant on the interval holding theta_c,
                # taken from numpy over the interval's middle half
                lo = th_n[j] + 0.25 * (th_n[j + 1] - th_n[j])
                hi = th_n[j] + 0.75 * (th_n[j + 1] - th_n[j])
                dens = (np.interp(hi, th_n, cdf) - np.interp(lo, th_n, cdf)) / (hi - lo)
                want = rec[7] * dens / math.sin(thc) / (2 * math.pi) * math.exp(-mu_s * (LY / 2 - rec[2]))
                assert rec[8] == pytest.approx(want, rel=1e-7)
                checked += 1
            d = rec[4:7]
    assert checked > 3000
