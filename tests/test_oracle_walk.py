"""Pins for the oracle's photon walk (Sec. 2.1, Sec. 2.6, Sec. 3.1.3).

Closed forms the walk must reproduce: Beer-Lambert ballistic transmission
(Eq. 1), the single-scattering camera image, exact weight bookkeeping under
implicit capture (Eq. 16) and the weight cut, the mean free path of Eq. 15,
and the camera estimate against a direct (analog) count of escaping photons.
Per-event invariants are checked on traces using the separately pinned
generator.
"""
import math

import numpy as np
import pytest

M_PS = complex(1.59 / 1.33, 0.0)
X_PS = 39.26990816987241
LX, LY, LZ = 45.0, 10.0, 10.0


@pytest.fixture(scope="module")
def mie_table(oracle_mod):
    return oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, X_PS)


def _hg_sr(g, mu):
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


@pytest.mark.parametrize("tau", [1.0, 5.0])
def test_ballistic_beer_lambert(oracle_mod, mie_table, tau):
    n = 400_000
    r = oracle_mod.walk(mu_s=tau / LX, table=mie_table, n_photons=n, nx=16, nz=16)
    p = math.exp(-tau)
    got = r["totals"][6] / n
    assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / n)


@pytest.mark.parametrize("phase", ["mie", "hg"])
def test_energy_conservation(oracle_mod, mie_table, phase):
    n = 50_000
    kw = dict(table=mie_table) if phase == "mie" else dict(phase="hg", hg_g=0.8667)
    r = oracle_mod.walk(mu_s=5 / LX, n_photons=n, nx=16, nz=16, **kw)
    t = r["totals"]
    assert t[0] + t[1] + t[2] == n  # exact: every escaping weight is 1.0
    assert t[3] == 0 and t[4] == 0 and t[5] == 0
    ra = oracle_mod.walk(mu_s=5 / LX, mu_a=0.05, n_photons=n, nx=16, nz=16,
                         rr_threshold=0.05, rr_survival=0.1, **kw)
    ta = ra["totals"]
    assert ta[3] > 0 and ta[4] != 0
    assert ta[0] + ta[1] + ta[2] + ta[3] + ta[4] + ta[5] == pytest.approx(n, rel=1e-12)


@pytest.mark.parametrize("mu_a", [0.0, 0.01])
def test_single_scatter_closed_form(oracle_mod, mu_a):
    """First collisions lie on the beam axis with d = +x, so d_y = 0 and the
    expected order-1 image is (mu_s/mu_ext) p_sr(0) exp(-mu_ext ly/2) times the
    probability of colliding inside each column, all in row nz/2."""
    g, tau, n, nx, nz = 0.8667, 2.0, 400_000, 32, 16
    mu_s = tau / LX - mu_a
    mu_ext = mu_s + mu_a
    r = oracle_mod.walk(mu_s=mu_s, mu_a=mu_a, phase="hg", hg_g=g, n_photons=n, nx=nx, nz=nz,
                        max_scatter=1)
    img = r["image"]
    assert np.count_nonzero(np.delete(img, nz // 2, axis=0)) == 0
    c = (mu_s / mu_ext) * _hg_sr(g, 0.0) * math.exp(-mu_ext * LY / 2)
    edges = np.arange(nx + 1) * LX / nx
    prob = np.exp(-mu_ext * edges[:-1]) - np.exp(-mu_ext * edges[1:])
    want = n * c * prob
    sigma = c * np.sqrt(n * prob * (1 - prob))
    z = (img[nz // 2] - want) / sigma
    assert np.max(np.abs(z)) < 5.0
    chi2 = float(np.sum(z ** 2))
    assert chi2 < nx + 6 * math.sqrt(2 * nx)
    # the rest of the weight is truncated or transmitted
    t = r["totals"]
    assert t[1] + t[5] + t[3] == pytest.approx(n, rel=1e-12)


def test_mirror_symmetry_in_z(oracle_mod, mie_table):
    # odd nz: on-axis collisions (z = 0 exactly) fall inside the centre row
    # instead of on a row edge, where the floor rule would favour the upper row
    n, nx, nz = 200_000, 16, 15
    r = oracle_mod.walk(mu_s=3 / LX, table=mie_table, n_photons=n, nx=nx, nz=nz)
    img, sq = r["image"], r["image_sq"]
    var = (sq - img ** 2 / n) * n / (n - 1)
    top, bot = img[: nz // 2], img[::-1][: nz // 2]
    vt, vb = var[: nz // 2], var[::-1][: nz // 2]
    assert img[nz // 2].sum() > 0
    ok = (vt + vb) > 0
    z = (top - bot)[ok] / np.sqrt((vt + vb)[ok])
    dof = z.size
    assert np.sum(z ** 2) < dof + 6 * math.sqrt(2 * dof)


def test_deterministic_weight_cut(oracle_mod):
    """Paper's cut (w < 0.001, no survival) in a medium unbounded ahead of the
    beam: a photon that stays inside makes exactly k collisions with
    a^k < 0.001 <= a^(k-1), absorbing 1 - a^k and cutting a^k. A nearly forward
    phase function keeps almost all photons from turning back to x = 0; the
    few that do leave there carry weight a^j after j < k collisions."""
    a, mu_ext, n, big = 0.7, 0.5, 3000, 1e9
    k = 1
    while a ** k >= 1e-3:
        k += 1
    r = oracle_mod.walk(mu_s=a * mu_ext, mu_a=(1 - a) * mu_ext, phase="hg", hg_g=0.999,
                        lx=big, ly=big, lz=big, n_photons=n, nx=4, nz=4,
                        rr_threshold=1e-3, rr_survival=0.0, n_trace=n, n_trace_events=k + 2)
    st = r["trace"][:, :, 0]
    n_cut = n_esc = 0
    esc_w = 0.0
    for p in range(n):
        last = int(np.max(np.nonzero(st[p] >= 0)[0]))
        if st[p, last] == 4:
            assert last == k - 1 and np.all(st[p, :last] == 0)
            n_cut += 1
        else:
            assert st[p, last] == 1 and last < k
            n_esc += 1
            esc_w += a ** last
    assert n_esc < 0.05 * n
    t = r["totals"]
    assert t[4] == pytest.approx(n_cut * a ** k, rel=1e-10)
    assert t[0] == pytest.approx(esc_w, rel=1e-10, abs=1e-300)
    assert t[3] == pytest.approx(n - t[4] - t[0], rel=1e-12)
    assert r["steps"] == int(np.sum(st >= 0))


def test_roulette_is_unbiased(oracle_mod):
    """Roulette changes the spread of the estimates, not their expectation:
    with absorption and a threshold most photons reach, the net weight it
    removes averages to zero, and every weight total agrees with the walk
    without roulette (independent seeds, 4 standard errors)."""
    mu_ext, a, n = 5.0 / LX, 0.7, 1_000_000
    kw = dict(mu_s=a * mu_ext, mu_a=(1 - a) * mu_ext, phase="hg", hg_g=0.5, n_photons=n, nx=8, nz=8)
    plain = oracle_mod.walk(rr_threshold=0.0, rr_survival=1.0, seed=3, **kw)
    rr = oracle_mod.walk(rr_threshold=0.3, rr_survival=0.25, seed=4, **kw)
    assert rr["steps"] < 0.97 * plain["steps"]        # roulette ends many walks early

    def mean_se(r, k):
        m = r["totals"][k] / n
        return m, math.sqrt(max(r["totals_sq"][k] / n - m * m, 0.0) / n)

    m, se = mean_se(rr, 4)
    assert se > 0 and abs(m) < 4 * se
    for k in (0, 1, 2, 3):                            # R, T far, T side, absorbed
        (m0, s0), (m1, s1) = mean_se(plain, k), mean_se(rr, k)
        assert abs(m1 - m0) < 4 * math.hypot(s0, s1), (k, m0, m1)


def test_finite_beam_enters_uniformly_over_its_disc(oracle_mod):
    """The top-hat beam: entry points uniform over the disc of radius R at
    x = 0. The first collision keeps the entry point's y and z (the photon
    flies along +x), so rho^2 / R^2 must be uniform on [0, 1) and the polar
    angle uniform on [0, 2 pi)."""
    R, n = 1.25, 40_000
    r = oracle_mod.walk(mu_s=0.5, phase="hg", hg_g=0.3, beam_radius=R, lx=1e9, n_photons=n, nx=4, nz=4,
                        n_trace=n, n_trace_events=1, max_events=1)
    assert np.all(r["trace"][:, 0, 0] == 0)           # every first event is a collision
    y, z = r["trace"][:, 0, 2], r["trace"][:, 0, 3]
    u = (y * y + z * z) / (R * R)
    assert u.max() < 1.0
    for q in (0.1, 0.25, 0.5, 0.75, 0.9):             # the uniform CDF of rho^2 / R^2
        assert abs(np.mean(u < q) - q) < 5 * math.sqrt(q * (1 - q) / n), q
    ang = np.mod(np.arctan2(z, y), 2 * math.pi) / (2 * math.pi)
    for q in (0.25, 0.5, 0.75):
        assert abs(np.mean(ang < q) - q) < 5 * math.sqrt(q * (1 - q) / n), q
    # the entry point is drawn independently of the first flight, whose
    # length x1 makes exp(-mu_ext x1) uniform on (0, 1)
    v = np.exp(-0.5 * r["trace"][:, 0, 1])
    assert abs(np.corrcoef(u, v)[0, 1]) < 5 / math.sqrt(n)
    assert abs(np.corrcoef(ang, v)[0, 1]) < 5 / math.sqrt(n)


@pytest.mark.parametrize("r_max", [2.0, 1.0])
def test_far_face_radial_profile_of_a_transparent_medium(oracle_mod, r_max):
    """Without scattering every photon crosses to the far face at its entry
    point, so the radial profile is the beam disc's share per ring: ring b
    of n_r on [0, r_max) holds ((b+1)^2 - b^2) (r_max/R)^2 / n_r^2 of the
    photons, the last ring also everything beyond r_max; the profile sums to
    the far-face total exactly."""
    R, n, nr = 2.0, 4_000_000, 16
    r = oracle_mod.walk(mu_s=1e-12, phase="hg", hg_g=0.0, beam_radius=R, r_max=r_max, n_radial=nr, n_photons=n,
                        nx=4, nz=4)
    far = r["totals"][1]
    assert r["radial"].sum() == far and far >= n - 2
    b = np.arange(nr)
    p = ((b + 1) ** 2 - b ** 2) / nr ** 2 * (r_max / R) ** 2
    p[-1] += 1 - (r_max / R) ** 2
    z = (r["radial"] - far * p) / np.sqrt(far * p * (1 - p))
    assert np.max(np.abs(z)) < 5
    assert np.sum(z ** 2) < nr + 6 * math.sqrt(2 * nr)


def test_mean_free_path(oracle_mod):
    mu_ext, n = 0.25, 4000
    big = 1e9
    r = oracle_mod.walk(mu_s=mu_ext, phase="hg", hg_g=0.3, lx=big, ly=big, lz=big,
                        n_photons=n, nx=4, nz=4, n_trace=n, n_trace_events=2,
                        max_events=2)
    x1 = r["trace"][:, 0, 1]  # first collision lies on the axis at x = s
    assert abs(x1.mean() - 1 / mu_ext) < 5 * (1 / mu_ext) / math.sqrt(n)
    assert x1.var() == pytest.approx(1 / mu_ext ** 2, rel=0.15)
    # the second flight either leaves through x = 0 or hits the event cap
    assert r["capped"] + r["totals"][0] == n


@pytest.mark.parametrize("mu_a", [0.0, 0.3 / LX])
def test_camera_estimate_matches_analog_count(oracle_mod, mu_a):
    """The summed camera image estimates the radiant intensity leaving the
    y = +ly/2 face along +y; counting escaping photons in a narrow cone around
    +y and dividing by its solid angle estimates the same quantity."""
    half = 0.15
    cone = math.cos(half)
    omega = 2 * math.pi * (1 - cone)
    n = 6_000_000
    r = oracle_mod.walk(mu_s=1.0 / LX - mu_a, mu_a=mu_a, phase="hg", hg_g=0.0, n_photons=n,
                        nx=8, nz=8, cone_cos=cone)
    nee = r["image"].sum()
    analog = r["totals"][7] / omega
    sig = math.sqrt(r["totals_sq"][7]) / omega
    # finite-cone bias from rays that leave through an x face is about 1 %
    assert abs(analog - nee) < 4 * sig + 0.02 * nee, (analog, nee, sig)


def _trace_case(oracle_mod, phase, table):
    n, ev = 300, 32
    kw = dict(table=table) if phase in ("mie", "coarse") else dict(phase="hg", hg_g=0.8667)
    mu_s, mu_a = 10 / LX, 0.02
    r = oracle_mod.walk(mu_s=mu_s, mu_a=mu_a, n_photons=n, nx=64, nz=64, n_trace=n,
                        n_trace_events=ev, seed=7, rr_threshold=1e-3, **kw)
    return r, mu_s, mu_a, n, ev


@pytest.mark.parametrize("phase", ["mie", "hg", "coarse"])
def test_trace_invariants(oracle_mod, mie_table, phase):
    # "coarse": a 16-bin table of the isotropic function, so that every bin,
    # the first and the last included, holds many camera directions
    table = oracle_mod.phase_table(oracle_mod.PHASE_HG, hg_g=0.0, n_bins=16) if phase == "coarse" else mie_table
    r, mu_s, mu_a, n, ev = _trace_case(oracle_mod, phase, table)
    mu_ext = mu_s + mu_a
    tr = r["trace"]
    ctr = np.zeros((n * ev, 4), dtype=np.uint32)
    ctr[:, 0] = np.repeat(np.arange(n), ev)
    ctr[:, 2] = np.tile(np.arange(ev), n)
    u = oracle_mod.philox4x32_10(ctr, 7).astype(np.float64)
    u = (np.floor(u / 512.0) * 2.0 ** -23 + 2.0 ** -24).reshape(n, ev, 4)
    checked = 0
    for p in range(n):
        pos = np.zeros(3)
        d = np.array([1.0, 0.0, 0.0])
        w = 1.0
        for e in range(ev):
            rec = tr[p, e]
            st = int(rec[0])
            if st < 0:
                break
            rp, dp = rec[1:4], rec[4:7]
            step = rp - pos
            s = -math.log(u[p, e, 0]) / mu_ext
            if st == 0 or st in (4, 5):
                # flight of length s along the old direction
                assert np.linalg.norm(step) == pytest.approx(s, rel=1e-12, abs=1e-12)
                assert np.allclose(step, s * d, rtol=0, atol=1e-10)
                assert abs(np.linalg.norm(dp) - 1) < 1e-12
                # Eq. 16
                w_after = w * (mu_s / mu_ext)
                # camera estimate
                if phase == "hg":
                    psr = _hg_sr(0.8667, d[1])
                else:
                    j = int(rec[10])
                    t = table
                    assert t["icdf"][j] <= d[1] <= t["icdf"][j + 1]
                    psr = t["pdf"][j] / (2 * math.pi)
                want = w_after * psr * math.exp(-mu_ext * (LY / 2 - rp[1]))
                assert rec[8] == pytest.approx(want, rel=1e-12)
                ix = min(max(int(math.floor(rp[0] / LX * 64)), 0), 63)
                iz = min(max(int(math.floor((rp[2] + LZ / 2) / LZ * 64)), 0), 63)
                assert int(rec[9]) == iz * 64 + ix
                if st == 0:
                    # the new direction keeps the sampled polar angle
                    if phase == "hg":
                        mu = _hg_inv(0.8667, u[p, e, 1])
                    else:
                        nb = len(table["icdf"]) - 1
                        mu = np.interp(u[p, e, 1] * nb, np.arange(nb + 1), table["icdf"])
                    assert float(np.dot(dp, d)) == pytest.approx(mu, abs=1e-12)
                    if w_after < 1e-3:
                        assert rec[7] == pytest.approx(w_after / 0.1, rel=1e-12)
                    else:
                        assert rec[7] == pytest.approx(w_after, rel=1e-12)
                    checked += 1
                w = rec[7]
                pos, d = rp, dp
                if st != 0:
                    break
            else:
                # escape: the flight is at most s and ends on the named face
                assert np.linalg.norm(step) <= s * (1 + 1e-12)
                if st == 1:
                    assert abs(rp[0]) < 1e-9
                elif st == 2:
                    assert abs(rp[0] - LX) < 1e-9
                else:
                    assert min(abs(abs(rp[1]) - LY / 2), abs(abs(rp[2]) - LZ / 2)) < 1e-9
                assert rec[7] == w
                break
    assert checked > 1000


def _hg_inv(g, xi):
    q = (1 - g * g) / (1 - g + 2 * g * xi)
    return (1 + g * g - q * q) / (2 * g)


def test_isotropic_table_equals_g0(oracle_mod):
    """A table built from g = 0 reproduces the isotropic closed-form walk."""
    t0 = oracle_mod.phase_table(oracle_mod.PHASE_HG, hg_g=0.0)
    a = oracle_mod.walk(mu_s=3 / LX, table=t0, n_photons=20000, nx=16, nz=16)
    b = oracle_mod.walk(mu_s=3 / LX, phase="hg", hg_g=0.0, n_photons=20000, nx=16, nz=16)
    np.testing.assert_allclose(a["image"], b["image"], rtol=1e-9, atol=1e-15)
    np.testing.assert_array_equal(a["totals"][:3], b["totals"][:3])


def test_split_ranges_add_up(oracle_mod, mie_table):
    full = oracle_mod.walk(mu_s=2 / LX, table=mie_table, n_photons=3000, nx=16, nz=16)
    a = oracle_mod.walk(mu_s=2 / LX, table=mie_table, n_photons=1234, nx=16, nz=16)
    b = oracle_mod.walk(mu_s=2 / LX, table=mie_table, n_photons=3000 - 1234, photon_offset=1234,
                        nx=16, nz=16)
    np.testing.assert_allclose(a["image"] + b["image"], full["image"], rtol=1e-12, atol=1e-18)
    assert a["steps"] + b["steps"] == full["steps"]


def test_walk_rejects_bad_arguments(oracle_mod, mie_table):
    with pytest.raises(ValueError):
        oracle_mod.walk(mu_s=-1.0, table=mie_table)
    with pytest.raises(ValueError):
        oracle_mod.walk(mu_s=0.1, phase="hg", hg_g=1.5)
    with pytest.raises(ValueError):
        oracle_mod.walk(mu_s=0.1, table=mie_table, nx=0)


@pytest.mark.parametrize("lz,nz", [(5.6997014, 24), (10.0, 64), (4.2667066, 30), (0.964, 2)])
def test_first_collisions_on_the_axis_fall_in_row_nz_over_2(oracle_mod, lz, nz):
    """The pixel-tie reading: a pencil beam's first collisions lie on z = 0,
    the edge between rows nz/2 - 1 and nz/2, and belong to row nz/2 for every
    cuvette height (with max_scatter = 1 only first collisions add camera
    terms)."""
    r = oracle_mod.walk(mu_s=0.1, phase="hg", hg_g=0.3, lx=20.0, ly=8.0, lz=lz, nx=8, nz=nz, n_photons=2000,
                        seed=3, max_scatter=1)
    rows = r["image"].sum(axis=1)
    assert rows[nz // 2] > 0 and rows.sum() == rows[nz // 2]
