"""Pins for the oracle's reweighted phase table and its gradients at phase
weights w != 1.

The phase function with weights is p_w = p h_w / Z(w): p the table's own
piecewise-constant density, h_w = sum_k w_k phi_k the hat functions' linear
interpolant of the weights, Z(w) = int p h_w. Pinned by:
  * unit weights give back the table itself;
  * closed forms: an isotropic table reweighted by two or three hats has a
    piecewise-quadratic distribution function whose levels solve quadratics;
  * every bin of a reweighted Mie table carries Z(w) / n of p h_w, integrated
    exactly (trapezoids on the merged breakpoints) with numpy;
  * Z(w) = sum_k w_k Z_k with Z_k the hat integrals;
  * gradients: single scattering in closed form (the camera sees every first
    collision at mu_c = 0, so dL/dw_k = L (phi_k(0) / h_w(0) - Z_k / Z(w))
    on every path), the scale invariance sum_k w_k dL/dw_k = 0 on every path,
    and central differences of E[L] over reweighted tables.
"""
import math

import numpy as np
import pytest

LX, LY, LZ = 45.0, 10.0, 10.0
M_PS = complex(1.59 / 1.33, 0.0)
X_PS = 39.26990816987241


@pytest.fixture(scope="module")
def table(oracle_mod):
    return oracle_mod.phase_table(oracle_mod.PHASE_MIE, M_PS, X_PS)


def _isotropic(n):
    omu = 2.0 * (1.0 - np.arange(n + 1) / n)
    return dict(omu=omu, icdf=1.0 - omu)


def _weights(n_w, seed):
    return np.random.default_rng(seed).uniform(0.5, 1.6, n_w)


def test_unit_weights_give_back_the_table(oracle_mod, table):
    for n_w in (2, 7, 64):
        r = oracle_mod.phase_table_reweighted(table, np.ones(n_w))
        np.testing.assert_allclose(r["omu"], table["omu"], rtol=1e-13, atol=1e-16)
        assert r["z"] == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("a,b", [(1.0, 3.0), (2.5, 0.4), (1.0, 1.0)])
def test_isotropic_two_hats_closed_form(oracle_mod, a, b):
    """p = 1/2 on [-1, 1], h = a (1 - t) + b t with t = (mu + 1) / 2: the
    distribution function in t is (a t + (b - a) t^2 / 2) / ((a + b) / 2)."""
    n = 1024
    r = oracle_mod.phase_table_reweighted(_isotropic(n), np.array([a, b]))
    q = np.arange(n + 1) / n
    if a == b:
        t = q
    else:
        t = (-a + np.sqrt(a * a + (b - a) * q * (a + b))) / (b - a)
    np.testing.assert_allclose(r["icdf"], 2.0 * t - 1.0, rtol=0, atol=1e-13)
    assert r["z"] == pytest.approx(0.5 * (a + b), rel=1e-14)


def test_isotropic_three_hats_closed_form(oracle_mod):
    """Three hats: h linear from w0 to w1 on mu in [-1, 0] and from w1 to w2
    on [0, 1]; each half's distribution function is a quadratic."""
    n = 2048
    w0, w1, w2 = 0.7, 2.0, 1.1
    r = oracle_mod.phase_table_reweighted(_isotropic(n), np.array([w0, w1, w2]))
    m1, m2 = 0.25 * (w0 + w1), 0.25 * (w1 + w2)      # masses of the halves (p = 1/2)
    z = m1 + m2
    want = np.empty(n + 1)
    for i in range(n + 1):
        c = z * i / n
        if c <= m1:   # solve 0.5 (w0 s + (w1 - w0) s^2 / 2) = c, s = mu + 1 in [0, 1]
            A, B, s0 = 0.25 * (w1 - w0), 0.5 * w0, -1.0
        else:
            c -= m1
            A, B, s0 = 0.25 * (w2 - w1), 0.5 * w1, 0.0
        s = 2 * c / (B + math.sqrt(B * B + 4 * A * c))   # root of A s^2 + B s - c = 0
        want[i] = s0 + s
    np.testing.assert_allclose(r["icdf"], want, rtol=0, atol=1e-13)
    assert r["z"] == pytest.approx(z, rel=1e-14)


def test_every_reweighted_bin_holds_an_equal_share(oracle_mod, table):
    n_w = 64
    w = _weights(n_w, 1)
    r = oracle_mod.phase_table_reweighted(table, w)
    n = table["omu"].size - 1
    # breakpoints in cos theta: old bin edges, hat nodes, new bin edges
    nodes = -1.0 + 2.0 * np.arange(n_w) / (n_w - 1)
    mu = np.union1d(np.union1d(table["icdf"], nodes), r["icdf"])
    mid = 0.5 * (mu[:-1] + mu[1:])
    j = np.clip(np.searchsorted(table["icdf"], mid, side="right") - 1, 0, n - 1)
    p = (1.0 / n) / (table["omu"][j] - table["omu"][j + 1])
    hmu = np.interp(mu, nodes, w)                       # h_w: the linear interpolant of the weights
    piece = p * 0.5 * (hmu[:-1] + hmu[1:]) * np.diff(mu)  # exact: linear on each piece
    z = piece.sum()
    assert r["z"] == pytest.approx(z, rel=1e-12)
    k = np.clip(np.searchsorted(r["icdf"], mid, side="right") - 1, 0, n - 1)
    mass = np.bincount(k, weights=piece, minlength=n)
    np.testing.assert_allclose(mass, z / n, rtol=1e-9)
    # Z(w) = sum_k w_k Z_k
    assert r["z"] == pytest.approx(float(np.dot(w, oracle_mod.hat_integrals(table, n_w))), rel=1e-12)


def _single(oracle_mod, base, w, n_w, n=200_000, mu_a=0.0):
    nx, nz = 32, 16
    tw = oracle_mod.phase_table_reweighted(base, w)
    adj = np.random.default_rng(5).uniform(-1, 1, (nz, nx))
    res = oracle_mod.adjoint(adj, n_w, w=w, base_table=base, mu_s=2.0 / LX, mu_a=mu_a, table=tw, n_photons=n,
                             nx=nx, nz=nz, max_scatter=1)
    return res, tw


@pytest.mark.parametrize("n_w", [5, 64])
def test_single_scatter_phase_weight_gradient_closed_form(oracle_mod, table, n_w):
    w = _weights(n_w, 2)
    res, tw = _single(oracle_mod, table, w, n_w)
    z = oracle_mod.hat_integrals(table, n_w)
    zw = float(np.dot(w, z))
    h0 = float(np.interp(0.0, -1.0 + 2.0 * np.arange(n_w) / (n_w - 1), w))
    v = res["value"]
    assert v != 0.0
    for k in range(n_w):
        want = v * (oracle_mod.hat(n_w, k, 0.0) / h0 - z[k] / zw)
        assert res["grad"][2 + k] == pytest.approx(want, rel=1e-9, abs=1e-12 * abs(v)), k


@pytest.mark.parametrize("n_w", [3, 8, 64])
def test_scale_invariance_at_other_weights(oracle_mod, table, n_w):
    """p h_{cw} / Z(cw) = p h_w / Z(w), so sum_k w_k dL/dw_k = 0 on every
    path, multiple scattering included."""
    w = _weights(n_w, 3)
    tw = oracle_mod.phase_table_reweighted(table, w)
    adj = np.random.default_rng(3).uniform(0, 1, (16, 16))
    r = oracle_mod.adjoint(adj, n_w, w=w, base_table=table, table=tw, mu_s=10 / LX, mu_a=0.01, n_photons=20_000,
                           nx=16, nz=16, seed=5)
    g = r["grad"][2:]
    assert abs(float(np.dot(w, g))) < 1e-12 * float(np.abs(w * g).sum()) and np.abs(g).sum() > 0


def test_replayed_value_at_other_weights_is_the_walk_functional(oracle_mod, table):
    w = _weights(8, 4)
    tw = oracle_mod.phase_table_reweighted(table, w)
    adj = np.random.default_rng(9).uniform(0, 1, (64, 64))
    kw = dict(mu_s=5 / LX - 0.01, mu_a=0.01, table=tw, n_photons=20_000, nx=64, nz=64, seed=4, rr_threshold=0.05)
    res = oracle_mod.adjoint(adj, 8, w=w, base_table=table, **kw)
    assert res["value"] == pytest.approx(float(np.sum(adj * oracle_mod.walk(**kw)["image"])), rel=1e-12)


def test_gradient_at_other_weights_matches_central_differences(oracle_mod, table):
    """Multiple scattering at w != 1: d/dw_k against a central difference of
    E[L] over tables reweighted at w +- eps e_k, each side estimated from
    independent runs (a new table moves every sampled angle, so common
    random numbers do not help)."""
    n_w = 8
    nx, nz, eps, runs, n_run = 32, 32, 0.2, 5, 4_000_000
    mu_s = 5.0 / LX
    w = _weights(n_w, 6)
    tw = oracle_mod.phase_table_reweighted(table, w)
    adj = np.random.default_rng(4).uniform(0, 1, (nz, nx))
    res = oracle_mod.adjoint(adj, n_w, w=w, base_table=table, table=tw, mu_s=mu_s, n_photons=n_run, nx=nx,
                             nz=nz, seed=7)
    g = res["grad"] / n_run
    sig_g = np.sqrt(np.maximum(res["grad_sq"] / n_run - g ** 2, 0) / n_run)
    z = oracle_mod.hat_integrals(table, n_w)
    zw = float(np.dot(w, z))
    for k in (3, 6):
        sides = []
        for sgn in (+1, -1):
            ws = w.copy()
            ws[k] += sgn * eps
            tk = oracle_mod.phase_table_reweighted(table, ws)
            v = [float(np.sum(adj * oracle_mod.walk(table=tk, mu_s=mu_s, n_photons=n_run, nx=nx, nz=nz,
                                                    seed=2000 + 10 * k + (0 if sgn > 0 else 5) + r)["image"]))
                 / n_run for r in range(runs)]
            sides.append((np.mean(v), np.std(v, ddof=1) / math.sqrt(runs)))
        fd = (sides[0][0] - sides[1][0]) / (2 * eps)
        sig_fd = math.hypot(sides[0][1], sides[1][1]) / (2 * eps)
        # curvature of 1/Z(w) across +- eps (the difference is exact for a quadratic)
        curv = 2 * (eps * z[k] / zw) ** 2 * abs(g[2 + k]) + 1e-3 * abs(g[2 + k])
        print("k %d: adjoint %.5g +- %.2g, central difference %.5g +- %.2g" % (k, g[2 + k], sig_g[2 + k], fd, sig_fd))
        assert abs(g[2 + k] - fd) < 4 * math.hypot(sig_fd, sig_g[2 + k]) + curv, (k, g[2 + k], fd)
