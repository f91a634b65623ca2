"""Pins for the oracle's likelihood-ratio gradients of the camera image.

Closed form: with one collision per photon (max_scatter = 1) the expected
image is (mu_s/mu_ext) p_sr(0) exp(-mu_ext ly/2) (exp(-mu_ext x_j) -
exp(-mu_ext x_{j+1})) in row nz/2 (the first collision lies on the beam axis
with d_y = 0), so d E[L]/d(mu_s, mu_a, w_k) of L = sum adj * image is known
exactly; the estimate must agree within its standard error. For the full
multiple-scattering walk the gradient must agree with a central difference
of the same estimator run with common random numbers.
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


def _expected_single(mu_s, mu_a, psr0, adj_row, nx):
    mu_ext = mu_s + mu_a
    edges = np.arange(nx + 1) * LX / nx
    prob = np.exp(-mu_ext * edges[:-1]) - np.exp(-mu_ext * edges[1:])
    return float(np.sum(adj_row * (mu_s / mu_ext) * psr0 * math.exp(-mu_ext * LY / 2) * prob))


@pytest.mark.parametrize("mu_a", [0.0, 0.01])
def test_single_scatter_gradient_closed_form(oracle_mod, table, mu_a):
    nx, nz, n = 32, 16, 400_000
    mu_s = 2.0 / LX
    rng = np.random.default_rng(5)
    adj = rng.uniform(-1, 1, (nz, nx))
    j0 = int(np.searchsorted(table["icdf"], 0.0, side="right")) - 1
    pdf0 = table["pdf"][j0]
    psr0 = pdf0 / (2 * math.pi)
    res = oracle_mod.adjoint(adj, 64, mu_s=mu_s, mu_a=mu_a, table=table, n_photons=n, nx=nx, nz=nz,
                             max_scatter=1)
    g, g2 = res["grad"], res["grad_sq"]
    sig = np.sqrt(np.maximum(g2 - g ** 2 / n, 0))
    row = adj[nz // 2]
    f = lambda ms, ma: n * _expected_single(ms, ma, psr0, row, nx)
    h = 1e-6
    d_s = (f(mu_s + h, mu_a) - f(mu_s - h, mu_a)) / (2 * h)
    d_a = (f(mu_s, mu_a + h) - f(mu_s, mu_a - h)) / (2 * h) if mu_a > 0 else \
        (f(mu_s, mu_a + h) - f(mu_s, mu_a)) / h
    assert abs(g[0] - d_s) < 4 * sig[0], (g[0], d_s, sig[0])
    assert abs(g[1] - d_a) < 4 * sig[1], (g[1], d_a, sig[1])
    # phase weights: d p_w(0)/d w_k = p(0) (phi_k(0) - Z_k) at w = 1
    z = oracle_mod.hat_integrals(table, 64)
    base = f(mu_s, mu_a)
    for k in range(64):
        want = base * (oracle_mod.hat(64, k, 0.0) - z[k])
        assert abs(g[2 + k] - want) < 4 * sig[2 + k] + 1e-9 * abs(base), (k, g[2 + k], want)
    # the functional itself matches the walk's image
    w = oracle_mod.walk(mu_s=mu_s, mu_a=mu_a, table=table, n_photons=n, nx=nx, nz=nz, max_scatter=1)
    assert res["value"] == pytest.approx(float(np.sum(adj * w["image"])), rel=1e-12)


@pytest.mark.parametrize("beam_radius", [0.0, 1.25])
def test_replay_matches_walk_functional(oracle_mod, table, beam_radius):
    rng = np.random.default_rng(9)
    adj = rng.uniform(0, 1, (64, 64))
    kw = dict(mu_s=5 / LX - 0.01, mu_a=0.01, table=table, n_photons=20_000, nx=64, nz=64, seed=4,
              rr_threshold=0.05, beam_radius=beam_radius)
    res = oracle_mod.adjoint(adj, 64, **kw)
    w = oracle_mod.walk(**kw)
    assert res["value"] == pytest.approx(float(np.sum(adj * w["image"])), rel=1e-12)


def test_gradient_matches_common_random_number_difference(oracle_mod, table):
    """Full walk: likelihood-ratio gradient vs central difference of the
    same estimator with common random numbers (agree in expectation)."""
    nx, nz, n = 32, 32, 300_000
    mu_s, mu_a = 2.0 / LX, 0.01
    rng = np.random.default_rng(2)
    adj = rng.uniform(0, 1, (nz, nx))
    base = dict(table=table, n_photons=n, nx=nx, nz=nz, seed=3)
    res = oracle_mod.adjoint(adj, 0, mu_s=mu_s, mu_a=mu_a, **base)
    g, g2 = res["grad"], res["grad_sq"]
    sig = np.sqrt(np.maximum(g2 - g ** 2 / n, 0))

    def L(ms, ma):
        return float(np.sum(adj * oracle_mod.walk(mu_s=ms, mu_a=ma, **base)["image"]))

    for i, (ms, ma) in enumerate(((mu_s, mu_a), (mu_s, mu_a))):
        h = 1e-3 * (mu_s if i == 0 else mu_a)
        if i == 0:
            fd = (L(mu_s + h, mu_a) - L(mu_s - h, mu_a)) / (2 * h)
        else:
            fd = (L(mu_s, mu_a + h) - L(mu_s, mu_a - h)) / (2 * h)
        # the difference estimator has its own spread: allow both
        assert abs(g[i] - fd) < 5 * sig[i] * math.sqrt(2), (i, g[i], fd, sig[i])


@pytest.mark.parametrize("n_w", [2, 7, 64])
def test_phase_weight_gradient_is_scale_invariant(oracle_mod, table, n_w):
    """The hats sum to one at every cosine, so w -> c w leaves the
    normalised phase function p h_w / Z(w) unchanged: on every path the
    weight derivatives sum to zero (to rounding), whatever the number of
    collisions; and the normalisation integrals Z_k sum to one."""
    assert oracle_mod.hat_integrals(table, n_w).sum() == pytest.approx(1.0, abs=1e-14)
    adj = np.random.default_rng(3).uniform(0, 1, (16, 16))
    r = oracle_mod.adjoint(adj, n_w, table=table, mu_s=10 / LX, mu_a=0.01, n_photons=20_000, nx=16, nz=16,
                           seed=5)
    g = r["grad"][2:]
    assert abs(g.sum()) < 1e-12 * np.abs(g).sum() + 1e-300 and np.abs(g).sum() > 0


def test_phase_weight_gradient_matches_weighted_tables(oracle_mod, table):
    """Multiple scattering: d/dw_k against a central difference of E[L]
    over tables built for p h_w / Z(w) with w_k = 1 +- eps, each side
    estimated from independent runs (changing the table moves every sampled
    angle, so common random numbers do not reduce the spread). Hats with
    small Z_k keep the curvature of 1/Z(w) negligible at this eps."""
    nx, nz, eps, runs, n_run = 32, 32, 0.25, 5, 4_000_000
    mu_s = 5.0 / LX
    rng = np.random.default_rng(4)
    adj = rng.uniform(0, 1, (nz, nx))
    z = oracle_mod.hat_integrals(table, 64)
    res = oracle_mod.adjoint(adj, 64, table=table, mu_s=mu_s, n_photons=n_run, nx=nx, nz=nz, seed=7)
    g = res["grad"] / n_run
    sig_g = np.sqrt(np.maximum(res["grad_sq"] / n_run - g ** 2, 0) / n_run)
    for k in (20, 61):
        sides = []
        for sgn in (+1, -1):
            w = np.ones(64)
            w[k] += sgn * eps
            tw = oracle_mod.phase_table_weighted(M_PS, X_PS, w)
            v = [float(np.sum(adj * oracle_mod.walk(table=tw, mu_s=mu_s, n_photons=n_run, nx=nx, nz=nz,
                                                    seed=1000 + 10 * k + (0 if sgn > 0 else 5) + r)["image"]))
                 / n_run for r in range(runs)]
            sides.append((np.mean(v), np.std(v, ddof=1) / math.sqrt(runs)))
        fd = (sides[0][0] - sides[1][0]) / (2 * eps)
        sig_fd = math.hypot(sides[0][1], sides[1][1]) / (2 * eps)
        curv = 2 * (eps * z[k]) ** 2 * abs(g[2 + k])
        assert abs(g[2 + k] - fd) < 4 * math.hypot(sig_fd, sig_g[2 + k]) + curv, \
            (k, g[2 + k], fd, sig_fd, sig_g[2 + k])
